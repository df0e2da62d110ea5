"""Seeded synthetic single-photon lidar inputs.

This module draws data from the observation model of Sec. II-A (Eq. lik_bg_poisson: counts per bin are
Poisson with mean r * s(t - d) + b) and builds the instrument responses and scenes the workloads use. It
holds none of the estimator's arithmetic: no beta power, no correlation, no posterior. The same arrays are
handed to the CPU oracle and to the CUDA library, so both sides see identical inputs.

Everything is deterministic given a seed. Sampling runs with torch on whichever device the caller names;
the CPU and CUDA random streams differ, so a test that compares the two implementations generates once and
copies the same tensor to both.

Depths are integer bins: the depth of a surface is the bin where the peak tap of the IRF lands (Sec. II-D
places the surface at the IRF maximum).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

# --------------------------------------------------------------------------------------------------------
# Instrument responses (tabulated, unit sum). The paper's measured IRFs are not available; these stand in
# for the Gaussian IRF of Sec. II-D and for the skewed real ones (a rise and a long tail).
# --------------------------------------------------------------------------------------------------------


def gaussian_irf(sigma: float, half_width: int) -> tuple[np.ndarray, int]:
    """Gaussian sampled at bin centres over taps -half_width..half_width, unit sum. Returns (h, peak)."""
    j = np.arange(-half_width, half_width + 1, dtype=np.float64)
    h = np.exp(-0.5 * (j / sigma) ** 2)
    h /= h.sum()
    return h.astype(np.float32), half_width


def asymmetric_irf(L: int = 48, shape: float = 4.0, scale: float = 1.6, tail_tau: float = 9.0,
                   tail_weight: float = 0.25) -> tuple[np.ndarray, int]:
    """Gamma-shaped rise plus an exponential tail, L taps, unit sum. Returns (h, peak = first maximum)."""
    t = np.arange(L, dtype=np.float64) + 0.5
    rise = t ** (shape - 1.0) * np.exp(-t / scale)
    rise /= rise.max()
    mode = (shape - 1.0) * scale
    tail = np.where(t > mode, np.exp(-(t - mode) / tail_tau), 0.0)
    h = rise + tail_weight * tail
    h /= h.sum()
    h = h.astype(np.float32)
    return h, int(np.argmax(h))


def band_irfs(nb: int, L: int = 48, peak: int = 12) -> np.ndarray:
    """nb asymmetric IRFs of different widths and tails (one per spectral band), each L taps with its maximum moved
    to tap `peak` (zero-padded on the left or cut on the right, then unit sum). Returns [nb, L] float32."""
    out = np.zeros((nb, L), np.float32)
    for b in range(nb):
        h, pk = asymmetric_irf(L=L, shape=3.0 + 0.7 * b, scale=1.2 + 0.35 * b, tail_tau=6.0 + 3.0 * b,
                               tail_weight=0.15 + 0.1 * b)
        h = h.astype(np.float64)
        g = np.zeros(L)
        sh = peak - pk
        if sh >= 0:
            g[sh:] = h[:L - sh]
        else:
            g[:L + sh] = h[-sh:]
        g /= g.sum()
        out[b] = g.astype(np.float32)
        assert int(np.argmax(out[b])) == peak
    return out


def stretched_irf(h: np.ndarray, L_new: int) -> tuple[np.ndarray, int]:
    """Resample an IRF onto L_new taps (linear interpolation), unit sum."""
    x_old = np.linspace(0.0, 1.0, len(h))
    x_new = np.linspace(0.0, 1.0, L_new)
    g = np.interp(x_new, x_old, h.astype(np.float64))
    g = np.clip(g, 0.0, None)
    g /= g.sum()
    g = g.astype(np.float32)
    return g, int(np.argmax(g))


# --------------------------------------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------------------------------------


def smooth_depth_map(H: int, W: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Sum of 4 random 2-D Gaussians, affinely rescaled to [lo, hi] and rounded to integer bins."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    f = np.zeros((H, W))
    side = max(H, W)
    for _ in range(4):
        a = rng.uniform(0.5, 1.5)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        s = rng.uniform(side / 8.0, side / 3.0)
        f += a * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    return np.rint(lo + f * (hi - lo)).astype(np.int64)


@dataclasses.dataclass
class MovingScene:
    """Static tilted background plane plus moving rectangles/ellipses (the video workload).

    depth[n] and signal[n] are [H, W] maps for frame n: integer depth bin of the IRF peak and the mean number
    of signal photons. The objects translate 1-3 pixels and 5-20 bins per frame and bounce off the bounds.
    """

    depth: np.ndarray   # [N, H, W] int64
    signal: np.ndarray  # [N, H, W] float64
    dlo: int
    dhi: int
    plane: np.ndarray = None  # [H, W] int64: the background plane's depth bin (where no object covers a pixel)

    def static_mask(self, n: int) -> np.ndarray:
        """Pixels that show the background plane in every frame 0 .. n (no object ever covered them)."""
        return np.all(self.depth[:n + 1] == self.plane, axis=0)

    def object_mask(self, n: int) -> np.ndarray:
        """Pixels covered by a moving object in frame n."""
        return self.depth[n] != self.plane


def moving_scene(H: int, W: int, N: int, dlo: int, dhi: int, seed: int, n_objects: int = 3,
                 signal_levels=(1.0, 5.0)) -> MovingScene:
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    span = dhi - dlo
    plane0 = dlo + 0.75 * span
    ty, tx = rng.uniform(-0.05, 0.05, size=2) * span / max(H, W)
    plane = np.clip(plane0 + ty * (yy - H / 2) + tx * (xx - W / 2), dlo, dhi)
    plane_sig = rng.uniform(*signal_levels)
    objs = []
    for _ in range(n_objects):
        objs.append(dict(
            kind=rng.integers(0, 2),
            cy=rng.uniform(0.2 * H, 0.8 * H), cx=rng.uniform(0.2 * W, 0.8 * W),
            ry=rng.uniform(0.08, 0.2) * H, rx=rng.uniform(0.08, 0.2) * W,
            vy=rng.choice([-1, 1]) * rng.uniform(1, 3), vx=rng.choice([-1, 1]) * rng.uniform(1, 3),
            d=rng.uniform(dlo + 0.1 * span, dlo + 0.6 * span),
            vd=rng.choice([-1, 1]) * rng.uniform(5, 20),
            sig=rng.uniform(*signal_levels),
        ))
    depth = np.empty((N, H, W), np.int64)
    signal = np.empty((N, H, W), np.float64)
    for n in range(N):
        d = plane.copy()
        s = np.full((H, W), plane_sig)
        for o in objs:
            if o["kind"] == 0:
                m = (np.abs(yy - o["cy"]) <= o["ry"]) & (np.abs(xx - o["cx"]) <= o["rx"])
            else:
                m = ((yy - o["cy"]) / o["ry"]) ** 2 + ((xx - o["cx"]) / o["rx"]) ** 2 <= 1.0
            d[m] = o["d"]
            s[m] = o["sig"]
        depth[n] = np.clip(np.rint(d), dlo, dhi).astype(np.int64)
        signal[n] = s
        for o in objs:  # advance and reflect at the bounds
            for k, v, lim in (("cy", "vy", H), ("cx", "vx", W)):
                o[k] += o[v]
                if o[k] < 0 or o[k] > lim - 1:
                    o[v] = -o[v]
                    o[k] = min(max(o[k], 0.0), lim - 1.0)
            o["d"] += o["vd"]
            if o["d"] < dlo or o["d"] > dhi:
                o["vd"] = -o["vd"]
                o["d"] = min(max(o["d"], dlo), dhi)
    return MovingScene(depth, signal, dlo, dhi, np.clip(np.rint(plane), dlo, dhi).astype(np.int64))


# --------------------------------------------------------------------------------------------------------
# Photon counts from Eq. lik_bg_poisson
# --------------------------------------------------------------------------------------------------------


def expected_counts(depth: torch.Tensor, signal: torch.Tensor, bg_per_bin, h: torch.Tensor, peak: int,
                    T: int) -> torch.Tensor:
    """Mean histogram r * h[t - d + peak] + b for every pixel: [..., T] float32 on depth's device."""
    L = h.numel()
    dev = depth.device
    t = torch.arange(T, device=dev)
    j = t.view(*([1] * depth.dim()), T) - depth.unsqueeze(-1) + peak          # tap index per bin
    inside = (j >= 0) & (j < L)
    tmpl = torch.where(inside, h.to(dev)[j.clamp(0, L - 1)], torch.zeros((), device=dev))
    bg = torch.as_tensor(bg_per_bin, dtype=torch.float32, device=dev)
    if bg.dim() > 0:
        bg = bg.unsqueeze(-1)
    return signal.to(torch.float32).unsqueeze(-1) * tmpl + bg


def poisson_histograms(mean: torch.Tensor, gen: torch.Generator, dtype=torch.uint16,
                       max_count: int | None = None) -> torch.Tensor:
    """Poisson draw of every bin; stored as uint16 (or float16) counts. Counts above max_count are clipped."""
    z = torch.poisson(mean, generator=gen)
    if max_count is not None:
        z = z.clamp_(max=max_count)
    if dtype == torch.uint16:
        return z.to(torch.int32).to(torch.uint16)
    return z.to(dtype)


def frame_histograms(depth: torch.Tensor, signal: torch.Tensor, bg_per_bin: float, h: torch.Tensor, peak: int,
                     T: int, gen: torch.Generator, pitch: int, dtype=torch.float16, chunk: int = 1 << 15,
                     max_count: int = 2048, out: torch.Tensor | None = None) -> torch.Tensor:
    """Poisson histograms of one frame straight into a zero-padded [P, pitch] buffer on depth's device, a chunk
    of pixels at a time (for frames too large for expected_counts): per bin Poisson(bg_per_bin) plus, at bins
    d - peak + j, Poisson(signal * h_j) (the same law as poisson_histograms(expected_counts(...)): a sum of
    independent Poisson counts). Counts above max_count are clipped. `out` ([P, pitch] of dtype) is filled in
    place when given."""
    dev = depth.device
    d = depth.reshape(-1).to(torch.int64)
    r = signal.reshape(-1).to(device=dev, dtype=torch.float32)
    hh = h.to(device=dev, dtype=torch.float32)
    L = hh.numel()
    P = d.numel()
    if out is None:
        out = torch.zeros(P, pitch, dtype=dtype, device=dev)
    elif pitch > T:
        out[:, T:].zero_()
    jj = torch.arange(L, device=dev)
    for p0 in range(0, P, chunk):
        p1 = min(P, p0 + chunk)
        z = torch.poisson(torch.full((p1 - p0, T), float(bg_per_bin), device=dev), generator=gen)
        sig = torch.poisson(r[p0:p1, None] * hh[None, :], generator=gen)
        z.scatter_add_(1, d[p0:p1, None] - peak + jj[None, :], sig)
        out[p0:p1, :T] = z.clamp_(max=max_count).to(dtype)
    return out


def pad_pitch(T: int, elem_bytes: int = 2, align: int = 16) -> int:
    """Row pitch (elements) rounding T up so each pixel's row starts on a 16-byte boundary."""
    per = align // elem_bytes
    return (T + per - 1) // per * per


def pitched(z: torch.Tensor, pitch: int) -> torch.Tensor:
    """Copy [..., T] counts into a zero-padded [..., pitch] buffer (pitch >= T)."""
    T = z.shape[-1]
    if pitch == T:
        return z.contiguous()
    out = torch.zeros(*z.shape[:-1], pitch, dtype=z.dtype, device=z.device)
    out[..., :T] = z
    return out


# --------------------------------------------------------------------------------------------------------
# Photon time-of-arrival lists (the ToA set y of Sec. II-A) in CSR form
# --------------------------------------------------------------------------------------------------------


def toa_lists(depth: np.ndarray, signal: np.ndarray, bg_per_bin: float, h: np.ndarray, peak: int, T: int,
              seed: int, max_photons: int = 30) -> tuple[np.ndarray, np.ndarray]:
    """Per pixel: K_sig ~ Poisson(signal) photons at d - peak + j with j ~ h, K_bg ~ Poisson(b*T) uniform
    photons; at most max_photons kept. Returns (offsets int32 [P+1], bins int32 [nnz]), bins sorted per pixel.
    """
    rng = np.random.default_rng(seed)
    d = depth.reshape(-1)
    s = signal.reshape(-1)
    P = d.size
    ks = rng.poisson(s)
    kb = rng.poisson(bg_per_bin * T, size=P)
    cdf = np.cumsum(h.astype(np.float64))
    cdf /= cdf[-1]
    offsets = np.zeros(P + 1, np.int64)
    chunks = []
    for p in range(P):
        taps = np.searchsorted(cdf, rng.random(ks[p]), side="right")
        sig_bins = d[p] - peak + np.minimum(taps, len(h) - 1)
        bg_bins = rng.integers(0, T, size=kb[p])
        b = np.concatenate([sig_bins, bg_bins])
        b = b[(b >= 0) & (b < T)]
        if b.size > max_photons:
            b = rng.permutation(b)[:max_photons]
        b.sort()
        chunks.append(b)
        offsets[p + 1] = offsets[p] + b.size
    bins = np.concatenate(chunks) if chunks else np.zeros(0, np.int64)
    return offsets.astype(np.int32), bins.astype(np.int32)


def csr_to_histograms(offsets: np.ndarray, bins: np.ndarray, T: int) -> np.ndarray:
    """Histogram (z_t = number of photons in bin t) of each pixel's ToA list: [P, T] uint16."""
    P = offsets.size - 1
    z = np.zeros((P, T), np.uint16)
    pix = np.repeat(np.arange(P), np.diff(offsets))
    np.add.at(z, (pix, bins), 1)
    return z


# --------------------------------------------------------------------------------------------------------
# The paper's fixed parameter values (Sec. IV): M = 5 cross, nu_0 = 0.5, sigma_RW = sqrt(3) bins.
# --------------------------------------------------------------------------------------------------------


def cross_weights(nu0: float = 0.5) -> np.ndarray:
    """3x3 mixture weights of the M = 5 neighbourhood: nu0 at the centre, (1 - nu0)/4 on N, S, E, W."""
    w = np.zeros(9, np.float32)
    w[4] = nu0
    for k in (1, 3, 5, 7):
        w[k] = (1.0 - nu0) / 4.0
    return w


SIGMA_RW2 = 3.0  # sigma_RW = sqrt(3) bins

__all__ = [n for n in dir() if not n.startswith("_") and n not in ("dataclasses", "math", "np", "torch")]


def toa_lists_torch(depth: torch.Tensor, signal: torch.Tensor, bg_total: float, h: torch.Tensor, peak: int, T: int,
                    gen: torch.Generator, max_photons: int = 30):
    """Vectorised photon lists on depth's device: per pixel K_sig ~ Poisson(signal) photons at d - peak + j with
    j drawn from h, K_bg ~ Poisson(bg_total) uniform photons, at most max_photons kept (a uniformly random
    subset), sorted by bin. Returns (offsets int32 [P+1], bins int32 [nnz])."""
    dev = depth.device
    d = depth.reshape(-1).to(torch.int64)
    P = d.numel()
    ks = torch.poisson(signal.reshape(-1).to(torch.float32).expand(P).contiguous(), generator=gen).to(torch.int64)
    kb = torch.poisson(torch.full((P,), float(bg_total), device=dev), generator=gen).to(torch.int64)
    k = ks + kb
    n = int(k.sum())
    pix = torch.repeat_interleave(torch.arange(P, device=dev), k)
    start = torch.cumsum(k, 0) - k
    rank = torch.arange(n, device=dev) - start[pix]
    is_sig = rank < ks[pix]
    cdf = torch.cumsum(h.to(torch.float64), 0)
    cdf = (cdf / cdf[-1]).to(dev)
    u = torch.rand(n, generator=gen, device=dev, dtype=torch.float64)
    tap = torch.searchsorted(cdf, u, right=True).clamp(max=h.numel() - 1)
    sig_bin = d[pix] - peak + tap
    bg_bin = torch.randint(0, T, (n,), generator=gen, device=dev)
    bins = torch.where(is_sig, sig_bin, bg_bin)
    keep = (bins >= 0) & (bins < T)
    pix, bins = pix[keep], bins[keep]
    # random subset of at most max_photons per pixel: order by (pixel, random key), keep the first ones
    key = torch.rand(pix.numel(), generator=gen, device=dev, dtype=torch.float64)
    order = torch.argsort(pix.to(torch.float64) + key)
    pix, bins = pix[order], bins[order]
    cnt = torch.bincount(pix, minlength=P)
    st = torch.cumsum(cnt, 0) - cnt
    r = torch.arange(pix.numel(), device=dev) - st[pix]
    sel = r < max_photons
    pix, bins = pix[sel], bins[sel]
    order = torch.argsort(pix * T + bins)
    bins = bins[order]
    cnt = torch.bincount(pix, minlength=P)
    offsets = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(cnt, 0)
    return offsets.to(torch.int32), bins.to(torch.int32)
