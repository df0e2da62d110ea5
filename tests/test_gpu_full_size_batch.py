"""GPU parity of the batched photon-list path at the full size of its workload: the 64 sequences of uneven
geometry (7.05 M pixels per frame) through the tuned persistent launch, compared with the FP64 oracle at sampled
pixels on dependency-cone crops (the crops reproduce the full-image oracle exactly: checked on small sequences on
the host). It runs after the other GPU tests: its inputs alone take about a second of device time and 1 GB."""
import numpy as np
import pytest
import torch

from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close, check_intensity
from test_gpu_batch import DEV, _run

pytestmark = pytest.mark.gpu


def _crop_histograms(off, bins, W, T, y0, y1, x0, x1):
    """Histograms [y1-y0, x1-x0, T] of the crop's pixels from a frame's CSR photon lists."""
    z = np.zeros((y1 - y0, x1 - x0, T))
    for yy in range(y0, y1):
        for xx in range(x0, x1):
            p = yy * W + xx
            z[yy - y0, xx - x0] = np.bincount(bins[off[p]:off[p + 1]], minlength=T)[:T]
    return z


def _crop_oracle(orc, oq, q, y, x, N):
    """The oracle's frames 0..N-1 at pixel (y, x) from a (2N+1)^2 dependency-cone crop (clipped at the edges):
    a list of (mu, var, argmax, ell row, histogram row) per frame. At frame 0 every crop pixel is exact (the flat
    initial state equals the out-of-frame substitute); a pixel at Chebyshev distance >= n from the crop's inner
    border stays exact after frame n."""
    H, W, T = q["H"], q["W"], q["T"]
    y0, y1 = max(0, y - N), min(H, y + N + 1)
    x0, x1 = max(0, x - N), min(W, x + N + 1)
    m, v = orc.state_init(oq, y1 - y0, x1 - x0)
    out = []
    for n in range(N):
        off, bins = q["frames"][n]
        z = _crop_histograms(off, bins, W, T, y0, y1, x0, x1)
        e = orc.filter_step(oq, q["h"], z, m, v, want_ell=True)
        cy, cx = y - y0, x - x0
        out.append((e["mu"][cy, cx], e["var"][cy, cx], e["argmax"][cy, cx],
                    e["ell"].reshape(y1 - y0, x1 - x0, -1)[cy, cx], z[cy, cx]))
        m, v = e["mu"], e["var"]
    return out


def _full_size_batch_inputs(N, device):
    """The 64-sequence photon-list workload at full size: sides 32-512 (square or 2:1), T 512-4096, Gaussian
    (sigma 2-6 bins, taps +-4 sigma) or 48-tap asymmetric IRFs, beta in [0.1, 1], Poisson(3) signal + Poisson(10)
    background photons truncated to 30 per pixel, drawn on the device; the lists are returned on the host."""
    import math
    rng = np.random.default_rng(4)
    gen = torch.Generator(device=device).manual_seed(4)
    seqs = []
    for s in range(64):
        side = int(rng.choice([32, 64, 128, 256, 512]))
        H, W = side, side * (2 if rng.random() < 0.5 else 1)
        T = int(rng.choice([512, 1024, 2048, 4096]))
        if rng.random() < 0.5:
            sig = rng.uniform(2.0, 6.0)
            h, peak = synth.gaussian_irf(sig, int(math.ceil(4 * sig)))
        else:
            h, peak = synth.asymmetric_irf(L=48)
        beta = float(rng.uniform(0.1, 1.0))
        L = len(h)
        sc = synth.moving_scene(H, W, N, peak + 8, T - L + peak - 8, 400 + s)
        hd = torch.from_numpy(h).to(device)
        frames = []
        for n in range(N):
            off, bins = synth.toa_lists_torch(torch.from_numpy(sc.depth[n]).to(device),
                                              torch.tensor(3.0, device=device), 10.0, hd, peak, T, gen)
            frames.append((off.cpu().numpy(), bins.cpu().numpy()))
        seqs.append(dict(H=H, W=W, T=T, h=h, peak=peak, L=L, beta=beta, s2=3.0, nu=synth.cross_weights(0.5),
                         frames=frames))
    return seqs


def test_full_size_batch_sampled(orc):
    """The 64-sequence workload at full size (7.05 M pixels per frame) through two frames of the tuned persistent
    launch, compared with the oracle at three sampled pixels of every sequence (two corners and an interior
    pixel) on dependency-cone crops: depth, moments and intensity at both frames."""
    N = 2
    seqs = _full_size_batch_inputs(N, DEV)
    res, flags, info = _run(seqs, N, tune=True)
    assert flags == 0 and info["units"] > 0
    assert sum(c["units"] for c in info["classes"]) == info["units"]
    pick = np.random.default_rng(41)
    for i, q in enumerate(seqs):
        H, W = q["H"], q["W"]
        oq = orc.params(q["T"], q["L"], q["peak"], beta=q["beta"], sigma_rw2=q["s2"], nu=q["nu"])
        for (y, x) in [(0, 0), (H - 1, W - 1), (int(pick.integers(1, H - 1)), int(pick.integers(1, W - 1)))]:
            p = y * W + x
            for n, (mu, var, am, ell, z) in enumerate(_crop_oracle(orc, oq, q, y, x, N)):
                g = res[n][i]
                what = f"seq {i} ({H}x{W}, T {q['T']}) pixel ({y},{x}) frame {n}"
                check_argmax(g["argmax"][p:p + 1], [am], ell[None, :], oq.dmin, f"{what} argmax")
                check_close(g["mu_out"][p:p + 1], [mu], f"{what} mu")
                check_close(g["var_out"][p:p + 1], [var], f"{what} var", atol=1e-6)
                check_intensity(orc, oq, q["h"], z[None, :], g["mu_out"][p:p + 1], [mu], g["refl"][p:p + 1],
                                g["bg"][p:p + 1])
