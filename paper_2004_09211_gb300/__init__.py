"""Python binding of libspl (include/spl.h): robust single-photon lidar depth estimation and online
spatio-temporal filtering after Legros et al., "Robust 3D reconstruction of dynamic scenes from single-photon
lidar using Beta-divergences" (arXiv 2004.09211), on sm_103a.

The functions below carry the C names and only marshal arguments: they check devices, dtypes and shapes of
torch tensors, allocate outputs with torch when the caller passes none, and hand raw device pointers and the
current CUDA stream to the library. Every step of the computation runs in the library's CUDA kernels; there is
no CPU or PyTorch fallback, and a missing library raises.
"""
from __future__ import annotations

import ctypes as ct

import torch

from . import _abi
from ._abi import (SPL_BATCH_BAD_BIN, SPL_BATCH_TOO_MANY, SPL_HIST_F16, SPL_HIST_F32, SPL_HIST_U16,
                   SPL_MAX_BINS, SPL_MAX_PHOTONS, SPL_MAX_TAPS, SplError, spl_hist, spl_params, spl_seq_frame)

__all__ = ["make_params", "spl_version", "spl_last_error", "spl_depth_cost", "spl_depth_estimate", "spl_depth_estimate_fine",
           "spl_filter_step", "spl_filter_step_fp32", "spl_filter_step_detect", "spl_filter_step_tc", "spl_state_init", "spl_pi_propagate", "spl_batch_create", "spl_batch_destroy",
           "spl_batch_set", "spl_batch_step", "spl_batch_tune", "spl_batch_info", "spl_batch_status",
           "spl_diff_scratch_size", "spl_diff_forward", "spl_diff_backward", "FilterLoss", "spl_depth_cost_tc",
           "spl_tc_status", "SplError",
           "spl_params", "spl_hist", "spl_seq_frame", "load_library", "cross_weights"]

_FMT = {torch.uint16: SPL_HIST_U16, torch.float16: SPL_HIST_F16, torch.float32: SPL_HIST_F32}


def load_library():
    """Load (building first if needed) the CUDA library; returns the ctypes handle."""
    return _abi.load()


def cross_weights(nu0: float = 0.5):
    """The paper's M = 5 neighbourhood weights (Sec. III-A): nu0 at the centre, (1 - nu0)/4 on N, S, E, W."""
    w = [0.0] * 9
    w[4] = nu0
    for k in (1, 3, 5, 7):
        w[k] = (1.0 - nu0) / 4.0
    return w


def make_params(H: int, W: int, T: int, L: int, peak: int, dmin: int | None = None, dmax: int | None = None,
                beta: float = 0.5, sigma_rw2: float = 3.0, nu=None) -> spl_params:
    """spl_params with dmin/dmax defaulting to the full-support range [peak, T - L + peak] and nu to the
    M = 5 cross with nu0 = 0.5."""
    q = spl_params()
    q.H, q.W, q.T, q.L, q.peak = int(H), int(W), int(T), int(L), int(peak)
    q.dmin = int(peak if dmin is None else dmin)
    q.dmax = int(T - L + peak if dmax is None else dmax)
    q.beta = float(beta)
    q.sigma_rw2 = float(sigma_rw2)
    w = cross_weights(0.5) if nu is None else [float(x) for x in (nu.tolist() if hasattr(nu, "tolist") else nu)]
    assert len(w) == 9
    for k in range(9):
        q.nu[k] = w[k]
    return q


def spl_version() -> str:
    return _abi.load().spl_version().decode()


def spl_last_error() -> str:
    m = _abi.load().spl_last_error()
    return m.decode() if m else ""


# ---------------------------------------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------------------------------------


def _P(prm: spl_params) -> int:
    return prm.H * prm.W


def _D(prm: spl_params) -> int:
    return prm.dmax - prm.dmin + 1


def _dev(t: torch.Tensor | None, name: str, dtype, numel: int | None = None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype} (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements (got {t.numel()})")
    return t.data_ptr()


def _hist(prm: spl_params, z: torch.Tensor) -> spl_hist:
    if not isinstance(z, torch.Tensor) or z.device.type != "cuda":
        raise TypeError("z must be a CUDA tensor")
    if z.dtype not in _FMT:
        raise TypeError(f"z must be uint16, float16 or float32 (got {z.dtype})")
    if not z.is_contiguous():
        raise ValueError("z must be contiguous ([..., pitch] rows)")
    pitch = z.shape[-1]
    if z.numel() != _P(prm) * pitch:
        raise ValueError(f"z has {z.numel()} elements; expected H*W*pitch = {_P(prm)}*{pitch}")
    hz = spl_hist()
    hz.fmt = _FMT[z.dtype]
    hz.data = z.data_ptr()
    hz.pitch = pitch
    return hz


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _empty(shape, dtype, like: torch.Tensor):
    return torch.empty(shape, dtype=dtype, device=like.device)


# ---------------------------------------------------------------------------------------------------------
# the C entry points
# ---------------------------------------------------------------------------------------------------------


def spl_depth_cost(prm: spl_params, z: torch.Tensor, h: torch.Tensor, cost: torch.Tensor | None = None,
                   argmax: torch.Tensor | None = None, want_cost: bool = True, stream=None):
    """C(d) for every candidate (Eq. beta_div2, histogram form) and its argmax. Returns (cost, argmax)."""
    P, D = _P(prm), _D(prm)
    if cost is None and want_cost:
        cost = _empty((P, D), torch.float32, z)
    if argmax is None:
        argmax = _empty((P,), torch.int32, z)
    lib = _abi.load()
    hz = _hist(prm, z)
    _abi.check(lib.spl_depth_cost(ct.byref(prm), ct.byref(hz), _dev(h, "h", torch.float32, prm.L),
                                  _dev(cost, "cost", torch.float32, P * D), _dev(argmax, "argmax", torch.int32, P),
                                  _stream(stream)))
    return cost, argmax


def spl_depth_cost_tc(prm: spl_params, z: torch.Tensor, h: torch.Tensor, cost: torch.Tensor | None = None,
                      argmax: torch.Tensor | None = None, want_cost: bool = True, stream=None):
    """C(d) on the tensor cores from FP16 histograms (hi/lo split FP16 operands, FP32 accumulation)."""
    P, D = _P(prm), _D(prm)
    if cost is None and want_cost:
        cost = _empty((P, D), torch.float32, z)
    if argmax is None:
        argmax = _empty((P,), torch.int32, z)
    lib = _abi.load()
    hz = _hist(prm, z)
    _abi.check(lib.spl_depth_cost_tc(ct.byref(prm), ct.byref(hz), _dev(h, "h", torch.float32, prm.L),
                                     _dev(cost, "cost", torch.float32, P * D),
                                     _dev(argmax, "argmax", torch.int32, P), _stream(stream)))
    return cost, argmax


def spl_tc_status() -> int:
    f = ct.c_uint32()
    _abi.check(_abi.load().spl_tc_status(ct.byref(f)))
    return int(f.value)


def spl_depth_estimate(prm: spl_params, z: torch.Tensor, h: torch.Tensor, prior_mu=None, prior_var=None,
                       present=None, intensity: bool = True, out: dict | None = None, stream=None) -> dict:
    """Single-frame pseudo-posterior estimate (Eq. approx_post). Returns dict(argmax, mu, var[, refl, bg])."""
    P = _P(prm)
    o = dict(out or {})
    o.setdefault("argmax", _empty((P,), torch.int32, z))
    o.setdefault("mu", _empty((P,), torch.float32, z))
    o.setdefault("var", _empty((P,), torch.float32, z))
    if intensity:
        o.setdefault("refl", _empty((P,), torch.float32, z))
        o.setdefault("bg", _empty((P,), torch.float32, z))
    lib = _abi.load()
    hz = _hist(prm, z)
    _abi.check(lib.spl_depth_estimate(
        ct.byref(prm), ct.byref(hz), _dev(h, "h", torch.float32, prm.L),
        _dev(prior_mu, "prior_mu", torch.float32, P), _dev(prior_var, "prior_var", torch.float32, P),
        _dev(present, "present", torch.uint8, P), _dev(o["argmax"], "argmax", torch.int32, P),
        _dev(o["mu"], "mu", torch.float32, P), _dev(o["var"], "var", torch.float32, P),
        _dev(o.get("refl"), "refl", torch.float32, P), _dev(o.get("bg"), "bg", torch.float32, P),
        _stream(stream)))
    return o


def spl_depth_estimate_fine(prm: spl_params, S: int, z: torch.Tensor, h: torch.Tensor, prior_mu=None, prior_var=None,
                            out: dict | None = None, stream=None) -> dict:
    """Single-frame estimate on the sub-bin grid dmin + k/S (continuous IRF by linear interpolation of the taps).
    Returns dict(argmax_k, mu, var); argmax_k is the fine index (depth dmin + argmax_k / S)."""
    P = _P(prm)
    o = dict(out or {})
    o.setdefault("argmax_k", _empty((P,), torch.int32, z))
    o.setdefault("mu", _empty((P,), torch.float32, z))
    o.setdefault("var", _empty((P,), torch.float32, z))
    lib = _abi.load()
    hz = _hist(prm, z)
    _abi.check(lib.spl_depth_estimate_fine(
        ct.byref(prm), int(S), ct.byref(hz), _dev(h, "h", torch.float32, prm.L),
        _dev(prior_mu, "prior_mu", torch.float32, P), _dev(prior_var, "prior_var", torch.float32, P),
        _dev(o.get("argmax_k"), "argmax_k", torch.int32, P), _dev(o["mu"], "mu", torch.float32, P),
        _dev(o["var"], "var", torch.float32, P), _stream(stream)))
    return o


def spl_depth_estimate_msl(prm: spl_params, z: torch.Tensor, h: torch.Tensor, prior_mu=None, prior_var=None,
                           want_cost: bool = False, out: dict | None = None, stream=None) -> dict:
    """Multispectral estimate (Appendix, Eq. div_MSL). z: [nbands, P, pitch] (or [nbands, H, W, pitch]) histograms,
    h: [nbands, L] IRFs. Returns dict(argmax, mu, var[, cost])."""
    if not isinstance(z, torch.Tensor) or z.dim() < 2 or not z.is_contiguous():
        raise TypeError("z must be a contiguous CUDA tensor [nbands, ..., pitch]")
    nb = int(z.shape[0])
    P, D = _P(prm), _D(prm)
    if h.numel() != nb * prm.L:
        raise ValueError(f"h must hold nbands * L = {nb} * {prm.L} taps")
    o = dict(out or {})
    o.setdefault("argmax", _empty((P,), torch.int32, z))
    o.setdefault("mu", _empty((P,), torch.float32, z))
    o.setdefault("var", _empty((P,), torch.float32, z))
    if want_cost:
        o.setdefault("cost", _empty((P, D), torch.float32, z))
    hz = _hist(prm, z[0])
    hz.data = z.data_ptr()
    lib = _abi.load()
    _abi.check(lib.spl_depth_estimate_msl(
        ct.byref(prm), nb, ct.byref(hz), _dev(h, "h", torch.float32, nb * prm.L),
        _dev(prior_mu, "prior_mu", torch.float32, P), _dev(prior_var, "prior_var", torch.float32, P),
        _dev(o.get("argmax"), "argmax", torch.int32, P), _dev(o["mu"], "mu", torch.float32, P),
        _dev(o["var"], "var", torch.float32, P), _dev(o.get("cost"), "cost", torch.float32, P * D), _stream(stream)))
    return o


def spl_filter_step(prm: spl_params, z: torch.Tensor, h: torch.Tensor, mu_in: torch.Tensor, var_in: torch.Tensor,
                    present_in=None, faulty=None, present_now=None, intensity: bool = True,
                    out: dict | None = None, stream=None, _entry: str = "spl_filter_step") -> dict:
    """One frame of the online filter (Algorithm 1). Returns dict(mu, var, argmax[, refl, bg])."""
    P = _P(prm)
    o = dict(out or {})
    o.setdefault("mu", _empty((P,), torch.float32, z))
    o.setdefault("var", _empty((P,), torch.float32, z))
    o.setdefault("argmax", _empty((P,), torch.int32, z))
    if intensity:
        o.setdefault("refl", _empty((P,), torch.float32, z))
        o.setdefault("bg", _empty((P,), torch.float32, z))
    lib = _abi.load()
    hz = _hist(prm, z)
    _abi.check(getattr(lib, _entry)(
        ct.byref(prm), ct.byref(hz), _dev(h, "h", torch.float32, prm.L),
        _dev(mu_in, "mu_in", torch.float32, P), _dev(var_in, "var_in", torch.float32, P),
        _dev(present_in, "present_in", torch.uint8, P), _dev(faulty, "faulty", torch.uint8, P),
        _dev(present_now, "present_now", torch.uint8, P),
        _dev(o["mu"], "mu", torch.float32, P), _dev(o["var"], "var", torch.float32, P),
        _dev(o.get("argmax"), "argmax", torch.int32, P),
        _dev(o.get("refl"), "refl", torch.float32, P), _dev(o.get("bg"), "bg", torch.float32, P),
        _stream(stream)))
    return o


def spl_toa_histogram(prm: spl_params, offsets: torch.Tensor, bins: torch.Tensor, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    """uint16 histograms [P][pitch] of one frame from its CSR photon lists (offsets int32 [P + 1], bins uint16):
    z_p[t] = the number of pixel p's photons in bin t. out (optional) sets the pitch (its last dimension);
    by default pitch = T rounded up to a multiple of 8."""
    P = _P(prm)
    if out is None:
        out = _empty((P, (prm.T + 7) // 8 * 8), torch.uint16, offsets)
    pitch = out.shape[-1]
    nph = bins.numel()
    lib = _abi.load()
    _abi.check(lib.spl_toa_histogram(
        ct.byref(prm), _dev(offsets, "offsets", torch.int32, P + 1),
        _dev(bins, "bins", torch.uint16) if nph > 0 else None, nph,
        _dev(out, "out", torch.uint16, P * pitch), pitch, _stream(stream)))
    return out


def spl_toa_status() -> int:
    f = ct.c_uint32()
    _abi.check(_abi.load().spl_toa_status(ct.byref(f)))
    return int(f.value)


def spl_filter_step_detect(prm: spl_params, z: torch.Tensor, h: torch.Tensor, mu_in: torch.Tensor,
                           var_in: torch.Tensor, present_in=None, faulty=None, pi0=None, out: dict | None = None,
                           stream=None) -> dict:
    """spl_filter_step with the presence decision made on the device by the detection surrogate.
    Returns dict(mu, var, argmax, pi, present, refl, bg); present (uint8) can be the next frame's present_in."""
    P = _P(prm)
    o = dict(out or {})
    for k, dt in (("mu", torch.float32), ("var", torch.float32), ("argmax", torch.int32), ("pi", torch.float32),
                  ("present", torch.uint8), ("refl", torch.float32), ("bg", torch.float32)):
        o.setdefault(k, _empty((P,), dt, z))
    lib = _abi.load()
    hz = _hist(prm, z)
    _abi.check(lib.spl_filter_step_detect(
        ct.byref(prm), ct.byref(hz), _dev(h, "h", torch.float32, prm.L),
        _dev(mu_in, "mu_in", torch.float32, P), _dev(var_in, "var_in", torch.float32, P),
        _dev(present_in, "present_in", torch.uint8, P), _dev(faulty, "faulty", torch.uint8, P),
        _dev(pi0, "pi0", torch.float32, P),
        _dev(o["mu"], "mu", torch.float32, P), _dev(o["var"], "var", torch.float32, P),
        _dev(o.get("argmax"), "argmax", torch.int32, P), _dev(o["pi"], "pi", torch.float32, P),
        _dev(o.get("present"), "present", torch.uint8, P),
        _dev(o["refl"], "refl", torch.float32, P), _dev(o["bg"], "bg", torch.float32, P),
        _stream(stream)))
    return o


def spl_filter_step_fp32(prm: spl_params, z: torch.Tensor, h: torch.Tensor, mu_in: torch.Tensor,
                         var_in: torch.Tensor, present_in=None, faulty=None, present_now=None, intensity: bool = True,
                         out: dict | None = None, stream=None) -> dict:
    """spl_filter_step on the FP32 CUDA-core kernel for every histogram format (the plain path)."""
    return spl_filter_step(prm, z, h, mu_in, var_in, present_in, faulty, present_now, intensity, out, stream,
                           _entry="spl_filter_step_fp32")


def spl_filter_step_tc(prm: spl_params, z: torch.Tensor, h: torch.Tensor, mu_in: torch.Tensor, var_in: torch.Tensor,
                       present_in=None, faulty=None, present_now=None, intensity: bool = True,
                       out: dict | None = None, stream=None) -> dict:
    """spl_filter_step with the data term on the tensor cores; z must be FP16 histograms."""
    return spl_filter_step(prm, z, h, mu_in, var_in, present_in, faulty, present_now, intensity, out, stream,
                           _entry="spl_filter_step_tc")


def spl_state_init(prm: spl_params, mu: torch.Tensor | None = None, var: torch.Tensor | None = None,
                   device="cuda", stream=None):
    """Initial Gaussians of Algorithm 1 (the weakly informative Gaussian everywhere). Returns (mu, var)."""
    P = _P(prm)
    if mu is None:
        mu = torch.empty(P, dtype=torch.float32, device=device)
    if var is None:
        var = torch.empty(P, dtype=torch.float32, device=mu.device)
    lib = _abi.load()
    _abi.check(lib.spl_state_init(ct.byref(prm), _dev(mu, "mu", torch.float32, P),
                                  _dev(var, "var", torch.float32, P), _stream(stream)))
    return mu, var


def spl_pi_propagate(prm: spl_params, pi_in: torch.Tensor, faulty=None, pi_out=None, stream=None):
    """Prior presence probabilities for the next frame (Eq. prior_detect). Returns pi_out."""
    P = _P(prm)
    if pi_out is None:
        pi_out = torch.empty_like(pi_in)
    lib = _abi.load()
    _abi.check(lib.spl_pi_propagate(ct.byref(prm), _dev(pi_in, "pi_in", torch.float32, P),
                                    _dev(faulty, "faulty", torch.uint8, P), _dev(pi_out, "pi_out", torch.float32, P),
                                    _stream(stream)))
    return pi_out


# ---------------------------------------------------------------------------------------------------------
# batched photon-list filtering
# ---------------------------------------------------------------------------------------------------------


def spl_batch_create(prms, nslots: int = 1):
    """Plan for len(prms) sequences and nslots frame tables. Returns an opaque handle (int)."""
    arr = (spl_params * len(prms))(*prms)
    h = ct.c_void_p()
    _abi.check(_abi.load().spl_batch_create(arr, len(prms), int(nslots), ct.byref(h)))
    return h.value


def spl_batch_destroy(handle) -> None:
    if handle:
        _abi.load().spl_batch_destroy(handle)


_FRAME_KEYS = {"h": torch.float32, "offsets": torch.int32, "bins": torch.int32, "mu_in": torch.float32,
               "var_in": torch.float32, "present_in": torch.uint8, "faulty": torch.uint8,
               "present_now": torch.uint8, "mu_out": torch.float32, "var_out": torch.float32,
               "argmax": torch.int32, "refl": torch.float32, "bg": torch.float32}


def spl_batch_set(handle, slot: int, frames) -> None:
    """Uploads one frame's device pointers for every sequence (frames: list of dicts of CUDA tensors keyed like
    spl_seq_frame). The tensors must stay alive while steps of this slot may run."""
    arr = (spl_seq_frame * len(frames))()
    for i, fr in enumerate(frames):
        for k, dt in _FRAME_KEYS.items():
            setattr(arr[i], k, _dev(fr.get(k), f"frames[{i}].{k}", dt))
    _abi.check(_abi.load().spl_batch_set(handle, int(slot), arr))


def spl_batch_step(handle, slot: int, stream=None) -> None:
    """One frame of every sequence from table `slot` (asynchronous; capturable in a CUDA graph)."""
    _abi.check(_abi.load().spl_batch_step(handle, int(slot), _stream(stream)))


def spl_batch_tune(handle, slot: int, stream=None) -> None:
    """Times the candidate tile sizes on table `slot` and keeps the fastest (synchronous)."""
    _abi.check(_abi.load().spl_batch_tune(handle, int(slot), _stream(stream)))


def spl_batch_info(handle) -> dict:
    """The plan's tile size and unit count, the launch geometry of its first size class, and under "classes" every
    class's units, CTAs, warps per CTA and longest candidate grid (spl_batch_class_info)."""
    lib = _abi.load()
    v = [ct.c_int() for _ in range(4)]
    _abi.check(lib.spl_batch_info(handle, *[ct.byref(x) for x in v]))
    classes = []
    nclass = 1
    c = 0
    while c < nclass:
        w = [ct.c_int() for _ in range(5)]
        _abi.check(lib.spl_batch_class_info(handle, c, *[ct.byref(x) for x in w]))
        nclass = w[0].value
        classes.append(dict(units=w[1].value, ctas=w[2].value, warps_per_cta=w[3].value,
                            max_candidates=w[4].value))
        c += 1
    return dict(tile=v[0].value, units=v[1].value, ctas=v[2].value, warps_per_cta=v[3].value, classes=classes)


def spl_batch_status(handle) -> int:
    """Reads and clears the device-side condition flags (SPL_BATCH_BAD_BIN, SPL_BATCH_TOO_MANY)."""
    f = ct.c_uint32()
    _abi.check(_abi.load().spl_batch_status(handle, ct.byref(f)))
    return int(f.value)


# ---------------------------------------------------------------------------------------------------------
# differentiable filter
# ---------------------------------------------------------------------------------------------------------


def spl_diff_scratch_size(prm: spl_params) -> int:
    n = ct.c_size_t()
    _abi.check(_abi.load().spl_diff_scratch_size(ct.byref(prm), ct.byref(n)))
    return int(n.value)


def _frames_hist(prm: spl_params, z: torch.Tensor, nframes: int) -> spl_hist:
    if not isinstance(z, torch.Tensor) or z.device.type != "cuda" or z.dtype != torch.uint16 or not z.is_contiguous():
        raise TypeError("z must be a contiguous CUDA uint16 tensor [nframes, P, pitch]")
    if z.numel() != nframes * _P(prm) * z.shape[-1]:
        raise ValueError("z must hold nframes * H * W rows")
    hz = spl_hist()
    hz.fmt = SPL_HIST_U16
    hz.data = z.data_ptr()
    hz.pitch = z.shape[-1]
    return hz


def spl_diff_forward(prm: spl_params, z: torch.Tensor, h: torch.Tensor, tau: float, d_ref=None, mu_states=None,
                     var_states=None, scratch=None, stream=None) -> dict:
    """Forward pass over the frames of z ([nframes, P, pitch] uint16). Returns dict(mu_states, var_states,
    dsoft, loss, scratch); row 0 of the states is initialised here with spl_state_init when not given."""
    nframes = z.shape[0]
    P = _P(prm)
    if mu_states is None:
        mu_states = torch.empty(nframes + 1, P, device=z.device)
        var_states = torch.empty(nframes + 1, P, device=z.device)
        spl_state_init(prm, mu_states[0], var_states[0], stream=stream)
    if scratch is None:
        scratch = torch.empty(spl_diff_scratch_size(prm), dtype=torch.uint8, device=z.device)
    dsoft = torch.empty(nframes, P, device=z.device)
    loss = torch.empty(1, device=z.device) if d_ref is not None else None
    hz = _frames_hist(prm, z, nframes)
    _abi.check(_abi.load().spl_diff_forward(
        ct.byref(prm), nframes, ct.byref(hz), _dev(h, "h", torch.float32, prm.L), float(tau),
        _dev(d_ref, "d_ref", torch.float32, nframes * P), _dev(mu_states, "mu_states", torch.float32),
        _dev(var_states, "var_states", torch.float32), _dev(dsoft, "dsoft", torch.float32),
        _dev(loss, "loss", torch.float32, 1), scratch.data_ptr(), scratch.numel(), _stream(stream)))
    return dict(mu_states=mu_states, var_states=var_states, dsoft=dsoft, loss=loss, scratch=scratch)


def spl_diff_backward(prm: spl_params, z: torch.Tensor, h: torch.Tensor, tau: float, d_ref: torch.Tensor,
                      mu_states: torch.Tensor, var_states: torch.Tensor, scratch=None, stream=None) -> dict:
    """Gradients of the loss with respect to h, beta and nu. Returns dict(grad_h, grad_beta, grad_nu)."""
    nframes = z.shape[0]
    if scratch is None:
        scratch = torch.empty(spl_diff_scratch_size(prm), dtype=torch.uint8, device=z.device)
    gh = torch.empty(prm.L, device=z.device)
    gb = torch.empty(1, device=z.device)
    gn = torch.empty(9, device=z.device)
    hz = _frames_hist(prm, z, nframes)
    _abi.check(_abi.load().spl_diff_backward(
        ct.byref(prm), nframes, ct.byref(hz), _dev(h, "h", torch.float32, prm.L), float(tau),
        _dev(d_ref, "d_ref", torch.float32, nframes * _P(prm)), _dev(mu_states, "mu_states", torch.float32),
        _dev(var_states, "var_states", torch.float32), gh.data_ptr(), gb.data_ptr(), gn.data_ptr(),
        scratch.data_ptr(), scratch.numel(), _stream(stream)))
    return dict(grad_h=gh, grad_beta=gb, grad_nu=gn)


class FilterLoss(torch.autograd.Function):
    """Loss of the differentiable filter as a torch autograd function of (h, beta, nu).

    forward(h [L] float32 CUDA, beta 0-d tensor, nu [9] tensor, z [nframes, P, pitch] uint16, d_ref
    [nframes, P] float32, geometry dict(H, W, T, peak, dmin, dmax, sigma_rw2), tau) -> loss (1-element tensor).
    Both passes run in the library's kernels (spl_diff_forward / spl_diff_backward); the per-frame states are
    the checkpoints the backward pass recomputes from."""

    @staticmethod
    def forward(ctx, h, beta, nu, z, d_ref, geom, tau):
        prm = make_params(geom["H"], geom["W"], geom["T"], h.numel(), geom["peak"], geom.get("dmin"),
                          geom.get("dmax"), beta=float(beta), sigma_rw2=geom.get("sigma_rw2", 3.0),
                          nu=nu.detach().cpu().tolist())
        hh = h.detach().contiguous().float()
        out = spl_diff_forward(prm, z, hh, tau, d_ref=d_ref)
        ctx.save_for_backward(hh, out["mu_states"], out["var_states"])
        ctx.prm, ctx.z, ctx.d_ref, ctx.tau, ctx.scratch = prm, z, d_ref, tau, out["scratch"]
        return out["loss"]

    @staticmethod
    def backward(ctx, gout):
        hh, ms, vs = ctx.saved_tensors
        g = spl_diff_backward(ctx.prm, ctx.z, hh, ctx.tau, ctx.d_ref, ms, vs, scratch=ctx.scratch)
        s = gout.reshape(())
        return g["grad_h"] * s, (g["grad_beta"] * s).reshape(()), g["grad_nu"] * s, None, None, None, None
