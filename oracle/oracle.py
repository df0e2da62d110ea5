"""ctypes wrapper of the FP64 CPU oracle (spl_oracle.c).

TEST INFRASTRUCTURE: imported only by tests/, by __graft_entry__.smoke() and by the CPU-baseline leg of
bench.py. It never touches the CUDA library and the CUDA library never touches it.

All arrays are numpy; inputs are converted to float64 (counts and IRF taps are exact in float64).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spl_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over pixels). Returns the path of the shared library."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_GNU_SOURCE",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ct.Structure):
    _fields_ = [("T", ct.c_int), ("L", ct.c_int), ("peak", ct.c_int), ("dmin", ct.c_int), ("dmax", ct.c_int),
                ("beta", ct.c_double), ("sigma_rw2", ct.c_double), ("nu", ct.c_double * 9)]


def params(T, L, peak, dmin=None, dmax=None, beta=0.5, sigma_rw2=3.0, nu=None) -> Params:
    """Oracle parameters; dmin/dmax default to the full-support range [peak, T - L + peak]."""
    q = Params()
    q.T, q.L, q.peak = int(T), int(L), int(peak)
    q.dmin = int(peak if dmin is None else dmin)
    q.dmax = int(T - L + peak if dmax is None else dmax)
    q.beta = float(beta)
    q.sigma_rw2 = float(sigma_rw2)
    w = np.zeros(9) if nu is None else np.asarray(nu, np.float64).reshape(9)
    if nu is None:
        w[4] = 1.0
    for k in range(9):
        q.nu[k] = float(w[k])
    return q


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            d = ct.POINTER(ct.c_double)
            u8 = ct.POINTER(ct.c_uint8)
            i32 = ct.POINTER(ct.c_int32)
            P = ct.POINTER(Params)
            L.orc_set_threads.argtypes = [ct.c_int]
            L.orc_set_threads.restype = ct.c_int
            L.orc_check_domain.argtypes = [P]
            L.orc_check_domain.restype = ct.c_int
            L.orc_template_power_sum.argtypes = [P, d, ct.c_int, ct.c_double]
            L.orc_template_power_sum.restype = ct.c_double
            L.orc_cost.argtypes = [P, d, d, ct.c_long, d]
            L.orc_cost_toa.argtypes = [P, d, i32, ct.c_int, d]
            L.orc_posterior.argtypes = [ct.c_int, ct.c_int, d, i32, d, d]
            L.orc_log_mixture.argtypes = [ct.c_int, d, d, d, ct.c_double]
            L.orc_log_mixture.restype = ct.c_double
            L.orc_estimate.argtypes = [P, d, d, ct.c_long, d, d, i32, d, d, d]
            L.orc_filter_step.argtypes = [P, ct.c_int, ct.c_int, d, d, u8, d, d, u8, i32, d, d, d]
            L.orc_intensity_mle.argtypes = [P, d, d, ct.c_int, d, d]
            L.orc_intensity.argtypes = [P, d, d, ct.c_long, d, i32, u8, u8, d, d]
            L.orc_pi_propagate.argtypes = [ct.c_int, ct.c_int, d, d, u8, d]
            L.orc_estimate_fine.argtypes = [P, ct.c_int, d, d, ct.c_long, d, d, i32, d, d, d, d]
            L.orc_log_lik_ratio.argtypes = [P, d, d, ct.c_int, ct.c_double, ct.c_double]
            L.orc_log_lik_ratio.restype = ct.c_double
            L.orc_detect.argtypes = [P, d, d, ct.c_long, d, i32, d, d, u8, d, d, u8, d, d]
            L.orc_estimate_msl.argtypes = [P, ct.c_int, d, d, ct.c_long, d, d, i32, d, d, d, d]
            _lib = L
    return _lib


def _d(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ctype))


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def check_domain(q: Params) -> int:
    return lib().orc_check_domain(ct.byref(q))


def template_power_sum(q: Params, h, d: int, expo: float) -> float:
    h = _d(h)
    return lib().orc_template_power_sum(ct.byref(q), _ptr(h, ct.c_double), int(d), float(expo))


def cost(q: Params, h, z) -> np.ndarray:
    """C[p, k] = C(dmin + k) for histograms z[..., T]."""
    assert check_domain(q) == 0
    h, z = _d(h), _d(z)
    P = z.size // q.T
    D = q.dmax - q.dmin + 1
    C = np.empty((P, D))
    lib().orc_cost(ct.byref(q), _ptr(h, ct.c_double), _ptr(z, ct.c_double), P, _ptr(C, ct.c_double))
    return C.reshape(*z.shape[:-1], D)


def cost_toa(q: Params, h, bins) -> np.ndarray:
    assert check_domain(q) == 0
    h = _d(h)
    y = np.ascontiguousarray(bins, dtype=np.int32)
    D = q.dmax - q.dmin + 1
    C = np.empty(D)
    lib().orc_cost_toa(ct.byref(q), _ptr(h, ct.c_double), _ptr(y, ct.c_int32), int(y.size), _ptr(C, ct.c_double))
    return C


def toa_histogram(T: int, offsets, bins):
    """Histograms of one frame from its photon ToA lists in CSR form (pixel p's photons are
    bins[offsets[p]:offsets[p + 1]]): z_p[t] = the number of its photons in bin t (Sec. II-A, the ToAs binned on the
    N_T bins of Eq. lik_ideal_poisson; the histogram of the histogram form below Eq. beta_div2). Photons outside
    [0, T) are dropped; a pixel whose offsets are not 0 <= b <= e <= len(bins) gets an empty row. Returns
    (z [P][T] int64, flags) with flags bit 0 = a photon was dropped, bit 2 = some pixel's offsets were invalid."""
    off = np.asarray(offsets, dtype=np.int64)
    y = np.asarray(bins, dtype=np.int64)
    P = off.size - 1
    z = np.zeros((P, T), dtype=np.int64)
    flags = 0
    for p in range(P):
        b, e = int(off[p]), int(off[p + 1])
        if not (0 <= b <= e <= y.size):
            flags |= 4
            continue
        yp = y[b:e]
        keep = (yp >= 0) & (yp < T)
        if not keep.all():
            flags |= 1
        z[p] = np.bincount(yp[keep], minlength=T)
    return z, flags


def posterior(ell, dmin: int):
    ell = _d(ell)
    a = np.zeros(1, np.int32)
    mu = np.zeros(1)
    var = np.zeros(1)
    lib().orc_posterior(int(ell.size), int(dmin), _ptr(ell, ct.c_double), _ptr(a, ct.c_int32),
                        _ptr(mu, ct.c_double), _ptr(var, ct.c_double))
    return int(a[0]), float(mu[0]), float(var[0])


def log_mixture(nu, m, s2, d: float) -> float:
    nu, m, s2 = _d(nu), _d(m), _d(s2)
    return lib().orc_log_mixture(int(nu.size), _ptr(nu, ct.c_double), _ptr(m, ct.c_double),
                                 _ptr(s2, ct.c_double), float(d))


def estimate(q: Params, h, z, prior_mu=None, prior_var=None, want_ell=False):
    """Single-frame estimate; returns dict(argmax, mu, var[, ell]) shaped like z[..., :]."""
    assert check_domain(q) == 0
    h, z = _d(h), _d(z)
    shape = z.shape[:-1]
    P = z.size // q.T
    D = q.dmax - q.dmin + 1
    a = np.empty(P, np.int32)
    mu = np.empty(P)
    var = np.empty(P)
    ell = np.empty((P, D)) if want_ell else None
    pm, pv = _d(prior_mu), _d(prior_var)
    lib().orc_estimate(ct.byref(q), _ptr(h, ct.c_double), _ptr(z, ct.c_double), P, _ptr(pm, ct.c_double),
                       _ptr(pv, ct.c_double), _ptr(a, ct.c_int32), _ptr(mu, ct.c_double),
                       _ptr(var, ct.c_double), _ptr(ell, ct.c_double))
    out = dict(argmax=a.reshape(shape), mu=mu.reshape(shape), var=var.reshape(shape))
    if want_ell:
        out["ell"] = ell.reshape(*shape, D)
    return out


def estimate_fine(q: Params, S: int, h, z, prior_mu=None, prior_var=None, want_ell=False, want_cost=False):
    """Single-frame estimate on the fine grid dmin + k/S (continuous IRF by linear interpolation of the taps, the
    template-power term of the beta-divergence kept): dict(argmax_k, mu, var[, ell][, cost]) shaped like z[..., :]."""
    assert check_domain(q) == 0 and S >= 1
    h, z = _d(h), _d(z)
    shape = z.shape[:-1]
    P = z.size // q.T
    Kf = (q.dmax - q.dmin) * S + 1
    a = np.empty(P, np.int32)
    mu = np.empty(P)
    var = np.empty(P)
    ell = np.empty((P, Kf)) if want_ell else None
    cst = np.empty((P, Kf)) if want_cost else None
    pm, pv = _d(prior_mu), _d(prior_var)
    lib().orc_estimate_fine(ct.byref(q), int(S), _ptr(h, ct.c_double), _ptr(z, ct.c_double), P,
                            _ptr(pm, ct.c_double), _ptr(pv, ct.c_double), _ptr(a, ct.c_int32),
                            _ptr(mu, ct.c_double), _ptr(var, ct.c_double), _ptr(ell, ct.c_double),
                            _ptr(cst, ct.c_double))
    out = dict(argmax_k=a.reshape(shape), mu=mu.reshape(shape), var=var.reshape(shape))
    if want_ell:
        out["ell"] = ell.reshape(*shape, Kf)
    if want_cost:
        out["cost"] = cst.reshape(*shape, Kf)
    return out


def estimate_msl(q: Params, h_bands, z_bands, prior_mu=None, prior_var=None, want_ell=False, want_cost=False):
    """Multispectral estimate (Appendix, Eq. div_MSL): h_bands [nb, L], z_bands [nb, H, W, T] (or [nb, P, T]).
    Returns dict(argmax, mu, var[, M][, ell]) shaped like one band's pixels."""
    hb = _d(h_bands).reshape(-1)
    zb = _d(z_bands)
    nb = zb.shape[0]
    shape = zb.shape[1:-1]
    P = int(np.prod(shape))
    D = q.dmax - q.dmin + 1
    L = hb.size // nb
    assert L == q.L, "every band has L taps"
    zf = np.ascontiguousarray(zb.reshape(nb, P, q.T))
    pm = None if prior_mu is None else _d(prior_mu).reshape(-1)
    pv = None if prior_var is None else _d(prior_var).reshape(-1)
    a = np.empty(P, np.int32)
    mu = np.empty(P)
    var = np.empty(P)
    M = np.empty((P, D)) if want_cost else None
    ell = np.empty((P, D)) if want_ell else None
    lib().orc_estimate_msl(ct.byref(q), nb, _ptr(hb, ct.c_double), _ptr(zf, ct.c_double), P, _ptr(pm, ct.c_double),
                           _ptr(pv, ct.c_double), _ptr(a, ct.c_int32), _ptr(mu, ct.c_double), _ptr(var, ct.c_double),
                           _ptr(M, ct.c_double), _ptr(ell, ct.c_double))
    out = dict(argmax=a.reshape(shape), mu=mu.reshape(shape), var=var.reshape(shape))
    if want_cost:
        out["M"] = M.reshape(*shape, D)
    if want_ell:
        out["ell"] = ell.reshape(*shape, D)
    return out


def filter_step(q: Params, h, z, mu_in, var_in, present_in=None, faulty=None, want_ell=False):
    """One frame of the online filter on an [H, W, T] histogram cube; returns dict(argmax, mu, var[, ell])."""
    assert check_domain(q) == 0
    h, z = _d(h), _d(z)
    H, W, T = z.shape
    assert T == q.T
    P = H * W
    D = q.dmax - q.dmin + 1
    a = np.empty(P, np.int32)
    mu = np.empty(P)
    var = np.empty(P)
    ell = np.empty((P, D)) if want_ell else None
    mi, vi = _d(mu_in), _d(var_in)
    pr, fa = _u8(present_in), _u8(faulty)
    lib().orc_filter_step(ct.byref(q), H, W, _ptr(h, ct.c_double), _ptr(z, ct.c_double), _ptr(fa, ct.c_uint8),
                          _ptr(mi, ct.c_double), _ptr(vi, ct.c_double), _ptr(pr, ct.c_uint8),
                          _ptr(a, ct.c_int32), _ptr(mu, ct.c_double), _ptr(var, ct.c_double),
                          _ptr(ell, ct.c_double))
    out = dict(argmax=a.reshape(H, W), mu=mu.reshape(H, W), var=var.reshape(H, W))
    if want_ell:
        out["ell"] = ell.reshape(H, W, D)
    return out


def intensity_mle(q: Params, h, z, dr: int):
    h, z = _d(h), _d(z)
    r = np.zeros(1)
    b = np.zeros(1)
    lib().orc_intensity_mle(ct.byref(q), _ptr(h, ct.c_double), _ptr(z, ct.c_double), int(dr),
                            _ptr(r, ct.c_double), _ptr(b, ct.c_double))
    return float(r[0]), float(b[0])


def intensity(q: Params, h, z, mu, present=None, faulty=None, dr=None):
    """(refl, bg) per pixel, shaped like mu."""
    h, z = _d(h), _d(z)
    shape = np.shape(mu)
    P = z.size // q.T
    m = _d(mu).reshape(-1)
    drr = None if dr is None else np.ascontiguousarray(dr, dtype=np.int32).reshape(-1)
    pr, fa = _u8(present), _u8(faulty)
    r = np.empty(P)
    b = np.empty(P)
    lib().orc_intensity(ct.byref(q), _ptr(h, ct.c_double), _ptr(z, ct.c_double), P, _ptr(m, ct.c_double),
                        _ptr(drr, ct.c_int32), _ptr(pr, ct.c_uint8), _ptr(fa, ct.c_uint8),
                        _ptr(r, ct.c_double), _ptr(b, ct.c_double))
    return r.reshape(shape), b.reshape(shape)


def log_lik_ratio(q: Params, h, z, dr: int, r: float, b: float) -> float:
    """Log-likelihood ratio of Eq. lik_bg_poisson, (r, b) at template position dr against r = 0, b = K/T."""
    return float(lib().orc_log_lik_ratio(ct.byref(q), _ptr(_d(h), ct.c_double), _ptr(_d(z), ct.c_double),
                                         int(dr), float(r), float(b)))


def detect(q: Params, h, z, mu, dmap=None, var=None, pi0=None, faulty=None):
    """Detection surrogate (maximum-point approximation of the Bayes factor at the pseudo-posterior mode dmap,
    with the Occam term of the pseudo-posterior variance var, combined with pi0), then the intensity rule at
    round(mu): dict(pi, llr, present, refl, bg) shaped like mu. dmap None: round(mu); var None: no Occam term."""
    h, z = _d(h), _d(z)
    shape = np.shape(mu)
    P = z.size // q.T
    m = _d(mu).reshape(-1)
    dm = None if dmap is None else np.ascontiguousarray(dmap, dtype=np.int32).reshape(-1)
    vr = None if var is None else _d(var).reshape(-1)
    p0 = None if pi0 is None else _d(pi0).reshape(-1)
    fa = _u8(faulty)
    pi, llr, r, b = (np.empty(P) for _ in range(4))
    pres = np.empty(P, dtype=np.uint8)
    lib().orc_detect(ct.byref(q), _ptr(h, ct.c_double), _ptr(z, ct.c_double), P, _ptr(m, ct.c_double),
                     _ptr(dm, ct.c_int32), _ptr(vr, ct.c_double), _ptr(p0, ct.c_double), _ptr(fa, ct.c_uint8), _ptr(pi, ct.c_double), _ptr(llr, ct.c_double),
                     _ptr(pres, ct.c_uint8), _ptr(r, ct.c_double), _ptr(b, ct.c_double))
    return dict(pi=pi.reshape(shape), llr=llr.reshape(shape), present=pres.reshape(shape), refl=r.reshape(shape),
                bg=b.reshape(shape))


def pi_propagate(nu, pi_in, faulty=None):
    pi = _d(pi_in)
    H, W = pi.shape
    nu = _d(nu).reshape(9)
    fa = _u8(faulty)
    out = np.empty((H, W))
    lib().orc_pi_propagate(H, W, _ptr(nu, ct.c_double), _ptr(pi, ct.c_double), _ptr(fa, ct.c_uint8),
                           _ptr(out, ct.c_double))
    return out


def state_init(q: Params, H: int, W: int):
    """Initial Gaussians of Algorithm 1 (n = 0): the weakly informative flat Gaussian everywhere."""
    mu = np.full((H, W), 0.5 * (q.dmin + q.dmax))
    var = np.full((H, W), (q.dmax - q.dmin) ** 2 / 12.0)
    return mu, var
