"""Comparison rules between the CUDA library (FP32) and the FP64 oracle, shared by the GPU tests.

Tolerances (derived from the arithmetic, stated once here):
  * argmax (an integer decided by floating point): identical, except a documented near-tie: the oracle's
    log pseudo-posterior at the GPU's index is within TIE_REL * max(1, |ell_max|) of the oracle's maximum.
    FP32 sums of <= 128 products carry a relative error of a few 1e-7, so 1e-5 leaves a wide margin while a
    wrong index on any non-flat posterior is still caught.
  * mu, var, C(d), refl, bg: relative 1e-4 (the accuracy target for FP32 results), plus a small absolute floor
    for values that are zero in exact arithmetic: var 1e-6 bins^2, C 1e-6 * max C, bg 1e-5 * K/T,
    refl 1e-5 * K / sum(h).
  * The template position of the intensity MLE is round-half-even(mu): when the oracle's mu lies within
    1e-4 * |mu| of a half-integer, the two sides may round differently, and the oracle's intensity is
    recomputed at the GPU's rounded mu instead (the decision is taken by the GPU's FP32 mu).
"""
import numpy as np

TIE_REL = 1e-5
RTOL = 1e-4


def check_argmax(gpu_idx, orc_idx, ell, dmin, what="argmax"):
    """ell: oracle log pseudo-posterior [P, D] (natural log); indices are depths. Returns #near-ties."""
    gpu_idx = np.asarray(gpu_idx).reshape(-1)
    orc_idx = np.asarray(orc_idx).reshape(-1)
    ell = np.asarray(ell).reshape(gpu_idx.size, -1)
    bad = np.nonzero(gpu_idx != orc_idx)[0]
    ties = 0
    for p in bad:
        k = gpu_idx[p] - dmin
        assert 0 <= k < ell.shape[1], f"{what}[{p}] = {gpu_idx[p]} outside the domain"
        m = ell[p].max()
        gap = m - ell[p, k]
        assert gap <= TIE_REL * max(1.0, abs(m)), \
            f"{what}[{p}]: GPU {gpu_idx[p]} vs oracle {orc_idx[p]}, oracle ell gap {gap:.3g} (max {m:.6g})"
        ties += 1
    return ties


def check_close(gpu, orc, name, rtol=RTOL, atol=0.0):
    gpu = np.asarray(gpu, np.float64).reshape(-1)
    orc = np.asarray(orc, np.float64).reshape(-1)
    assert np.all(np.isfinite(gpu)), f"{name}: non-finite GPU values"
    err = np.abs(gpu - orc)
    tol = rtol * np.abs(orc) + atol
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, (f"{name}: {bad.size} of {gpu.size} outside rtol={rtol} atol={atol}; first {bad[:5]}: "
                           f"gpu {gpu[bad[:5]]} oracle {orc[bad[:5]]}")


def check_intensity(orc_mod, q, h, z, mu_gpu, mu_orc, refl_gpu, bg_gpu, present=None, faulty=None):
    """Compares (refl, bg) with the oracle; near-half template positions follow the GPU's rounding."""
    z = np.asarray(z, np.float64).reshape(-1, q.T)
    mu_orc = np.asarray(mu_orc, np.float64).reshape(-1)
    mu_gpu = np.asarray(mu_gpu, np.float64).reshape(-1)
    dr = np.rint(mu_orc).astype(np.int32)
    frac = np.abs(np.abs(mu_orc - np.floor(mu_orc)) - 0.5)
    near = frac <= 1e-4 * np.maximum(np.abs(mu_orc), 1.0)
    dr[near] = np.rint(mu_gpu[near].astype(np.float32)).astype(np.int32)
    r, b = orc_mod.intensity(q, h, z, mu_orc, present=present, faulty=faulty, dr=dr)
    K = z.sum(axis=1)
    hs = float(np.sum(np.clip(np.asarray(h, np.float64), 0, None)))
    check_close(bg_gpu, b, "bg", atol=1e-5 * K / q.T + 1e-12)
    check_close(refl_gpu, r, "refl", atol=1e-5 * K / hs + 1e-12)
    return int(near.sum())
