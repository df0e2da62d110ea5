"""Sub-bin depth (spl_depth_estimate_fine) against the FP64 oracle's fine-grid estimate.

Tolerances as in tests/parity.py: argmax identical up to documented near-ties of the oracle's log
pseudo-posterior, mu and var relative 1e-4 (var with a 1e-6 bins^2 floor)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0) if torch.cuda.is_available() else None


def _gpu_hist(z, T, dtype=torch.uint16):
    P = z.reshape(-1, T).shape[0]
    pitch = synth.pad_pitch(T, 2 if dtype != torch.float32 else 4)
    out = torch.zeros(P, pitch, dtype=dtype)
    zz = torch.from_numpy(z.reshape(P, T))
    out[:, :T] = zz.to(torch.int32).to(dtype) if dtype == torch.uint16 else zz.to(dtype)
    return out.to(DEV)


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("S,L,T,dtype,prior", [
    (1, 24, 300, torch.uint16, True),
    (2, 48, 500, torch.uint16, False),
    (4, 48, 700, torch.uint16, True),
    (7, 33, 260, torch.float32, True),
    (3, 128, 400, torch.float16, False),
    (16, 9, 90, torch.uint16, True),
    (2, 128, 8192, torch.uint16, True),  # largest histogram and IRF: 16129 fine candidates, one or two warps per CTA
])
def test_fine_grid_matches_the_oracle(orc, S, L, T, dtype, prior):
    H, W = 3, 11
    rng = np.random.default_rng(S * 100 + L)
    h, peak = synth.asymmetric_irf(L=L) if L > 12 else synth.gaussian_irf(1.5, L // 2)
    q = orc.params(T, len(h), peak, beta=0.45)
    z = rng.poisson(0.4, size=(H, W, T)).astype(np.float64)
    for y in range(H):
        for x in range(W):
            d = int(rng.integers(q.dmin, q.dmax + 1))
            z[y, x, d - peak:d - peak + len(h)] += rng.poisson(12 * h / h.max())
    # the prior as the GPU receives it (FP32), for both sides
    pm = rng.uniform(q.dmin, q.dmax, size=(H, W)).astype(np.float32).astype(np.float64) if prior else None
    pv = rng.uniform(50, 4000, size=(H, W)).astype(np.float32).astype(np.float64) if prior else None
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.45)
    dp = (lambda a: torch.from_numpy(a.astype(np.float32)).to(DEV).reshape(-1)) if prior else (lambda a: None)
    o = spl.spl_depth_estimate_fine(prm, S, _gpu_hist(z, T, dtype), torch.from_numpy(h).to(DEV),
                                    prior_mu=dp(pm) if prior else None, prior_var=dp(pv) if prior else None)
    torch.cuda.synchronize()
    e = orc.estimate_fine(q, S, h, z, prior_mu=pm, prior_var=pv, want_ell=True)
    ties = check_argmax(_np(o["argmax_k"]), e["argmax_k"].reshape(-1), e["ell"].reshape(H * W, -1), 0, "argmax_k")
    assert ties <= 2
    check_close(_np(o["mu"]), e["mu"], "mu")
    check_close(_np(o["var"]), e["var"], "var", atol=1e-6)


def test_one_step_per_bin_equals_the_integer_estimate(orc):
    """S = 1 and spl_depth_estimate compute the same estimate (both within FP32 rounding of the oracle)."""
    H, W, T = 4, 16, 600
    h, peak = synth.asymmetric_irf(L=48)
    rng = np.random.default_rng(9)
    z = rng.poisson(0.1, size=(H, W, T)).astype(np.float64)
    for y in range(H):
        for x in range(W):
            d = int(rng.integers(peak + 50, T - 48 + peak - 50))
            z[y, x, d - peak:d - peak + 48] += rng.poisson(20 * h)
    prm = spl.make_params(H, W, T, 48, peak, beta=0.5)
    zg, hd = _gpu_hist(z, T), torch.from_numpy(h).to(DEV)
    a = spl.spl_depth_estimate(prm, zg, hd, intensity=False)
    b = spl.spl_depth_estimate_fine(prm, 1, zg, hd)
    torch.cuda.synchronize()
    assert np.array_equal(_np(a["argmax"]), _np(b["argmax_k"]) + prm.dmin)
    check_close(_np(b["mu"]), _np(a["mu"]), "mu", rtol=2e-5)
    check_close(_np(b["var"]), _np(a["var"]), "var", rtol=2e-4, atol=1e-6)


def test_fractional_surface_is_resolved_below_one_bin(orc):
    """Surfaces at fractional depths (counts = the template h_c at d*, scaled and rounded, no background): the
    sub-bin argmax resolves the depth well below one bin, where the integer grid keeps its rounding error."""
    H, W, T, S = 8, 32, 400, 8
    # sigma = 4 bins: the dropped constant (the sampled template's power sum) no longer depends on the phase
    h, peak = synth.gaussian_irf(4.0, 16)
    rng = np.random.default_rng(21)
    dstar = rng.uniform(100.0, 300.0, size=(H * W))
    t = np.arange(T)
    hpad = np.concatenate([[0.0], h.astype(np.float64), [0.0]])
    z = np.zeros((H * W, T))
    for p in range(H * W):
        x = t - dstar[p] + peak                          # the continuous template at d*
        z[p] = np.rint(4000.0 * np.interp(x, np.arange(-1, len(h) + 1), hpad, left=0.0, right=0.0))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5)
    zg, hd = _gpu_hist(z, T, torch.float32), torch.from_numpy(h).to(DEV)
    a = spl.spl_depth_estimate(prm, zg, hd, intensity=False)
    b = spl.spl_depth_estimate_fine(prm, S, zg, hd)
    torch.cuda.synchronize()
    rmse_int = np.sqrt(np.mean((_np(a["argmax"]) - dstar) ** 2))
    rmse_fine = np.sqrt(np.mean((prm.dmin + _np(b["argmax_k"]) / S - dstar) ** 2))
    assert rmse_int > 0.2 and rmse_fine < rmse_int / 3


def test_off_centre_posterior_moments(orc):
    """A tall, narrow data peak (2-4 photons in one bin, Gaussian IRF sigma = 1 bin) 2.2-3.2 prior standard
    deviations away from a broad Gaussian prior: the maximiser sits on the peak while most of the mass lies under
    the prior, so the mean is far from the maximiser (m1^2 > 4 var + 1 in fine units for about half the pixels,
    checked on the oracle) and the moments are taken again about the rounded mean."""
    S, T, H, W = 4, 700, 4, 8
    h, peak = synth.gaussian_irf(1.0, 4)
    q = orc.params(T, len(h), peak, beta=0.5)
    rng = np.random.default_rng(77)
    z = np.zeros((H, W, T))
    pm = np.zeros((H, W), np.float32)
    pv = np.zeros((H, W), np.float32)
    for y in range(H):
        for x in range(W):
            d1 = int(rng.integers(q.dmin + 150, q.dmax - 150))
            z[y, x, d1] += int(rng.integers(2, 5))
            sd = float(rng.uniform(60, 110))
            pm[y, x] = d1 + peak + rng.choice([-1, 1]) * rng.uniform(2.2, 3.2) * sd
            pv[y, x] = sd * sd
    e = orc.estimate_fine(q, S, h, z, prior_mu=pm.astype(np.float64), prior_var=pv.astype(np.float64),
                          want_ell=True)
    m1 = (e["mu"].reshape(-1) - q.dmin) * S - e["argmax_k"].reshape(-1)
    far = m1 * m1 > 4 * e["var"].reshape(-1) * S * S + 1
    assert 8 <= far.sum() < H * W  # both branches of the moment pass
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5)
    o = spl.spl_depth_estimate_fine(prm, S, _gpu_hist(z, T, torch.uint16), torch.from_numpy(h).to(DEV),
                                    prior_mu=torch.from_numpy(pm).to(DEV).reshape(-1),
                                    prior_var=torch.from_numpy(pv).to(DEV).reshape(-1))
    torch.cuda.synchronize()
    check_argmax(_np(o["argmax_k"]), e["argmax_k"].reshape(-1), e["ell"].reshape(H * W, -1), 0, "argmax_k")
    check_close(_np(o["mu"]), e["mu"], "mu")
    check_close(_np(o["var"]), e["var"], "var", atol=1e-6)
