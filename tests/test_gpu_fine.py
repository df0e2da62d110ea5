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
    pm = rng.uniform(q.dmin, q.dmax, size=(H, W)) if prior else None
    pv = rng.uniform(50, 4000, size=(H, W)) if prior else None
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
