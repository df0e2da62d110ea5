"""GPU parity of the pseudo-posterior epilogue (pruning, linear-domain weights, log-domain fallback, recentred
sums) on edge cases, against the FP64 oracle.

Photon-starved rows over long candidate grids put most blocks of 32 candidates out of reach of every photon, so
the prior alone decides which blocks survive the pruning bound. The cases: Gaussian priors with variances from
below 9 to above D^2 bins^2 and means on and just outside the ends of the grid; the maximum inside a block that
no photon reaches (weak data far from a broad prior); a mean more than two standard deviations from the maximum
(the sums taken again about the rounded mean); mixtures of up to nine components from the filter step's stencil;
a flat prior over the longest histogram (255 blocks); and the photon-list form of the batched step. Tolerances as
everywhere (tests/parity.py)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _gpu_hist(z, T):
    t = torch.from_numpy(np.ascontiguousarray(z).reshape(-1, T).astype(np.int32)).to(torch.uint16)
    return synth.pitched(t, synth.pad_pitch(T)).to(DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _sparse_photons(rng, P, T, counts, lo=0, hi=None):
    """[P, T] histograms with counts[p] photons each at uniform bins of [lo, hi)."""
    hi = T if hi is None else hi
    z = np.zeros((P, T))
    for p in range(P):
        for t in rng.integers(lo, hi, size=int(counts[p])):
            z[p, t] += 1.0
    return z


def _estimate_both(orc, h, peak, z, pm, pv, beta, H, W, T):
    f32 = lambda a: None if a is None else np.asarray(a, np.float32).astype(np.float64)  # both sides see FP32 priors
    pm, pv = f32(pm), f32(pv)
    q = orc.params(T, len(h), peak, beta=beta)
    e = orc.estimate(q, h, z.reshape(H, W, T), prior_mu=None if pm is None else pm.reshape(H, W),
                     prior_var=None if pv is None else pv.reshape(H, W), want_ell=True)
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta)
    dv = lambda a: None if a is None else torch.from_numpy(a.astype(np.float32)).to(DEV)
    o = spl.spl_depth_estimate(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV), prior_mu=dv(pm), prior_var=dv(pv))
    torch.cuda.synchronize()
    return q, e, o


def _compare(q, e, o):
    check_argmax(_np(o["argmax"]), e["argmax"], e["ell"], q.dmin)
    check_close(_np(o["mu"]), e["mu"], "mu")
    check_close(_np(o["var"]), e["var"], "var", atol=1e-6)


@pytest.mark.parametrize("beta", [0.2, 0.5, 1.0])
def test_gaussian_prior_edges(orc, beta):
    """128 pixels, T = 2048 (2001 candidates): 0-8 photons each; prior variances log-uniform on [9, D^2] plus the
    limits (8.9, 9, 9.1, 0.99 D^2, 1.01 D^2) and means on the grid's ends (dmin - 0.5, dmin, dmax, dmax + 0.5, and
    dmin - 0.6 just outside)."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 8, 16, 2048
    P = H * W
    dmin, dmax = peak, T - len(h) + peak
    D = dmax - dmin + 1
    rng = np.random.default_rng(int(beta * 1000) + 7)
    z = _sparse_photons(rng, P, T, rng.choice([0, 1, 2, 3, 5, 8], size=P))
    pm = rng.uniform(dmin, dmax, size=P)
    pv = np.exp(rng.uniform(np.log(9.0), np.log(float(D) ** 2), size=P))
    edges_v = [8.9, 9.0, 9.1, 0.99 * D * D, 1.01 * D * D]
    edges_m = [dmin - 0.5, dmin, dmax, dmax + 0.5, dmin - 0.6]
    for i, v in enumerate(edges_v):
        for j, m in enumerate(edges_m):
            k = i * len(edges_m) + j
            pv[k], pm[k] = v, m
    q, e, o = _estimate_both(orc, h, peak, z, pm, pv, beta, H, W, T)
    _compare(q, e, o)


def test_maximum_in_a_block_no_photon_reaches(orc):
    """Weak data (beta = 1, one to three photons) at least 300 bins from a broad prior's mean: the maximum is the
    prior's mode, inside a block that no photon reaches, so the exact search over the prior-only blocks must find
    it."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 4, 8, 1500
    P = H * W
    dmin = peak
    rng = np.random.default_rng(21)
    pm = rng.uniform(dmin + 500, dmin + 900, size=P)
    pv = rng.uniform(5e3, 2e4, size=P)  # broad: about 40 of the 46 blocks are kept, almost all without data
    z = np.zeros((P, T))
    for p in range(P):  # one or two photons at least 300 bins away from the prior mean
        for t in rng.integers(50, 150, size=1 + p % 2):
            z[p, t] += 1.0
        if p % 3 == 0:  # and one aligned with the depth 350 bins past the prior mean
            z[p, int(pm[p]) + 350] += 1.0
    q, e, o = _estimate_both(orc, h, peak, z, pm, pv, 1.0, H, W, T)
    assert np.all(np.abs(e["argmax"].reshape(-1) - pm) <= 1.0), "the case should put the maximum at the prior mode"
    _compare(q, e, o)


@pytest.mark.parametrize("beta", [0.2, 0.5])
def test_recentred_sums(orc, beta):
    """A data peak 150-450 bins from a Gaussian prior's mean (variance 900-6400; 2-8 photons in the one bin that
    puts the template's peak tap there): where the peak is taller than the prior's bump but holds a small part of
    the mass, the mean lies more than two standard deviations from the maximum, so the epilogue takes its sums again
    about the rounded mean (the oracle's posterior confirms such pixels are in the set)."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 2048
    dmin = peak
    cfg = [(off, n, pv) for off in range(150, 451, 25) for n in range(2, 9) for pv in (900.0, 1600.0, 3600.0, 6400.0)]
    P = len(cfg)  # 364
    H, W = 4, P // 4
    z = np.zeros((P, T))
    pm = np.full(P, dmin + 800.0)
    pv = np.array([c[2] for c in cfg])
    for p, (off, n, _) in enumerate(cfg):  # the template of depth d has its peak tap at bin d
        z[p, dmin + 800 + off] += n
    q, e, o = _estimate_both(orc, h, peak, z, pm, pv, beta, H, W, T)
    far = (e["mu"] - e["argmax"]) ** 2 > 4 * e["var"] + 1
    assert far.sum() >= 5, "too few pixels with the mean more than two standard deviations from the maximum"
    _compare(q, e, o)


@pytest.mark.parametrize("entry", ["spl_filter_step_tc", "spl_filter_step_fp32"])
@pytest.mark.parametrize("nu0,diag", [(0.5, 0.0), (0.4, 0.02)])
def test_mixture_priors(orc, nu0, diag, entry):
    """One filter step from given states, on the tensor-core route and on the FP32 kernel: 3 x 3 stencils of up to
    nine distinct components, variances log-uniform on [5, 1e5], means anywhere on the grid, 0-6 photons per
    pixel."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 12, 14, 1500
    P = H * W
    L = len(h)
    dmin, dmax = peak, T - L + peak
    rng = np.random.default_rng(31 + int(diag * 100))
    mu = rng.uniform(dmin, dmax, size=(H, W)).astype(np.float32).astype(np.float64)
    var = np.exp(rng.uniform(np.log(5.0), np.log(1e5), size=(H, W))).astype(np.float32).astype(np.float64)
    z = _sparse_photons(rng, P, T, rng.integers(0, 7, size=P)).reshape(H, W, T)
    nu = synth.cross_weights(nu0)
    if diag:  # the four corners too: nine distinct components where the neighbour states differ
        nu = nu.copy()
        nu[[0, 2, 6, 8]] = diag
        nu[4] -= 4 * diag
    q = orc.params(T, L, peak, beta=0.5, sigma_rw2=3.0, nu=nu)
    e = orc.filter_step(q, h, z, mu, var, want_ell=True)
    prm = spl.make_params(H, W, T, L, peak, beta=0.5, sigma_rw2=3.0, nu=nu)
    o = getattr(spl, entry)(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV),
                            torch.from_numpy(mu.astype(np.float32)).reshape(-1).to(DEV),
                            torch.from_numpy(var.astype(np.float32)).reshape(-1).to(DEV), intensity=False)
    torch.cuda.synchronize()
    _compare(q, e, o)


def test_flat_prior_longest_histogram(orc):
    """No prior (a flat one) over T = SPL_MAX_BINS (255 blocks, eight ballot words per survivor scan), 0-4 photons
    per pixel."""
    h, peak = synth.asymmetric_irf(L=48)
    T = spl._abi.SPL_MAX_BINS
    H, W = 4, 8
    P = H * W
    rng = np.random.default_rng(41)
    z = _sparse_photons(rng, P, T, rng.integers(0, 5, size=P))
    for beta in (0.3, 1.0):
        q, e, o = _estimate_both(orc, h, peak, z, None, None, beta, H, W, T)
        _compare(q, e, o)


def test_photon_lists_long_histograms(orc):
    """The batched photon-list step (the same epilogue) on sequences of 4096 and 2048 bins with a few photons per
    pixel and frame, three frames from the initial state, against the oracle's histogram form."""
    from test_gpu_batch import _make_frames, _run
    from parity import check_intensity
    specs = [(6, 10, 4096, synth.asymmetric_irf(L=48), 0.5, 3.0, synth.cross_weights(0.5), 2.0, 3.0),
             (8, 8, 2048, synth.gaussian_irf(3.0, 12), 1.0, 10.0, synth.cross_weights(0.6), 1.0, 2.0)]
    seqs = _make_frames(specs, N=3, seed=17)
    res, flags, info = _run(seqs, 3)
    assert flags == 0
    for i, q in enumerate(seqs):
        oq = orc.params(q["T"], q["L"], q["peak"], beta=q["beta"], sigma_rw2=q["s2"], nu=q["nu"])
        mu, var = orc.state_init(oq, q["H"], q["W"])
        for n in range(3):
            off, bins = q["frames"][n]
            z = synth.csr_to_histograms(off, bins, q["T"]).astype(np.float64).reshape(q["H"], q["W"], q["T"])
            e = orc.filter_step(oq, q["h"], z, mu, var, want_ell=True)
            g = res[n][i]
            check_argmax(g["argmax"], e["argmax"], e["ell"], oq.dmin, f"seq {i} frame {n} argmax")
            check_close(g["mu_out"], e["mu"], f"seq {i} frame {n} mu")
            check_close(g["var_out"], e["var"], f"seq {i} frame {n} var", atol=1e-6)
            check_intensity(orc, oq, q["h"], z, g["mu_out"], e["mu"], g["refl"], g["bg"])
            mu, var = e["mu"], e["var"]
