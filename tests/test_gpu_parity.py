"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle, element by element, on seeded
synthetic inputs shaped like the paper's workloads. Tolerances are documented in tests/parity.py."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close, check_intensity

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _gpu_hist(z_np, T, dtype=torch.uint16):
    """[..., T] counts -> contiguous device tensor [P, pitch] with 16-byte rows."""
    z = torch.from_numpy(np.ascontiguousarray(z_np).astype(np.float32)).reshape(-1, T)
    esz = 4 if dtype == torch.float32 else 2
    pitch = synth.pad_pitch(T, esz)
    if dtype == torch.uint16:
        z = z.to(torch.int32).to(torch.uint16)
    else:
        z = z.to(dtype)
    return synth.pitched(z, pitch).to(DEV)


def single_frame_inputs(H=32, W=32, T=1024, seed=1, signal=10.0, bg_total=50.0):
    """The single-frame workload: Gaussian IRF sigma = 3 bins over +-12 taps, smooth random surface scaled
    to bins 100..900, Poisson signal mean `signal` at the shifted IRF plus background `bg_total` over all
    bins."""
    h, peak = synth.gaussian_irf(3.0, 12)
    depth = synth.smooth_depth_map(H, W, 100, 900, seed)
    g = torch.Generator().manual_seed(seed)
    mean = synth.expected_counts(torch.from_numpy(depth), torch.full((H, W), signal, dtype=torch.float64),
                                 bg_total / T, torch.from_numpy(h), peak, T)
    z = torch.poisson(mean, generator=g).numpy().astype(np.float64)
    return h, peak, depth, z


def video_inputs(H, W, N, T, sbr, seed, L=48):
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(H, W, N, peak + 8, T - L + peak - 8, seed)
    g = torch.Generator().manual_seed(seed)
    zs = []
    for n in range(N):
        b = float(sc.signal[n].mean()) / (sbr * T)
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]), torch.from_numpy(sc.signal[n]), b,
                                     torch.from_numpy(h), peak, T)
        zs.append(torch.poisson(mean, generator=g).numpy().astype(np.float64))
    return h, peak, sc, zs


def _np(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------------------------------------------------
# spl_depth_cost
# ------------------------------------------------------------------------------------------------------------


@pytest.mark.parametrize("bg_total", [50.0, 3000.0])
def test_cost_single_frame(orc, bg_total):
    h, peak, depth, z = single_frame_inputs(bg_total=bg_total)
    H, W, T = z.shape
    q = orc.params(T, len(h), peak, beta=0.5)
    C_orc = orc.cost(q, h, z).reshape(H * W, -1)
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5)
    hd = torch.from_numpy(h).to(DEV)
    cost, am = spl.spl_depth_cost(prm, _gpu_hist(z, T), hd)
    torch.cuda.synchronize()
    check_close(_np(cost), C_orc, "C", atol=1e-6 * C_orc.max())
    ties = check_argmax(_np(am), C_orc.argmax(1) + q.dmin, C_orc, q.dmin, "argmax C")
    assert ties <= 2
    if bg_total < 100:   # strong enough signal: the minimum-divergence argmax lands on the true depth
        assert np.mean(np.abs(_np(am).reshape(H, W) - depth) <= 3) > 0.8


@pytest.mark.parametrize("dtype", [torch.float16, torch.float32])
def test_cost_formats_agree_exactly(orc, dtype):
    """Counts are exact in every storage format, so the three formats give bit-identical C(d)."""
    h, peak, depth, z = single_frame_inputs(H=8, W=12, T=1000, seed=3)
    H, W, T = z.shape
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5)
    hd = torch.from_numpy(h).to(DEV)
    c16, a16 = spl.spl_depth_cost(prm, _gpu_hist(z, T, torch.uint16), hd)
    cx, ax = spl.spl_depth_cost(prm, _gpu_hist(z, T, dtype), hd)
    torch.cuda.synchronize()
    assert torch.equal(c16, cx) and torch.equal(a16, ax)


# ------------------------------------------------------------------------------------------------------------
# spl_depth_estimate
# ------------------------------------------------------------------------------------------------------------


@pytest.mark.parametrize("beta,bg_total", [(0.2, 50.0), (0.5, 50.0), (1.0, 50.0), (0.5, 3000.0)])
def test_estimate_uniform_prior(orc, beta, bg_total):
    """bg_total 50: about 60 non-empty bins per pixel (zero-skip correlation); 3000: about 950 (dense)."""
    h, peak, depth, z = single_frame_inputs(seed=11, bg_total=bg_total)
    H, W, T = z.shape
    q = orc.params(T, len(h), peak, beta=beta)
    e = orc.estimate(q, h, z, want_ell=True)
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta)
    o = spl.spl_depth_estimate(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV))
    torch.cuda.synchronize()
    check_argmax(_np(o["argmax"]), e["argmax"], e["ell"], q.dmin)
    check_close(_np(o["mu"]), e["mu"], "mu")
    check_close(_np(o["var"]), e["var"], "var", atol=1e-6)
    check_intensity(orc, q, h, z, _np(o["mu"]), e["mu"], _np(o["refl"]), _np(o["bg"]))


def test_estimate_gaussian_prior_and_presence(orc):
    h, peak, depth, z = single_frame_inputs(H=16, W=20, seed=12, signal=4.0, bg_total=200.0)
    H, W, T = z.shape
    rng = np.random.default_rng(12)
    pm = (depth + rng.normal(0, 15, size=depth.shape)).astype(np.float32)
    pv = rng.uniform(1.0, 400.0, size=depth.shape).astype(np.float32)
    present = (rng.random(depth.shape) < 0.7).astype(np.uint8)
    q = orc.params(T, len(h), peak, beta=0.4)
    e = orc.estimate(q, h, z, prior_mu=pm, prior_var=pv, want_ell=True)
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.4)
    o = spl.spl_depth_estimate(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV),
                               prior_mu=torch.from_numpy(pm).to(DEV).reshape(-1),
                               prior_var=torch.from_numpy(pv).to(DEV).reshape(-1),
                               present=torch.from_numpy(present).to(DEV).reshape(-1))
    torch.cuda.synchronize()
    check_argmax(_np(o["argmax"]), e["argmax"], e["ell"], q.dmin)
    check_close(_np(o["mu"]), e["mu"], "mu")
    check_close(_np(o["var"]), e["var"], "var", atol=1e-6)
    check_intensity(orc, q, h, z, _np(o["mu"]), e["mu"], _np(o["refl"]), _np(o["bg"]), present=present)


# ------------------------------------------------------------------------------------------------------------
# spl_filter_step over short videos
# ------------------------------------------------------------------------------------------------------------


def _run_filter(orc, q, prm, h, zs, T, present=None, faulty=None, present_now=None, dtype=torch.uint16,
                step=None, tie_rel=None):
    """Runs the GPU chain and the oracle chain independently and compares every frame."""
    step = step or spl.spl_filter_step
    H, W = prm.H, prm.W
    hd = torch.from_numpy(h).to(DEV)
    mu_g, var_g = spl.spl_state_init(prm)
    mu_o, var_o = orc.state_init(q, H, W)
    dp = lambda a: None if a is None else torch.from_numpy(a).to(DEV).reshape(-1)
    ties = 0
    for n, z in enumerate(zs):
        o = step(prm, _gpu_hist(z, T, dtype), hd, mu_g, var_g, present_in=dp(present), faulty=dp(faulty),
                 present_now=dp(present_now))
        e = orc.filter_step(q, h, z, mu_o, var_o, present_in=present, faulty=faulty, want_ell=True)
        torch.cuda.synchronize()
        ties += check_argmax(_np(o["argmax"]), e["argmax"], e["ell"], q.dmin, f"argmax frame {n}")
        check_close(_np(o["mu"]), e["mu"], f"mu frame {n}")
        check_close(_np(o["var"]), e["var"], f"var frame {n}", atol=1e-6)
        check_intensity(orc, q, h, z, _np(o["mu"]), e["mu"], _np(o["refl"]), _np(o["bg"]), present=present_now,
                        faulty=faulty)
        mu_g, var_g = o["mu"], o["var"]
        mu_o, var_o = e["mu"], e["var"]
    return ties


@pytest.mark.parametrize("sbr,beta,T", [(0.01, 0.5, 400), (0.1, 0.2, 400), (1.0, 1.0, 400), (0.002, 0.5, 600)])
def test_filter_video(orc, sbr, beta, T):
    """SBR 0.002 puts about 450 non-empty bins in each pixel (dense correlation); the others use zero skip."""
    H, W, N = 20, 24, 5
    h, peak, sc, zs = video_inputs(H, W, N, T, sbr, seed=200 + int(sbr * 100))
    q = orc.params(T, len(h), peak, beta=beta, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta, sigma_rw2=3.0)
    ties = _run_filter(orc, q, prm, h, zs, T)
    assert ties <= 3


def test_filter_masks_and_stencil(orc):
    """Absent and faulty pixels, a full asymmetric 3x3 stencil, presence-dependent intensity."""
    H, W, N, T = 13, 17, 4, 300
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.1, seed=31, L=32)
    rng = np.random.default_rng(31)
    nu = np.array([0.05, 0.10, 0.02, 0.15, 0.40, 0.20, 0.03, 0.05, 0.0])
    present = (rng.random((H, W)) < 0.8).astype(np.uint8)
    faulty = (rng.random((H, W)) < 0.05).astype(np.uint8)
    pnow = (rng.random((H, W)) < 0.6).astype(np.uint8)
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=2.0, nu=nu)
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5, sigma_rw2=2.0, nu=nu)
    _run_filter(orc, q, prm, h, zs, T, present=present, faulty=faulty, present_now=pnow)


@pytest.mark.parametrize("H,W,T,L,peak,dmin,dmax", [
    (1, 37, 77, 1, 0, None, None),          # one-tap IRF, single row
    (5, 1, 130, 7, 3, 20, 97),              # single column, sub-range of depths
    (3, 3, 64, 64, 10, None, None),         # L = T: exactly one candidate
    (7, 9, 333, 45, 40, None, None),        # odd T, padded pitch, D not a multiple of 32
    (2, 70, 2049, 128, 60, None, None),     # largest supported IRF
])
def test_ragged_shapes(orc, H, W, T, L, peak, dmin, dmax):
    rng = np.random.default_rng(H * 1000 + W)
    h = rng.uniform(0.0, 1.0, size=L).astype(np.float32)
    h[peak] = 2.0
    h /= h.sum()
    q = orc.params(T, L, peak, dmin, dmax, beta=0.6, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    z = rng.poisson(0.3, size=(H, W, T)).astype(np.float64)
    dlo, dhi = q.dmin, q.dmax
    for y in range(H):
        for x in range(W):
            d = int(rng.integers(dlo, dhi + 1))
            z[y, x, d - peak:d - peak + L] += rng.poisson(6 * h)
    prm = spl.make_params(H, W, T, L, peak, dmin, dmax, beta=0.6, sigma_rw2=3.0)
    cost, am = spl.spl_depth_cost(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV))
    torch.cuda.synchronize()
    C = orc.cost(q, h, z).reshape(H * W, -1)
    check_close(_np(cost), C, "C", atol=1e-6 * C.max())
    check_argmax(_np(am), C.argmax(1) + q.dmin, C, q.dmin)
    _run_filter(orc, q, prm, h, [z, z[::-1].copy()], T)


@pytest.mark.parametrize("L,peak,bg", [
    (33, 12, 0.02),    # two tap groups of 32, the second with one tap
    (100, 40, 0.05),   # four tap groups
    (128, 90, 0.1),    # largest supported IRF
    (48, 20, 0.135),   # 110-140 non-empty bins: both sides of the zero-skip limit (128)
])
def test_sparse_rows_long_templates(orc, L, peak, bg):
    """Photon-starved rows (zero-skip correlation) with templates over several groups of 32 taps."""
    H, W, T = 4, 33, 900
    rng = np.random.default_rng(L * 7 + 1)
    h = rng.uniform(0.0, 1.0, size=L).astype(np.float32)
    h[peak] = 2.0
    h /= h.sum()
    q = orc.params(T, L, peak, beta=0.4, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    z = rng.poisson(bg, size=(H, W, T)).astype(np.float64)
    for y in range(H):
        for x in range(W):
            d = int(rng.integers(q.dmin, q.dmax + 1))
            z[y, x, d - peak:d - peak + L] += rng.poisson(4 * h)
    prm = spl.make_params(H, W, T, L, peak, beta=0.4, sigma_rw2=3.0)
    cost, am = spl.spl_depth_cost(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV))
    torch.cuda.synchronize()
    C = orc.cost(q, h, z).reshape(H * W, -1)
    check_close(_np(cost), C, "C", atol=1e-6 * C.max())
    check_argmax(_np(am), C.argmax(1) + q.dmin, C, q.dmin)
    _run_filter(orc, q, prm, h, [z, z[:, ::-1].copy()], T)


@pytest.mark.parametrize("dtype", [torch.uint16, torch.float16, torch.float32])
def test_largest_supported_histogram(orc, dtype):
    """T = SPL_MAX_BINS (8192) with the largest IRF (L = SPL_MAX_TAPS = 128): the largest shared-memory slices
    (one warp per CTA for FP32 rows), 253 candidate blocks, and dense and zero-skip rows side by side."""
    H, W, T, L, peak = 2, 9, 8192, 128, 70
    rng = np.random.default_rng(8192)
    h = rng.uniform(0.0, 1.0, size=L).astype(np.float32)
    h[peak] = 2.0
    h /= h.sum()
    q = orc.params(T, L, peak, beta=0.6, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    bg = np.where(np.arange(W) % 2 == 0, 0.002, 0.05)  # 27-127 and 390-550 non-empty bins per row
    z = rng.poisson(np.broadcast_to(bg[None, :, None], (H, W, T))).astype(np.float64)
    for y in range(H):
        for x in range(W):
            d = int(rng.integers(q.dmin, q.dmax + 1))
            # weak (broad posterior over 8065 candidates) and strong (var < 0.1 bin^2) surfaces
            z[y, x, d - peak:d - peak + L] += rng.poisson((20.0 if (x + y) % 3 == 0 else 300.0) * h)
    prm = spl.make_params(H, W, T, L, peak, beta=0.6, sigma_rw2=3.0)
    cost, am = spl.spl_depth_cost(prm, _gpu_hist(z, T, dtype), torch.from_numpy(h).to(DEV))
    torch.cuda.synchronize()
    C = orc.cost(q, h, z).reshape(H * W, -1)
    check_close(_np(cost), C, "C", atol=1e-6 * C.max())
    check_argmax(_np(am), C.argmax(1) + q.dmin, C, q.dmin)
    _run_filter(orc, q, prm, h, [z, z[::-1].copy()], T, dtype=dtype)


def _logit(p):
    p = np.clip(np.asarray(p, np.float64), 1e-300, 1 - 1e-16)
    return np.log(p) - np.log1p(-p)


@pytest.mark.parametrize("sbr,beta", [(0.1, 0.5), (1.0, 0.3), (0.02, 0.5)])
def test_filter_step_detect(orc, sbr, beta):
    """The on-device presence decision (detection surrogate) against the oracle, frame by frame on the GPU's
    own inputs: a scene whose left third has no surface (background only), faulty pixels, pi0 from
    Eq. prior_detect of the previous frame's pi and present_in from the previous frame's decision."""
    H, W, N, T = 18, 24, 4, 500
    h, peak = synth.asymmetric_irf(L=48)
    sc = synth.moving_scene(H, W, N, peak + 8, T - 48 + peak - 8, 77)
    g = torch.Generator().manual_seed(77)
    rng = np.random.default_rng(77)
    faulty = (rng.random((H, W)) < 0.05).astype(np.uint8)
    q = orc.params(T, len(h), peak, beta=beta, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta, sigma_rw2=3.0)
    hd = torch.from_numpy(h).to(DEV)
    fd = torch.from_numpy(faulty).to(DEV).reshape(-1)
    mu_g, var_g = spl.spl_state_init(prm)
    pres_g, pi0_g = None, None
    decided = flipped = 0
    for n in range(N):
        sig = sc.signal[n].copy()
        sig[:, : W // 3] = 0.0                                   # no surface: background only
        b = float(sc.signal[n].mean()) / (sbr * T)
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]), torch.from_numpy(sig), b,
                                     torch.from_numpy(h), peak, T)
        z = torch.poisson(mean, generator=g).numpy().astype(np.float64)
        o = spl.spl_filter_step_detect(prm, _gpu_hist(z, T), hd, mu_g, var_g, present_in=pres_g, faulty=fd,
                                       pi0=pi0_g)
        torch.cuda.synchronize()
        pin = None if pres_g is None else _np(pres_g).reshape(H, W)
        e = orc.filter_step(q, h, z, _np(mu_g).reshape(H, W), _np(var_g).reshape(H, W), present_in=pin,
                            faulty=faulty)
        check_close(_np(o["mu"]), e["mu"], f"mu frame {n}")
        check_close(_np(o["var"]), e["var"], f"var frame {n}", atol=1e-6)
        p0 = None if pi0_g is None else _np(pi0_g).reshape(H, W)
        d = orc.detect(q, h, z, _np(o["mu"]).reshape(H, W), dmap=_np(o["argmax"]).reshape(H, W),
                       var=_np(o["var"]).reshape(H, W), pi0=p0, faulty=faulty)
        pi_g = _np(o["pi"]).reshape(-1)
        pi_o = d["pi"].reshape(-1)
        # pi = sigmoid(x): an error dx of the evidence x (relative 1e-4, absolute 1e-3) moves pi by
        # pi (1 - pi) dx, and storing pi in FP32 adds at most 1.2e-7
        x_o = _logit(pi_o)
        tol = pi_o * (1 - pi_o) * (1e-3 + 1e-4 * np.abs(x_o)) + 1.2e-7
        bad = np.abs(pi_g - pi_o) > tol
        assert not bad.any(), f"pi frame {n}: gpu {pi_g[bad][:5]} oracle {pi_o[bad][:5]}"
        pr_g = _np(o["present"]).reshape(-1).astype(bool)
        pr_o = d["present"].reshape(-1).astype(bool)
        near = np.abs(x_o) <= 1e-3 + 1e-4 * np.abs(x_o)
        assert np.all((pr_g == pr_o) | near), f"present frame {n}: {np.nonzero((pr_g != pr_o) & ~near)[0][:5]}"
        assert np.all(pr_g == (pi_g > 0.5))
        same = pr_g == pr_o
        K = z.reshape(-1, T).sum(1)
        hs = float(np.sum(h.astype(np.float64)))
        check_close(_np(o["bg"])[same], d["bg"].reshape(-1)[same], f"bg frame {n}", atol=1e-5 * (K[same] / T) + 1e-12)
        check_close(_np(o["refl"])[same], d["refl"].reshape(-1)[same], f"refl frame {n}",
                    atol=1e-5 * K[same] / hs + 1e-12)
        assert np.all(pi_g[faulty.reshape(-1) == 1] == 0.5)
        decided += pr_g.sum()
        flipped += int((~same).sum())
        pi0_g = spl.spl_pi_propagate(prm, o["pi"], faulty=fd)
        pres_g = o["present"]
        mu_g, var_g = o["mu"], o["var"]
    # both decisions occur: the surface region is mostly detected, the empty third mostly not
    assert 0 < decided < N * H * W
    assert flipped <= 2


def test_pd_experiment_estimates_match_the_oracle(orc):
    """The single-pixel p_d experiment (Sec. IV-A, Gaussian IRF, prior N(600, 2500)) on a small grid: the GPU
    pseudo-posterior means equal the oracle's, and so do the satisfactory-detection indicators |mu - d| < 28
    (except where the oracle's error is within 1e-3 of the threshold)."""
    import bench
    sbr, msc = [0.001, 1.0, 50.0], [12.0, 300.0]
    n_mc = 40
    h, peak, depth, z = bench.pd_inputs(sbr, msc, n_mc, 5, DEV)
    P = z.shape[0]
    T = bench.PD_T
    q = orc.params(T, len(h), peak, beta=0.5)
    prm = spl.make_params(1, P, T, len(h), peak, beta=0.5)
    pm = torch.full((P,), bench.PD_PRIOR_MU, device=DEV)
    pv = torch.full((P,), bench.PD_PRIOR_VAR, device=DEV)
    o = spl.spl_depth_estimate(prm, z, torch.from_numpy(h).to(DEV), pm, pv, intensity=False)
    torch.cuda.synchronize()
    zc = _np(z)[:, :T].astype(np.float64)
    e = orc.estimate(q, h, zc.reshape(1, P, T), prior_mu=np.full((1, P), bench.PD_PRIOR_MU),
                     prior_var=np.full((1, P), bench.PD_PRIOR_VAR))
    mu_o = e["mu"].reshape(-1)
    check_close(_np(o["mu"]), mu_o, "mu")
    d = _np(depth).astype(np.float64)
    ok_g = np.abs(_np(o["mu"]) - d) < bench.PD_ETA
    ok_o = np.abs(mu_o - d) < bench.PD_ETA
    edge = np.abs(np.abs(mu_o - d) - bench.PD_ETA) < 1e-3
    assert np.all((ok_g == ok_o) | edge)
    # the grid spans failure and success: 12 signal photons under 6000 background photons leave about the
    # prior's own rate (|N(0, 2500)| < 28: 0.42); 300 photons at SBR 50 succeed
    cell = ok_o.reshape(len(msc), len(sbr), n_mc).mean(-1)
    assert cell[1, 2] > 0.85 and cell[0, 0] < 0.7


def test_empty_histograms_give_the_prior(orc):
    """No photons: the GPU posterior moments equal the prior's (and the oracle's)."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 6, 6, 500
    z = np.zeros((H, W, T))
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5)
    _run_filter(orc, q, prm, h, [z, z, z], T)


# ------------------------------------------------------------------------------------------------------------
# Auxiliary kernels
# ------------------------------------------------------------------------------------------------------------


def test_pi_propagate(orc):
    H, W = 33, 45
    rng = np.random.default_rng(7)
    pi = rng.uniform(0, 1, size=(H, W)).astype(np.float32)
    pi[0, :5] = [0.0, 1.0, 1e-9, 1 - 1e-9, 0.5]
    faulty = (rng.random((H, W)) < 0.05).astype(np.uint8)
    nu = synth.cross_weights(0.5)
    prm = spl.make_params(H, W, 64, 8, 4, nu=nu)
    out = spl.spl_pi_propagate(prm, torch.from_numpy(pi).to(DEV).reshape(-1),
                               faulty=torch.from_numpy(faulty).to(DEV).reshape(-1))
    torch.cuda.synchronize()
    ref = orc.pi_propagate(nu, pi, faulty)
    check_close(_np(out), ref, "pi0", rtol=1e-5, atol=1e-6)


def test_state_init(orc):
    prm = spl.make_params(5, 7, 300, 20, 6, dmin=30, dmax=250)
    mu, var = spl.spl_state_init(prm)
    torch.cuda.synchronize()
    q = orc.params(300, 20, 6, 30, 250)
    m, v = orc.state_init(q, 5, 7)
    check_close(_np(mu), m, "mu0", rtol=0)
    check_close(_np(var), v, "var0", rtol=1e-7)


# ------------------------------------------------------------------------------------------------------------
# Full-size frame (the video workload's 256 x 256 x 1500 geometry), checked on sampled pixels
# ------------------------------------------------------------------------------------------------------------


@pytest.mark.parametrize("sbr,beta", [(0.1, 0.5), (0.01, 0.2), (1.0, 1.0)])
def test_full_size_video_frames_sampled(orc, sbr, beta):
    """Two frames of a 256 x 256, T = 1500 video with the full launch configuration, compared on sampled
    pixels: after n frames a pixel depends only on inputs within Chebyshev distance n (the oracle's
    dependency-cone pin), so the oracle runs on (2n+1)^2 crops. Every output of both frames is compared: mu, var,
    argmax (near-tie rule) and the intensity pair (refl, bg). Three (SBR, beta) runs of the video job: a dense
    row at SBR 0.01 with beta 0.2, the middle run, and photon-starved broad posteriors at SBR 1 with beta 1."""
    H = W = 256
    N, T, L = 2, 1500, 48
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(H, W, N, peak + 8, T - L + peak - 8, seed=251)
    g = torch.Generator(device=DEV).manual_seed(251)
    hd = torch.from_numpy(h).to(DEV)
    prm = spl.make_params(H, W, T, L, peak, beta=beta, sigma_rw2=3.0)
    pitch = synth.pad_pitch(T)
    zs = []
    for n in range(N):
        b = float(sc.signal[n].mean()) / (sbr * T)
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]).to(DEV), torch.from_numpy(sc.signal[n]).to(DEV),
                                     b, hd, peak, T)
        zs.append(synth.pitched(synth.poisson_histograms(mean, g).reshape(-1, T), pitch))
    mu, var = spl.spl_state_init(prm)
    outs = []
    for n in range(N):
        o = spl.spl_filter_step(prm, zs[n], hd, mu, var)
        mu, var = o["mu"], o["var"]
        outs.append({k: _np(v).reshape(H, W) for k, v in o.items()})
    torch.cuda.synchronize()
    q = orc.params(T, L, peak, beta=beta, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    samples = [(0, 0), (0, 255), (255, 0), (255, 255), (128, 77), (3, 200), (200, 1), (97, 254)]
    zc = [z[:, :T].reshape(H, W, T) for z in zs]
    for (y, x) in samples:
        y0, y1 = max(0, y - N), min(H, y + N + 1)
        x0, x1 = max(0, x - N), min(W, x + N + 1)
        m, v = orc.state_init(q, y1 - y0, x1 - x0)
        for n in range(N):
            crop = _np(zc[n][y0:y1, x0:x1]).astype(np.float64)
            e = orc.filter_step(q, h, crop, m, v, want_ell=True)
            m, v = e["mu"], e["var"]
            cy, cx = y - y0, x - x0
            o = outs[n]
            what = f"[{y},{x}] frame {n}"
            check_close(o["mu"][y, x], m[cy, cx], f"mu{what}")
            check_close(o["var"][y, x], v[cy, cx], f"var{what}", atol=1e-6)
            check_argmax(o["argmax"][y, x], e["argmax"][cy, cx], e["ell"][cy, cx], q.dmin, f"argmax{what}")
            check_intensity(orc, q, h, crop[cy, cx], o["mu"][y, x], m[cy, cx], o["refl"][y, x], o["bg"][y, x])


# ------------------------------------------------------------------------------------------------------------
# Epilogue paths: linear-domain weights, their fallback, narrow components
# ------------------------------------------------------------------------------------------------------------


def test_broad_posterior_fallback_when_weights_underflow(orc):
    """1000 photons in each of 79 consecutive bins: the photon-count bound of the data term exceeds the best
    value by far more than the float range, so the linear-domain weights underflow and the exact log-domain
    path must take over; results still match the oracle."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 2, 3, 600
    z = np.zeros((H, W, T))
    for i, s in enumerate((100, 250, 400, 130, 333, 480)):
        z[i // W, i % W, s:s + 79] = 1000.0
    q = orc.params(T, len(h), peak, beta=0.1)
    e = orc.estimate(q, h, z, want_ell=True)
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.1)
    o = spl.spl_depth_estimate(prm, _gpu_hist(z, T), torch.from_numpy(h).to(DEV))
    torch.cuda.synchronize()
    check_argmax(_np(o["argmax"]), e["argmax"], e["ell"], q.dmin)
    check_close(_np(o["mu"]), e["mu"], "mu")
    check_close(_np(o["var"]), e["var"], "var", atol=1e-6)


@pytest.mark.parametrize("sigma_rw2", [0.3, 50.0])
def test_filter_component_widths(orc, sigma_rw2):
    """sigma_RW^2 = 0.3 makes mixture components narrower than the recurrence allows (exact log path);
    50 keeps every posterior broad (linear-domain path on most pixels)."""
    H, W, N, T = 12, 14, 4, 350
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.3, seed=41)
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=sigma_rw2, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5, sigma_rw2=sigma_rw2)
    _run_filter(orc, q, prm, h, zs, T)
