"""GPU parity of spl_filter_step_tc (the filter step with the data term on the tensor cores) against the FP64
oracle on FP16 histograms.

Each frame is checked as a step function: the oracle runs from exactly the state the GPU received (the GPU's
previous output), on the same histograms, and the outputs are compared with the tolerances of the FP32 filter
(tests/parity.py). The tensor-core data term carries each powered tap g = h^beta as two FP16 parts of g * 2^15
(relative error <= 2^-22 per tap; products with integer counts are exact in FP32), so ell = lambda log2(e) C
moves by at most lambda log2(e) C 2^-22 bits, about 4e-5 bits for C = 20 at beta = 0.2: the moments move by a
few 1e-5 relative, inside 1e-4.
Independently, the whole GPU chain is compared with the whole oracle chain at 1e-3: over several frames the
per-step differences feed back through the neighbours' states, and a pixel whose posterior is bimodal can
amplify them (observed: 2.5e-4 after five frames from 2e-5 per step)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close, check_intensity
from test_gpu_parity import DEV, _gpu_hist, _np, video_inputs

pytestmark = pytest.mark.gpu


CHAIN_RTOL = 1e-3


def _run_tc(orc, q, prm, h, zs, T, present=None, faulty=None, present_now=None):
    """Per frame: GPU step, oracle step from the GPU's input state (compared at the parity tolerances) and the
    independent oracle chain (compared at CHAIN_RTOL). Returns the number of documented argmax near-ties."""
    H, W = prm.H, prm.W
    hd = torch.from_numpy(h).to(DEV)
    mu_g, var_g = spl.spl_state_init(prm)
    mu_c, var_c = orc.state_init(q, H, W)
    dp = lambda a: None if a is None else torch.from_numpy(a).to(DEV).reshape(-1)
    ties = 0
    for n, z in enumerate(zs):
        m_in = _np(mu_g).reshape(H, W).astype(np.float64)
        v_in = _np(var_g).reshape(H, W).astype(np.float64)
        o = spl.spl_filter_step_tc(prm, _gpu_hist(z, T, torch.float16), hd, mu_g, var_g, present_in=dp(present),
                                   faulty=dp(faulty), present_now=dp(present_now))
        e = orc.filter_step(q, h, z, m_in, v_in, present_in=present, faulty=faulty, want_ell=True)
        c = orc.filter_step(q, h, z, mu_c, var_c, present_in=present, faulty=faulty)
        torch.cuda.synchronize()
        ties += check_argmax(_np(o["argmax"]), e["argmax"], e["ell"], q.dmin, f"argmax frame {n}")
        check_close(_np(o["mu"]), e["mu"], f"mu frame {n}")
        check_close(_np(o["var"]), e["var"], f"var frame {n}", atol=1e-6)
        check_intensity(orc, q, h, z, _np(o["mu"]), e["mu"], _np(o["refl"]), _np(o["bg"]), present=present_now,
                        faulty=faulty)
        check_close(_np(o["mu"]), c["mu"], f"mu frame {n} (chain)", rtol=CHAIN_RTOL)
        check_close(_np(o["var"]), c["var"], f"var frame {n} (chain)", rtol=CHAIN_RTOL, atol=1e-5)
        mu_g, var_g = o["mu"], o["var"]
        mu_c, var_c = c["mu"], c["var"]
    return ties


def _status_clear():
    torch.cuda.synchronize()
    assert spl.spl_tc_status() == 0


@pytest.mark.parametrize("sbr,beta,T", [(0.01, 0.5, 400), (0.1, 0.2, 700), (1.0, 1.0, 400), (0.002, 0.5, 600)])
def test_filter_tc_video(orc, sbr, beta, T):
    H, W, N = 20, 24, 5
    h, peak, sc, zs = video_inputs(H, W, N, T, sbr, seed=300 + int(sbr * 100))
    q = orc.params(T, len(h), peak, beta=beta, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta, sigma_rw2=3.0)
    ties = _run_tc(orc, q, prm, h, zs, T)
    assert ties <= 3
    _status_clear()


def test_filter_tc_masks_and_stencil(orc):
    """Absent and faulty pixels, a full asymmetric 3x3 stencil, presence-dependent intensity."""
    H, W, N, T = 13, 17, 4, 300
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.1, seed=33, L=32)
    rng = np.random.default_rng(33)
    nu = np.array([0.05, 0.10, 0.02, 0.15, 0.40, 0.20, 0.03, 0.05, 0.0])
    present = (rng.random((H, W)) < 0.8).astype(np.uint8)
    faulty = (rng.random((H, W)) < 0.05).astype(np.uint8)
    pnow = (rng.random((H, W)) < 0.6).astype(np.uint8)
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=2.0, nu=nu)
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5, sigma_rw2=2.0, nu=nu)
    _run_tc(orc, q, prm, h, zs, T, present=present, faulty=faulty, present_now=pnow)
    _status_clear()


@pytest.mark.parametrize("H,W,T,L,peak,dmin,dmax", [
    (1, 37, 77, 1, 0, None, None),          # one-tap IRF, single row, one candidate tile
    (5, 1, 130, 7, 3, 20, 97),              # single column, dmin - peak = 17: a leading count-only slab, delta 1
    (3, 3, 64, 64, 10, None, None),         # L = T: exactly one candidate
    (7, 9, 333, 45, 40, None, None),        # odd T, padded pitch, D not a multiple of 64
    (2, 70, 2049, 128, 60, None, None),     # largest supported IRF (4 slabs per window, deeper intensity window)
    (9, 31, 1000, 80, 20, 300, 500),        # sub-range far from bin 0 (count-only slabs on both sides)
    (2, 9, 8192, 128, 70, None, None),      # largest supported histogram and IRF (128 slabs per row)
])
def test_filter_tc_ragged_shapes(orc, H, W, T, L, peak, dmin, dmax):
    rng = np.random.default_rng(H * 1000 + W + 7)
    h = rng.uniform(0.0, 1.0, size=L).astype(np.float32)
    h[peak] = 2.0
    h /= h.sum()
    q = orc.params(T, L, peak, dmin, dmax, beta=0.6, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    z = rng.poisson(0.3, size=(H, W, T)).astype(np.float64)
    for y in range(H):
        for x in range(W):
            d = int(rng.integers(q.dmin, q.dmax + 1))
            z[y, x, d - peak:d - peak + L] += rng.poisson(6 * h)
    prm = spl.make_params(H, W, T, L, peak, dmin, dmax, beta=0.6, sigma_rw2=3.0)
    _run_tc(orc, q, prm, h, [z, z[::-1].copy(), z], T)
    _status_clear()


def test_filter_tc_empty_histograms_give_the_prior(orc):
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 6, 6, 500
    z = np.zeros((H, W, T))
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5)
    _run_tc(orc, q, prm, h, [z, z, z], T)
    _status_clear()


def test_filter_tc_strong_counts(orc):
    """Counts up to 2048 (exact in FP16) from strong Poisson returns: posteriors concentrated on one or two
    candidates."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 4, 5, 600
    rng = np.random.default_rng(5)
    z = rng.poisson(2.0, size=(H, W, T)).astype(np.float64)
    for i in range(H * W):
        y, x = divmod(i, W)
        s = int(rng.integers(60, 480))
        z[y, x, s - peak:s - peak + 48] += rng.poisson(2000 * h / h.max())
    z = np.minimum(z, 2048)
    q = orc.params(T, len(h), peak, beta=0.1, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.1, sigma_rw2=3.0)
    _run_tc(orc, q, prm, h, [z, z], T)
    _status_clear()


def test_filter_tc_exact_plateaus_given_its_data_term(orc):
    """Degenerate ties: 1000 photons in each of 79 consecutive bins, so about 30 candidates share exactly the
    same C (about 3e4) and the posterior is flat over them. The tensor cores add the terms of C in a different
    order for every candidate, so their FP32 rounding (about 1e-7 relative, i.e. ~0.1 bit of ell at
    lambda log2(e) = 16) breaks the tie at random: against the FP64 oracle the mean moves by up to ~0.03 bins,
    which is the data term's accuracy, not the filter's. The filter is therefore checked given its own data
    term: the FP64 posterior of ell = lambda C_tc + log f, with C_tc the tensor-core costs of the same tiles
    (spl_depth_cost_tc runs the same MMA sequence; C_tc itself is checked against the oracle in
    test_gpu_tc.py), must match the fused kernel's argmax, mean and variance at the usual tolerances."""
    h, peak = synth.asymmetric_irf(L=48)
    H, W, T = 2, 3, 600
    z = np.zeros((H, W, T))
    for i, s in enumerate((100, 250, 400, 130, 333, 480)):
        z[i // W, i % W, s:s + 79] = 1000.0
    q = orc.params(T, len(h), peak, beta=0.1, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.1, sigma_rw2=3.0)
    hd = torch.from_numpy(h).to(DEV)
    zt = _gpu_hist(z, T, torch.float16)
    mu0, var0 = spl.spl_state_init(prm)
    o = spl.spl_filter_step_tc(prm, zt, hd, mu0, var0)
    ctc, _ = spl.spl_depth_cost_tc(prm, zt, hd)
    _status_clear()
    m0, v0 = orc.state_init(q, H, W)
    e = orc.filter_step(q, h, z, m0, v0, want_ell=True)
    lam = (q.beta + 1.0) / q.beta
    ell = e["ell"].reshape(H * W, -1)
    log_prior = ell - lam * orc.cost(q, h, z).reshape(H * W, -1)
    ell_tc = lam * _np(ctc).astype(np.float64) + log_prior
    for p in range(H * W):
        a, m, v = orc.posterior(ell_tc[p], q.dmin)
        check_argmax(_np(o["argmax"][p:p + 1]), [a], ell_tc[p:p + 1], q.dmin, f"argmax[{p}]")
        check_close(_np(o["mu"][p]), m, f"mu[{p}]")
        check_close(_np(o["var"][p]), v, f"var[{p}]", atol=1e-6)


@pytest.mark.parametrize("sigma_rw2", [0.3, 50.0])
def test_filter_tc_component_widths(orc, sigma_rw2):
    H, W, N, T = 12, 14, 4, 350
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.3, seed=43)
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=sigma_rw2, nu=synth.cross_weights(0.5))
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5, sigma_rw2=sigma_rw2)
    _run_tc(orc, q, prm, h, zs, T)
    _status_clear()


def test_filter_tc_agrees_with_fp32_path():
    """The tensor-core step and the FP32 CUDA-core step on the same FP16 frames give the same states."""
    H, W, N, T = 40, 36, 4, 900
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.05, seed=61)
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.5, sigma_rw2=3.0)
    hd = torch.from_numpy(h).to(DEV)
    m1, v1 = spl.spl_state_init(prm)
    m2, v2 = m1.clone(), v1.clone()
    for z in zs:
        zt = _gpu_hist(z, T, torch.float16)
        a = spl.spl_filter_step_fp32(prm, zt, hd, m1, v1)
        b = spl.spl_filter_step_tc(prm, zt, hd, m2, v2)
        torch.cuda.synchronize()
        check_close(_np(b["mu"]), _np(a["mu"]), "mu tc vs fp32", rtol=1e-4)
        check_close(_np(b["var"]), _np(a["var"]), "var tc vs fp32", rtol=1e-3, atol=1e-5)
        check_close(_np(b["bg"]), _np(a["bg"]), "bg tc vs fp32", rtol=1e-4, atol=1e-7)
        m1, v1, m2, v2 = a["mu"], a["var"], b["mu"], b["var"]
    _status_clear()


def test_filter_tc_full_size_frames_sampled(orc):
    """Two frames of the mixed-precision workload's geometry (1024 x 1024 pixels, T = 4096, 64-tap IRF, SBR
    0.05, FP16 counts) through the full launch configuration, compared on sampled pixels against the oracle
    on (2n+1)^2 crops (after n frames a pixel depends only on inputs within Chebyshev distance n)."""
    H = W = 1024
    N, T, L = 2, 4096, 64
    h, peak = synth.stretched_irf(synth.asymmetric_irf(L=48)[0], L)
    sc = synth.moving_scene(H, W, N, peak + 8, T - L + peak - 8, seed=3)
    g = torch.Generator(device=DEV).manual_seed(3)
    hd = torch.from_numpy(h).to(DEV)
    prm = spl.make_params(H, W, T, L, peak, beta=0.5, sigma_rw2=3.0)
    pitch = synth.pad_pitch(T)
    zs = []
    for n in range(N):
        b = float(sc.signal[n].mean()) / (0.05 * T)
        zs.append(synth.frame_histograms(torch.from_numpy(sc.depth[n]).to(DEV), torch.from_numpy(sc.signal[n]).to(DEV),
                                         b, hd, peak, T, g, pitch))
    mu, var = spl.spl_state_init(prm)
    states = [(mu, var)]
    outs = []
    for n in range(N):
        o = spl.spl_filter_step_tc(prm, zs[n], hd, mu, var)
        mu, var = o["mu"], o["var"]
        states.append((mu, var))
        outs.append(o)
    _status_clear()
    q = orc.params(T, L, peak, beta=0.5, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    samples = [(0, 0), (0, 1023), (1023, 0), (1023, 1023), (512, 77), (3, 700), (700, 1), (397, 1022), (640, 640)]
    zc = [z[:, :T].reshape(H, W, T) for z in zs]
    for (y, x) in samples:
        i = y * W + x
        # each frame as a step from the GPU's own input state (3x3 neighbourhood)
        y0, y1, x0, x1 = max(0, y - 1), min(H, y + 2), max(0, x - 1), min(W, x + 2)
        k = (y - y0) * (x1 - x0) + (x - x0)
        for n in range(N):
            m_in = _np(states[n][0].reshape(H, W)[y0:y1, x0:x1]).astype(np.float64)
            v_in = _np(states[n][1].reshape(H, W)[y0:y1, x0:x1]).astype(np.float64)
            crop = _np(zc[n][y0:y1, x0:x1]).astype(np.float64)
            e = orc.filter_step(q, h, crop, m_in, v_in, want_ell=True)
            check_close(_np(outs[n]["mu"][i]), e["mu"].reshape(-1)[k], f"mu[{y},{x}] frame {n}")
            check_close(_np(outs[n]["var"][i]), e["var"].reshape(-1)[k], f"var[{y},{x}] frame {n}", atol=1e-6)
            check_argmax(_np(outs[n]["argmax"][i:i + 1]), e["argmax"].reshape(-1)[k:k + 1],
                         e["ell"].reshape((y1 - y0) * (x1 - x0), -1)[k:k + 1], q.dmin, f"argmax[{y},{x}] frame {n}")
        # the independent chain on the (2N+1)^2 dependency cone
        y0, y1, x0, x1 = max(0, y - N), min(H, y + N + 1), max(0, x - N), min(W, x + N + 1)
        m, v = orc.state_init(q, y1 - y0, x1 - x0)
        for n in range(N):
            e = orc.filter_step(q, h, _np(zc[n][y0:y1, x0:x1]).astype(np.float64), m, v)
            m, v = e["mu"], e["var"]
        check_close(_np(mu[i]), m[y - y0, x - x0], f"mu[{y},{x}] (chain)", rtol=CHAIN_RTOL)
        check_close(_np(var[i]), v[y - y0, x - x0], f"var[{y},{x}] (chain)", rtol=CHAIN_RTOL, atol=1e-5)
