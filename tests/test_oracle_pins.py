"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a library routine that the method reduces
to in a special case, a closed form, an invariant, or an alternative formulation the paper states as
equivalent. They are chosen so that a plausible slip (a dropped or extra factor lambda, a reversed template,
an off-by-one peak index, 0^beta = 1, a missing random-walk variance, a transposed stencil, a wrong edge
rule) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2004_09211_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


def _rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------------------------------------------------------
# Robust data term C(d) = z^T s_d^beta (Eq. beta_div2, histogram form)
# ------------------------------------------------------------------------------------------------------


def test_beta_one_is_matched_filter(orc):
    """beta = 1 reduces to matched filtering (Sec. II-B): C(d) = numpy.correlate(z, h)[d - peak]."""
    h, peak = synth.asymmetric_irf(L=13)
    T = 64
    z = _rng(0).poisson(2.0, size=(5, T)).astype(np.float64)
    q = orc.params(T, len(h), peak, beta=1.0)
    C = orc.cost(q, h, z)
    for p in range(5):
        ref = np.correlate(z[p], h.astype(np.float64), mode="valid")   # ref[u] = sum_j z[u + j] h[j]
        np.testing.assert_allclose(C[p], ref[q.dmin - peak:q.dmax - peak + 1], rtol=1e-13, atol=1e-15)


def test_photon_list_form_equals_histogram_form(orc):
    """Sum over photons of f0(y_k|d)^beta (Eq. beta_div2) equals z^T s_d^beta on their histogram."""
    h, peak = synth.asymmetric_irf(L=11)
    T = 50
    rng = _rng(1)
    for beta in (0.2, 0.5, 1.0, 1.7):
        y = rng.integers(0, T, size=40).astype(np.int32)      # repeated bins included
        z = np.bincount(y, minlength=T).astype(np.float64)
        q = orc.params(T, len(h), peak, beta=beta)
        np.testing.assert_allclose(orc.cost_toa(q, h, y), orc.cost(q, h, z[None])[0], rtol=1e-13)


def test_toa_histogram_hand_example(orc):
    """A worked example counted by hand: three pixels with 3, 0 and 2 photons on T = 4 bins."""
    z, flags = orc.toa_histogram(4, [0, 3, 3, 5], [2, 0, 2, 1, 1])
    assert flags == 0
    np.testing.assert_array_equal(z, [[1, 0, 2, 0], [0, 0, 0, 0], [0, 2, 0, 0]])


def test_toa_histogram_carries_the_photon_sum_form(orc):
    """Each row of toa_histogram is the histogram of the histogram form of Eq. beta_div2: C(d) on it equals the
    photon-sum form on the pixel's list in any order, and the row sums to the pixel's photon count K."""
    h, peak = synth.asymmetric_irf(L=11)
    T = 50
    rng = _rng(21)
    counts = rng.integers(0, 30, size=12)
    counts[[0, 5]] = 0
    off = np.concatenate([[0], np.cumsum(counts)])
    y = rng.integers(0, T, size=int(off[-1]))
    z, flags = orc.toa_histogram(T, off, y)
    assert flags == 0 and z.shape == (12, T)
    q = orc.params(T, len(h), peak, beta=0.5)
    for p in range(12):
        yp = y[off[p]:off[p + 1]]
        assert z[p].sum() == counts[p]
        if counts[p] == 0:
            assert not z[p].any()
            continue
        np.testing.assert_allclose(orc.cost(q, h, z[p][None].astype(np.float64))[0],
                                   orc.cost_toa(q, h, rng.permutation(yp).astype(np.int32)), rtol=1e-13)


def test_toa_histogram_input_errors(orc):
    """Photons outside [0, T) are dropped (flag 1); a pixel with decreasing or out-of-range offsets gets an empty
    row (flag 4) and the other pixels keep theirs."""
    z, flags = orc.toa_histogram(4, [0, 2, 4], [1, 4, 3, 3])
    assert flags == 1
    np.testing.assert_array_equal(z, [[0, 1, 0, 0], [0, 0, 0, 2]])
    z, flags = orc.toa_histogram(4, [0, 2, 1, 3, 9], [1, 1, 2])
    assert flags == 4
    np.testing.assert_array_equal(z, [[0, 2, 0, 0], [0, 0, 0, 0], [0, 1, 1, 0], [0, 0, 0, 0]])


def test_zero_taps_contribute_nothing(orc):
    """0^beta = 0: an IRF with holes gives C(d) = (1/m)^beta * (photons on the non-zero taps), a windowed
    count computed with numpy.correlate against the tap mask."""
    L, T = 9, 40
    mask = np.ones(L)
    mask[[2, 5, 6]] = 0.0
    h = (mask / mask.sum()).astype(np.float32)
    peak = 0
    z = _rng(2).poisson(1.5, size=T).astype(np.float64)
    for beta in (0.05, 0.5, 1.0):
        q = orc.params(T, L, peak, beta=beta)
        ref = np.correlate(z, mask, mode="valid") * float(h[0]) ** beta   # h[0] = float32(1/m)
        np.testing.assert_allclose(orc.cost(q, h, z[None])[0], ref, rtol=1e-12)


@pytest.mark.parametrize("beta", [0.2, 0.5, 1.0, 2.0])
def test_noiseless_template_is_recovered_strictly(orc, beta):
    """z = A s_{d*} (no background): by Hoelder, sum_t s_{d*} s_d^beta < sum_t s_{d*}^{1+beta} for every
    d != d*, so the minimum-divergence argmax is exactly d* and strict."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 300
    q = orc.params(T, len(h), peak, beta=beta)
    for dstar in (q.dmin, 130, q.dmax):
        z = np.zeros(T)
        z[dstar - peak:dstar - peak + len(h)] = 1e4 * h
        C = orc.cost(q, h, z[None])[0]
        k = dstar - q.dmin
        assert int(np.argmax(C)) == k
        others = np.delete(C, k)
        assert C[k] > others.max() * (1 + 1e-9)
        est = orc.estimate(q, h, z[None])
        assert int(est["argmax"][0]) == dstar


def test_template_power_integral_is_shift_invariant(orc):
    """On the full-support range the integral of f0^(1+beta) does not depend on d (the condition under
    Eq. beta_div2); just outside it does, and the domain check rejects such ranges."""
    h, peak = synth.asymmetric_irf(L=20)
    T = 70
    beta = 0.4
    q = orc.params(T, len(h), peak, beta=beta)
    ref = float(np.sum(h.astype(np.float64) ** (1 + beta)))
    vals = [orc.template_power_sum(q, h, d, 1 + beta) for d in range(q.dmin, q.dmax + 1)]
    np.testing.assert_allclose(vals, ref, rtol=1e-13)
    assert orc.template_power_sum(q, h, q.dmin - 1, 1 + beta) < ref * (1 - 1e-6)
    assert orc.template_power_sum(q, h, q.dmax + 1, 1 + beta) < ref * (1 - 1e-6)
    assert orc.check_domain(orc.params(T, len(h), peak, dmin=peak - 1)) != 0
    assert orc.check_domain(orc.params(T, len(h), peak, dmax=T - len(h) + peak + 1)) != 0
    assert orc.check_domain(orc.params(T, len(h), peak, beta=0.0)) != 0


# ------------------------------------------------------------------------------------------------------
# Pseudo-posterior and its moments (Eq. approx_post, Sec. II-C)
# ------------------------------------------------------------------------------------------------------


def _sum_int(a, b):
    return (a + b) * (b - a + 1) / 2.0


def _sum_sq(a, b):
    f = lambda n: n * (n + 1) * (2 * n + 1) / 6.0
    return f(b) - f(a - 1)


@pytest.mark.parametrize("beta", [0.3, 0.5, 1.0])
def test_one_photon_box_irf_closed_form(orc, beta):
    """One photon at t0 and a box IRF (h = 1/L): C(d) = L^-beta on the L depths whose template covers t0,
    0 elsewhere. With a uniform prior the pseudo-posterior weights are E = exp(lambda L^-beta) on that window
    and 1 elsewhere, lambda = (beta+1)/beta (Eq. beta_CE), so the moments are ratios of arithmetic series and
    the argmax is the window's first depth."""
    L, T, peak = 8, 90, 3
    h = np.full(L, 1.0 / L, np.float32)          # 1/8 is exact in float32
    t0 = 40
    z = np.zeros(T)
    z[t0] = 1.0
    q = orc.params(T, L, peak, beta=beta)
    a, b = q.dmin, q.dmax
    w0, w1 = t0 + peak - L + 1, t0 + peak
    E = math.exp((beta + 1) / beta * L ** (-beta))
    S0 = (b - a + 1) + (E - 1) * L
    S1 = _sum_int(a, b) + (E - 1) * _sum_int(w0, w1)
    S2 = _sum_sq(a, b) + (E - 1) * _sum_sq(w0, w1)
    mu = S1 / S0
    var = S2 / S0 - mu * mu
    est = orc.estimate(q, h, z[None])
    assert int(est["argmax"][0]) == w0
    np.testing.assert_allclose(est["mu"][0], mu, rtol=1e-12)
    np.testing.assert_allclose(est["var"][0], var, rtol=1e-9)


def test_translation_shifts_estimate(orc):
    """Shifting the histogram and the prior mean by delta bins shifts argmax and mean by delta and leaves
    the variance unchanged (away from the domain edges)."""
    h, peak = synth.asymmetric_irf(L=30)
    T = 400
    q = orc.params(T, len(h), peak, beta=0.5)
    rng = _rng(4)
    z = np.zeros(T)
    z[100:300] = rng.poisson(0.3, size=200)           # zeros near both ends, so shifts never wrap photons
    z[150 - peak:150 - peak + len(h)] += rng.poisson(8 * h)
    for delta in (1, 17, -23):
        z1 = z
        z2 = np.roll(z, delta)
        e1 = orc.estimate(q, h, z1[None], prior_mu=[160.0], prior_var=[300.0])
        e2 = orc.estimate(q, h, z2[None], prior_mu=[160.0 + delta], prior_var=[300.0])
        assert int(e2["argmax"][0]) == int(e1["argmax"][0]) + delta
        np.testing.assert_allclose(e2["mu"][0], e1["mu"][0] + delta, rtol=1e-12)
        np.testing.assert_allclose(e2["var"][0], e1["var"][0], rtol=1e-8)


def test_large_count_flat_prior_concentrates(orc):
    """Symmetric IRF, many photons exactly on a template, uniform prior: mean -> d*, variance -> 0."""
    h, peak = synth.gaussian_irf(3.0, 12)
    T = 200
    q = orc.params(T, len(h), peak, beta=0.5)
    z = np.zeros(T)
    z[90 - peak:90 - peak + len(h)] = np.rint(2000 * h)
    e = orc.estimate(q, h, z[None])
    assert int(e["argmax"][0]) == 90
    assert abs(e["mu"][0] - 90) < 1e-6
    assert e["var"][0] < 1e-6


# ------------------------------------------------------------------------------------------------------
# Spatio-temporal prior and filter step (Eq. predict, Eq. KL_div, Algorithm 1)
# ------------------------------------------------------------------------------------------------------

NU_ASYM = np.array([0.05, 0.10, 0.0, 0.15, 0.40, 0.20, 0.0, 0.10, 0.0])


def test_empty_histogram_posterior_is_the_mixture_prior(orc):
    """With no photons the pseudo-posterior is the prior of Eq. predict, a Gaussian mixture whose mean and
    variance have closed forms: mu = sum nu_c m_c, var = sum nu_c (s_c^2 + m_c^2) - mu^2 with
    s_c^2 = var_c + sigma_RW^2. On an integer grid far from the domain edges the discrete moments equal
    these to ~exp(-2 pi^2 s^2). An asymmetric stencil catches transposed or mirrored neighbour offsets."""
    h, peak = synth.gaussian_irf(3.0, 12)
    T = 1200
    sig2 = GOLD["sigma_rw2"]
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=sig2, nu=NU_ASYM)
    H = W = 3
    rng = _rng(5)
    mu_in = rng.uniform(560, 640, size=(H, W))
    var_in = rng.uniform(0.5, 20.0, size=(H, W))
    z = np.zeros((H, W, T))
    out = orc.filter_step(q, h, z, mu_in, var_in)
    m = []
    s2 = []
    nus = []
    for k in range(9):               # neighbour (dy, dx) = (k // 3 - 1, k % 3 - 1) of the centre (1, 1)
        if NU_ASYM[k] > 0:
            nus.append(NU_ASYM[k])
            m.append(mu_in[1 + k // 3 - 1, 1 + k % 3 - 1])
            s2.append(var_in[1 + k // 3 - 1, 1 + k % 3 - 1] + sig2)
    nus, m, s2 = map(np.array, (nus, m, s2))
    mu = np.sum(nus * m)
    var = np.sum(nus * (s2 + m * m)) - mu * mu
    np.testing.assert_allclose(out["mu"][1, 1], mu, rtol=1e-10)
    np.testing.assert_allclose(out["var"][1, 1], var, rtol=1e-8)


def test_uniform_state_makes_weights_irrelevant(orc):
    """A uniform state field makes every mixture component identical, so the result cannot depend on nu."""
    h, peak = synth.asymmetric_irf(L=24)
    T = 200
    rng = _rng(6)
    z = rng.poisson(0.4, size=(4, 5, T)).astype(np.float64)
    mu_in = np.full((4, 5), 101.0)
    var_in = np.full((4, 5), 40.0)
    outs = []
    for nu in (synth.cross_weights(0.5), NU_ASYM, np.eye(1, 9, 4).ravel()):
        q = orc.params(T, len(h), peak, beta=0.5, nu=nu)
        o = orc.filter_step(q, h, z, mu_in, var_in)
        outs.append(o)
    for o in outs[1:]:
        # interior pixel only: edge pixels see out-of-view (flat) components with nu-dependent weight
        np.testing.assert_array_equal(o["argmax"][1:-1, 1:-1], outs[0]["argmax"][1:-1, 1:-1])
        np.testing.assert_allclose(o["mu"][1:-1, 1:-1], outs[0]["mu"][1:-1, 1:-1], rtol=1e-12)
        np.testing.assert_allclose(o["var"][1:-1, 1:-1], outs[0]["var"][1:-1, 1:-1], rtol=1e-10)


def test_filter_prior_with_centre_weight_only_equals_gaussian_prior(orc):
    """nu = centre only: the prior is N(mu_in, var_in + sigma_RW^2) and the filter step equals the
    single-frame estimate with that Gaussian prior."""
    h, peak = synth.asymmetric_irf(L=24)
    T = 150
    rng = _rng(7)
    z = rng.poisson(0.5, size=(3, 4, T)).astype(np.float64)
    mu_in = rng.uniform(40, 120, size=(3, 4))
    var_in = rng.uniform(1, 50, size=(3, 4))
    q = orc.params(T, len(h), peak, beta=0.7, sigma_rw2=2.5, nu=np.eye(1, 9, 4).ravel())
    f = orc.filter_step(q, h, z, mu_in, var_in)
    e = orc.estimate(q, h, z, prior_mu=mu_in, prior_var=var_in + 2.5)
    np.testing.assert_array_equal(f["argmax"], e["argmax"])
    np.testing.assert_allclose(f["mu"], e["mu"], rtol=1e-12)
    np.testing.assert_allclose(f["var"], e["var"], rtol=1e-10)


def _cube(seed, H, W, T, h, peak):
    rng = _rng(seed)
    d = rng.integers(peak + 10, T - len(h) + peak - 10, size=(H, W))
    z = rng.poisson(0.2, size=(H, W, T)).astype(np.float64)
    for y in range(H):
        for x in range(W):
            z[y, x, d[y, x] - peak:d[y, x] - peak + len(h)] += rng.poisson(4 * h)
    return z


def test_filter_is_translation_equivariant(orc):
    """Shifting the whole input (histograms and state) by one pixel shifts interior outputs by one pixel."""
    h, peak = synth.asymmetric_irf(L=16)
    T = 120
    q = orc.params(T, len(h), peak, beta=0.5, nu=NU_ASYM)
    H, W = 6, 7
    z = _cube(8, H, W, T, h, peak)
    rng = _rng(9)
    mu_in = rng.uniform(30, 100, size=(H, W))
    var_in = rng.uniform(1, 30, size=(H, W))
    a = orc.filter_step(q, h, z, mu_in, var_in)
    b = orc.filter_step(q, h, np.roll(z, (1, 1), (0, 1)), np.roll(mu_in, (1, 1), (0, 1)),
                        np.roll(var_in, (1, 1), (0, 1)))
    for k in ("argmax", "mu", "var"):
        np.testing.assert_allclose(b[k][2:-1, 2:-1], a[k][1:-2, 1:-2], rtol=1e-12)


def test_edge_pixels_see_flat_components(orc):
    """An edge pixel equals the same pixel inside a larger image whose extra ring is absent (Sec. III-A:
    out-of-view neighbours contribute the weakly informative Gaussian)."""
    h, peak = synth.asymmetric_irf(L=16)
    T = 120
    q = orc.params(T, len(h), peak, beta=0.5, nu=NU_ASYM)
    H, W = 4, 5
    z = _cube(10, H, W, T, h, peak)
    rng = _rng(11)
    mu_in = rng.uniform(30, 100, size=(H, W))
    var_in = rng.uniform(1, 30, size=(H, W))
    a = orc.filter_step(q, h, z, mu_in, var_in)
    zp = np.zeros((H + 2, W + 2, T))
    zp[1:-1, 1:-1] = z
    mp = np.full((H + 2, W + 2), 500.0)
    vp = np.full((H + 2, W + 2), 2.0)
    mp[1:-1, 1:-1] = mu_in
    vp[1:-1, 1:-1] = var_in
    pres = np.zeros((H + 2, W + 2), np.uint8)
    pres[1:-1, 1:-1] = 1
    b = orc.filter_step(q, h, zp, mp, vp, present_in=pres)
    for k in ("argmax", "mu", "var"):
        np.testing.assert_allclose(b[k][1:-1, 1:-1], a[k], rtol=1e-12)
    # a faulty neighbour is treated like an absent one
    fa = np.zeros((H, W), np.uint8)
    fa[2, 2] = 1
    pr = np.ones((H, W), np.uint8)
    pr[2, 2] = 0
    c = orc.filter_step(q, h, z, mu_in, var_in, faulty=fa)
    d = orc.filter_step(q, h, z, mu_in, var_in, present_in=pr)
    for k in ("argmax", "mu", "var"):
        m = np.ones((H, W), bool)
        m[2, 2] = False
        np.testing.assert_allclose(c[k][m], d[k][m], rtol=1e-12)


def test_faulty_pixel_posterior_is_prior(orc):
    """A faulty pixel has no observations: its pseudo-posterior is its prior (Sec. III-B), the same as an
    empty histogram. Its presence probability is 0.5, so in every prior (its own included) it enters as
    the weakly informative Gaussian, like an absent pixel."""
    h, peak = synth.asymmetric_irf(L=16)
    T = 120
    q = orc.params(T, len(h), peak, beta=0.5, nu=synth.cross_weights(0.5))
    H, W = 3, 3
    z = _cube(12, H, W, T, h, peak)
    mu_in = np.full((H, W), 60.0)
    var_in = np.full((H, W), 5.0)
    fa = np.zeros((H, W), np.uint8)
    fa[1, 1] = 1
    a = orc.filter_step(q, h, z, mu_in, var_in, faulty=fa)
    z0 = z.copy()
    z0[1, 1] = 0
    pr = np.ones((H, W), np.uint8)
    pr[1, 1] = 0
    b = orc.filter_step(q, h, z0, mu_in, var_in, present_in=pr)
    for k in ("argmax", "mu", "var"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12)


def test_dependency_cone(orc):
    """After n frames a pixel depends only on inputs within Chebyshev distance n: a crop with an n-pixel
    margin reproduces the full-image result on its interior (this is how large frames are checked)."""
    h, peak = synth.asymmetric_irf(L=16)
    T = 100
    q = orc.params(T, len(h), peak, beta=0.5, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    H, W, N = 9, 10, 3
    zs = [_cube(20 + n, H, W, T, h, peak) for n in range(N)]
    mu, var = orc.state_init(q, H, W)
    for n in range(N):
        o = orc.filter_step(q, h, zs[n], mu, var)
        mu, var = o["mu"], o["var"]
    y0, y1, x0, x1 = 2, 7, 3, 8            # crop with a margin of N around [5:4, 6:5] -> interior [5,6]
    cm, cv = orc.state_init(q, y1 - y0, x1 - x0)
    for n in range(N):
        o = orc.filter_step(q, h, zs[n][y0:y1, x0:x1], cm, cv)
        cm, cv = o["mu"], o["var"]
    yy, xx = 2, 2                          # crop coordinates of full-image pixel (4, 5)
    assert cm[yy, xx] == pytest.approx(mu[4, 5], rel=1e-12)
    assert cv[yy, xx] == pytest.approx(var[4, 5], rel=1e-12)


# ------------------------------------------------------------------------------------------------------
# Background and reflectivity (Sec. II-E, MLE under Eq. lik_bg_poisson)
# ------------------------------------------------------------------------------------------------------


def test_intensity_box_irf_closed_form(orc):
    """Box IRF (h = 1/L on the window): the Poisson MLE has per-region rates, b = K_out/(T-L) and
    r/L + b = K_in/L, i.e. r = K_in - L K_out/(T-L) when that is >= 0; otherwise r = 0, b = K/T."""
    L, T, peak = 8, 200, 4
    h = np.full(L, 1.0 / L, np.float32)          # 1/8 is exact in float32
    q = orc.params(T, L, peak)
    rng = _rng(13)
    for trial in range(20):
        z = rng.poisson(rng.uniform(0.05, 2.0), size=T).astype(np.float64)
        d = int(rng.integers(q.dmin, q.dmax + 1))
        z[d - peak:d - peak + L] += rng.poisson(rng.uniform(0, 5), size=L) * (trial % 3 != 0)
        Kin = z[d - peak:d - peak + L].sum()
        Kout = z.sum() - Kin
        r_ref = Kin - L * Kout / (T - L)
        b_ref = Kout / (T - L)
        if r_ref < 0:
            r_ref, b_ref = 0.0, z.sum() / T
        r, b = orc.intensity_mle(q, h, z, d)
        assert r == pytest.approx(r_ref, rel=1e-9, abs=1e-9)
        assert b == pytest.approx(b_ref, rel=1e-9, abs=1e-12)


def test_intensity_noiseless_no_background(orc):
    """All photons on the template and none outside: b = 0 and r = K / sum(h)."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 500
    q = orc.params(T, len(h), peak)
    z = np.zeros(T)
    z[200 - peak:200 - peak + len(h)] = np.rint(500 * h)
    r, b = orc.intensity_mle(q, h, z, 200)
    assert b == pytest.approx(0.0, abs=1e-9)
    assert r == pytest.approx(z.sum() / float(np.sum(h.astype(np.float64))), rel=1e-9)


def test_intensity_matches_generic_optimizer(orc):
    """The MLE agrees with scipy's bounded optimiser on the 2-D Poisson log-likelihood (KKT point)."""
    opt = pytest.importorskip("scipy.optimize")
    h, peak = synth.asymmetric_irf(L=48)
    hd = h.astype(np.float64)
    T = 400
    q = orc.params(T, len(h), peak)
    rng = _rng(14)
    for trial in range(8):
        d = int(rng.integers(q.dmin, q.dmax + 1))
        b_true = rng.uniform(0.005, 0.3)
        r_true = rng.uniform(2, 40)
        lam = np.full(T, b_true)
        lam[d - peak:d - peak + len(h)] += r_true * hd
        z = rng.poisson(lam).astype(np.float64)
        r, b = orc.intensity_mle(q, h, z, d)

        def nll(v):
            rr, bb = v
            m = np.full(T, bb)
            m[d - peak:d - peak + len(h)] += rr * hd
            m = np.maximum(m, 1e-300)
            return -(np.sum(z * np.log(m)) - m.sum())

        res = opt.minimize(nll, x0=[max(r, 1.0), max(b, 1e-3)], bounds=[(0, None), (1e-12, None)],
                           method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12, maxiter=10000))
        assert nll([r, b]) <= res.fun + 1e-7
        assert r == pytest.approx(res.x[0], rel=1e-3, abs=1e-3)
        assert b == pytest.approx(res.x[1], rel=1e-3, abs=1e-6)


def _box_closed_form(z, d, L, peak):
    """(r, b) of the box-IRF Poisson MLE with the window at depth d (closed form, see above)."""
    T = len(z)
    Kin = z[d - peak:d - peak + L].sum()
    Kout = z.sum() - Kin
    r, b = Kin - L * Kout / (T - L), Kout / (T - L)
    if r < 0:
        r, b = 0.0, z.sum() / T
    return r, b


def test_intensity_rule_per_pixel(orc):
    """The per-pixel rule of Sec. II-E around the MLE: an absent pixel has r = 0 and b = K/T (K counted here by
    hand); a faulty pixel has r = b = 0; a present pixel has the box-IRF closed form with the window at
    round-half-even(mu) (x.5 goes to the even neighbour, x.4 down, x.6 up); present = NULL means every pixel is
    present; an explicit template position overrides mu."""
    L, T, peak = 8, 160, 3
    h = np.full(L, 1.0 / L, np.float32)
    q = orc.params(T, L, peak)
    rng = _rng(31)
    # eight pixels, each with a strong burst whose window position differs by one bin between the two
    # roundings, so that the wrong rounding gives a visibly different (r, b)
    mus = np.array([40.5, 41.5, 40.4, 40.6, 57.5, 90.5, 91.5, 77.0])
    P = len(mus)
    z = rng.poisson(0.3, size=(P, T)).astype(np.float64)
    for p, m in enumerate(mus):
        lo = int(math.floor(m)) - peak
        z[p, lo:lo + L + 1] += rng.poisson(6.0, size=L + 1)
        z[p, lo] += 9.0          # the bin that only the lower window holds
        z[p, lo + L] += 2.0      # the bin that only the upper window holds
    expect_pos = np.array([40, 42, 40, 41, 58, 90, 92, 77])
    assert np.array_equal(np.rint(mus).astype(int), expect_pos)  # numpy rounds half to even as well
    present = np.array([1, 1, 1, 1, 0, 1, 1, 1], np.uint8)
    faulty = np.array([0, 0, 0, 0, 0, 0, 0, 1], np.uint8)
    r, b = orc.intensity(q, h, z, mus, present=present, faulty=faulty)
    for p in range(P):
        if faulty[p]:
            assert r[p] == 0.0 and b[p] == 0.0
        elif not present[p]:
            assert r[p] == 0.0
            assert b[p] == pytest.approx(float(sum(z[p])) / T, rel=1e-15)
        else:
            rr, bb = _box_closed_form(z[p], int(expect_pos[p]), L, peak)
            fl = int(math.floor(mus[p]))
            other = fl + 1 if expect_pos[p] == fl else fl  # the other neighbour of mu
            ro, _ = _box_closed_form(z[p], other, L, peak)
            assert abs(rr - ro) > 0.5, "fixture must separate the two roundings"
            assert r[p] == pytest.approx(rr, rel=1e-9, abs=1e-9)
            assert b[p] == pytest.approx(bb, rel=1e-9, abs=1e-12)
    r_all, b_all = orc.intensity(q, h, z, mus)
    for p in range(P):
        rr, bb = _box_closed_form(z[p], int(expect_pos[p]), L, peak)
        assert r_all[p] == pytest.approx(rr, rel=1e-9, abs=1e-9)
        assert b_all[p] == pytest.approx(bb, rel=1e-9, abs=1e-12)
    dr = np.array([45, 46, 47, 48, 49, 50, 51, 52], np.int32)
    r_dr, b_dr = orc.intensity(q, h, z, mus, dr=dr)
    for p in range(P):
        rr, bb = _box_closed_form(z[p], int(dr[p]), L, peak)
        assert r_dr[p] == pytest.approx(rr, rel=1e-9, abs=1e-9)
        assert b_dr[p] == pytest.approx(bb, rel=1e-9, abs=1e-12)


# ------------------------------------------------------------------------------------------------------
# Multispectral data (Appendix, Eq. div_MSL): M(d) = prod_l C_l(d) / K_l
# ------------------------------------------------------------------------------------------------------


def _msl_inputs(seed, nb=3, H=3, W=4, T=220, L=24, peak=8, signal=25.0, bg=0.05):
    hb = synth.band_irfs(nb, L, peak)
    rng = _rng(seed)
    dmin, dmax = peak, T - L + peak
    depth = rng.integers(dmin + 3, dmax - 3, size=(H, W))
    z = np.empty((nb, H, W, T))
    for b in range(nb):
        mean = synth.expected_counts(torch.from_numpy(depth), torch.full((H, W), signal, dtype=torch.float64), bg,
                                     torch.from_numpy(hb[b]), peak, T)
        z[b] = rng.poisson(mean.numpy())
    return hb, peak, depth, z


def test_msl_one_band_is_the_single_band_estimate(orc):
    """With one band, M = C / K and lambda K M = lambda C: the single-band pseudo-posterior of Eq. approx_post."""
    hb, peak, _, z = _msl_inputs(41, nb=1)
    q = orc.params(z.shape[-1], hb.shape[1], peak, beta=0.6)
    rng = _rng(42)
    pm = rng.uniform(q.dmin, q.dmax, size=z.shape[1:3])
    pv = rng.uniform(10, 400, size=z.shape[1:3])
    for prior in (None, (pm, pv)):
        a = orc.estimate_msl(q, hb, z, *(prior or (None, None)))
        e = orc.estimate(q, hb[0], z[0], *(prior or (None, None)))
        assert np.array_equal(a["argmax"], e["argmax"])
        np.testing.assert_allclose(a["mu"], e["mu"], rtol=1e-12)
        np.testing.assert_allclose(a["var"], e["var"], rtol=1e-9)


def test_msl_photon_list_form(orc):
    """Eq. div_MSL is written over the photons' times of arrival: prod_l (1/K_l) sum_k h_l[y_{l,k} - d + peak]^beta,
    evaluated here photon by photon from lists drawn from the histograms, against the oracle's histogram form."""
    hb, peak, _, z = _msl_inputs(43, nb=3)
    nb, H, W, T = z.shape
    L = hb.shape[1]
    beta = 0.45
    q = orc.params(T, L, peak, beta=beta)
    M = orc.estimate_msl(q, hb, z, want_cost=True)["M"]
    d = np.arange(q.dmin, q.dmax + 1)
    for y in range(H):
        for x in range(W):
            ref = np.ones(d.size)
            for b in range(nb):
                ys = np.repeat(np.arange(T), z[b, y, x].astype(int))
                if ys.size == 0:
                    continue
                j = ys[None, :] - d[:, None] + peak
                inside = (j >= 0) & (j < L)
                g = np.where(inside, hb[b].astype(np.float64)[np.clip(j, 0, L - 1)], 0.0) ** beta
                ref *= g.sum(axis=1) / ys.size
            np.testing.assert_allclose(M[y, x], ref, rtol=1e-12, atol=1e-300)


def test_msl_identical_bands(orc):
    """nb copies of one band: M = (C / K)^nb, so the minimum-divergence estimate is the single band's, and the log
    pseudo-posterior is lambda nb K (C / K)^nb (the data's K counted once per band)."""
    hb, peak, _, z = _msl_inputs(44, nb=1)
    T, L = z.shape[-1], hb.shape[1]
    beta = 0.5
    q = orc.params(T, L, peak, beta=beta)
    one = orc.estimate(q, hb[0], z[0], want_ell=True)
    lam = (beta + 1) / beta
    for nb in (2, 3):
        a = orc.estimate_msl(q, np.repeat(hb, nb, 0), np.repeat(z, nb, 0), want_ell=True)
        assert np.array_equal(a["argmax"], one["argmax"])
        K = z[0].sum(-1, keepdims=True)
        C = one["ell"] / lam
        np.testing.assert_allclose(a["ell"], lam * nb * K * (C / K) ** nb, rtol=1e-10)


@pytest.mark.parametrize("beta", [0.2, 0.7, 1.0])
def test_msl_noiseless_templates_are_recovered(orc, beta):
    """Each band holds A_l s_{l,d*} with its own IRF and amplitude, no background: every factor C_l / K_l peaks
    strictly at d* (Hoelder, as for one band), so the product does too."""
    nb, L, peak, T = 4, 24, 8, 180
    hb = synth.band_irfs(nb, L, peak).astype(np.float64)
    q = orc.params(T, L, peak, beta=beta)
    rng = _rng(45)
    for trial in range(6):
        ds = int(rng.integers(q.dmin, q.dmax + 1))
        z = np.zeros((nb, 1, 1, T))
        for b in range(nb):
            z[b, 0, 0, ds - peak:ds - peak + L] = rng.uniform(1e3, 1e5) * hb[b]
        a = orc.estimate_msl(q, hb, z)
        assert int(a["argmax"][0, 0]) == ds


def test_msl_empty_band_and_band_order(orc):
    """A band without photons contributes no factor; the bands' order does not matter."""
    hb, peak, _, z = _msl_inputs(46, nb=3)
    q = orc.params(z.shape[-1], hb.shape[1], peak, beta=0.5)
    base = orc.estimate_msl(q, hb, z, want_cost=True)
    ze = np.concatenate([z, np.zeros_like(z[:1])])
    he = np.concatenate([hb, synth.band_irfs(4, hb.shape[1], peak)[3:]])
    e = orc.estimate_msl(q, he, ze, want_cost=True)
    np.testing.assert_array_equal(e["M"], base["M"])
    perm = [2, 0, 1]
    r = orc.estimate_msl(q, hb[perm], z[perm], want_cost=True)
    np.testing.assert_allclose(r["M"], base["M"], rtol=1e-13)
    assert np.array_equal(r["argmax"], base["argmax"])
    zero = orc.estimate_msl(q, hb, np.zeros_like(z))
    prior_free = (q.dmin + q.dmax) / 2.0
    np.testing.assert_allclose(zero["mu"], prior_free, rtol=1e-12)


# ------------------------------------------------------------------------------------------------------
# Sub-bin depth (fine candidate grid, continuous IRF by linear interpolation of the taps)
# ------------------------------------------------------------------------------------------------------


def test_fine_grid_with_one_step_per_bin_is_the_integer_estimate(orc):
    """S = 1: the fine-grid estimate is the integer-grid estimate (same candidates, same taps)."""
    h, peak = synth.asymmetric_irf(L=24)
    T = 200
    q = orc.params(T, len(h), peak, beta=0.6)
    rng = _rng(61)
    z = rng.poisson(0.3, size=(3, T)).astype(np.float64)
    for p, d in enumerate((40, 90, 150)):
        z[p, d - peak:d - peak + len(h)] += rng.poisson(20 * h)
    pm, pv = np.array([60.0, 100.0, 140.0]), np.array([400.0, 900.0, 90.0])
    for prior in ((None, None), (pm, pv)):
        a = orc.estimate(q, h, z, prior_mu=prior[0], prior_var=prior[1])
        b = orc.estimate_fine(q, 1, h, z, prior_mu=prior[0], prior_var=prior[1])
        assert np.array_equal(a["argmax"], b["argmax_k"] + q.dmin)
        assert np.allclose(a["mu"], b["mu"], rtol=1e-13) and np.allclose(a["var"], b["var"], rtol=1e-12)


def test_fine_grid_half_bin_is_the_average_at_beta_one(orc):
    """beta = 1: the data term is linear in the template, and the template at d + 1/2 is the average of the
    templates at d and d + 1 (linear interpolation, zero beyond the taps), so C(d + 1/2) = (C(d) + C(d+1)) / 2."""
    h, peak = synth.asymmetric_irf(L=30)
    T = 180
    q = orc.params(T, len(h), peak, beta=1.0)
    rng = _rng(67)
    z = rng.poisson(1.5, size=(2, T)).astype(np.float64)
    e = orc.estimate_fine(q, 2, h, z, want_cost=True)
    C = e["cost"]
    assert np.allclose(C[:, 1::2], 0.5 * (C[:, 0:-1:2] + C[:, 2::2]), rtol=1e-12, atol=1e-12)
    Ci = orc.cost(q, h, z)
    assert np.allclose(C[:, 0::2], Ci, rtol=1e-12)


def test_fine_grid_recovers_a_fractional_surface_exactly(orc):
    """The histogram equal to A s_{d*} (expected counts of a surface at a fractional depth d* on the fine grid, no
    background, real-valued) makes the beta-divergence to s_d zero at d = d* and positive elsewhere, so with a flat
    prior the maximiser is d* itself, for every beta. (Without the template-power term the maximiser is pulled
    to whole bins, where the interpolated template is more peaked.)"""
    h, peak = synth.gaussian_irf(2.5, 10)
    T, S = 160, 8
    hp = np.concatenate([[0.0], h.astype(np.float64), [0.0]])
    for beta in (0.3, 0.7, 1.0):
        q = orc.params(T, len(h), peak, beta=beta)
        for kstar in (0, 3, 5):
            dstar = 70 + kstar / S
            x = np.arange(T) - dstar + peak
            z = 1e4 * np.interp(x, np.arange(-1, len(h) + 1), hp, left=0.0, right=0.0)
            e = orc.estimate_fine(q, S, h, z[None])
            assert q.dmin + e["argmax_k"][0] / S == dstar


def test_fine_grid_translation(orc):
    """Shifting the histogram and the prior mean by one bin shifts the fine argmax by S and the mean by 1."""
    h, peak = synth.asymmetric_irf(L=20)
    T = 160
    q = orc.params(T, len(h), peak, beta=0.4)
    rng = _rng(71)
    z = rng.poisson(0.2, size=T).astype(np.float64)
    z[60 - peak:60 - peak + len(h)] += rng.poisson(15 * h)
    z1 = np.concatenate([[0.0], z[:-1]])                 # one bin later (the last bin is empty)
    S = 4
    a = orc.estimate_fine(q, S, h, z[None], prior_mu=np.array([70.0]), prior_var=np.array([300.0]))
    b = orc.estimate_fine(q, S, h, z1[None], prior_mu=np.array([71.0]), prior_var=np.array([300.0]))
    assert b["argmax_k"][0] == a["argmax_k"][0] + S
    # edge effects: the shifted histogram loses its last bin and sees a shorter candidate range; the posterior
    # mass there is negligible for this surface
    assert b["mu"][0] == pytest.approx(a["mu"][0] + 1.0, abs=1e-6)
    assert b["var"][0] == pytest.approx(a["var"][0], rel=1e-6)


def test_fine_grid_empty_histogram_gives_the_prior_moments(orc):
    """No photons: the weights are the Gaussian prior sampled every 1/S bin; away from the domain edges its
    mean and variance are the prior's (Poisson summation: the grid error is far below 1e-9)."""
    h, peak = synth.asymmetric_irf(L=16)
    T = 400
    q = orc.params(T, len(h), peak, beta=0.5)
    z = np.zeros((2, T))
    e = orc.estimate_fine(q, 3, h, z, prior_mu=np.array([180.0, 201.3]), prior_var=np.array([64.0, 30.25]))
    assert np.allclose(e["mu"], [180.0, 201.3], atol=1e-9)
    assert np.allclose(e["var"], [64.0, 30.25], rtol=1e-9)


# ------------------------------------------------------------------------------------------------------
# Detection surrogate (BIC-approximated Bayes factor under Eq. lik_bg_poisson, combined with pi0)
# ------------------------------------------------------------------------------------------------------


def _logit(p):
    return math.log(p) - math.log1p(-p)


def test_detect_box_irf_likelihood_ratio_closed_form(orc):
    """Box IRF: the maximised two-region Poisson likelihood ratio is
    K_in log(K_in T / (K L)) + K_out log(K_out T / (K (T - L))) when the window rate exceeds the outside
    rate, and 0 otherwise (then r = 0 is the maximiser)."""
    L, T, peak = 8, 200, 4
    h = np.full(L, 1.0 / L, np.float32)
    q = orc.params(T, L, peak)
    rng = _rng(41)
    for trial in range(24):
        z = rng.poisson(rng.uniform(0.05, 1.5), size=T).astype(np.float64)
        d = int(rng.integers(q.dmin, q.dmax + 1))
        z[d - peak:d - peak + L] += rng.poisson(rng.uniform(0, 4), size=L) * (trial % 3 != 0)
        K = z.sum()
        Kin = z[d - peak:d - peak + L].sum()
        Kout = K - Kin
        if Kin / L > Kout / (T - L):
            ref = (Kin * math.log(Kin * T / (K * L)) if Kin > 0 else 0.0) + \
                  (Kout * math.log(Kout * T / (K * (T - L))) if Kout > 0 else 0.0)
        else:
            ref = 0.0
        out = orc.detect(q, h, z[None, :], np.array([float(d)]), pi0=np.array([0.3]))
        assert out["llr"][0] == pytest.approx(ref, rel=1e-9, abs=1e-9)


def test_detect_bayes_factor_does_not_depend_on_the_prior(orc):
    """logit(pi) - logit(pi0) is the log Bayes factor: the same for every pi0 (and it is LLR - log(K)/2),
    pi grows with pi0, and the decision follows pi > 0.5."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 600
    q = orc.params(T, len(h), peak)
    rng = _rng(43)
    P = 12
    z = rng.poisson(0.05, size=(P, T)).astype(np.float64)
    mu = rng.integers(q.dmin, q.dmax + 1, size=P).astype(np.float64)
    for p in range(P):
        d = int(mu[p])
        z[p, d - peak:d - peak + len(h)] += rng.poisson((p % 4) * 0.25 * h / h.max())
    outs = [orc.detect(q, h, z, mu, pi0=np.full(P, v)) for v in (0.1, 0.5, 0.9)]
    K = z.sum(1)
    checked = 0
    for p in range(P):
        if not all(1e-9 < o["pi"][p] < 1 - 1e-9 for o in outs):
            continue  # saturated: the log Bayes factor is not recoverable from pi in double precision
        checked += 1
        lbf = [_logit(o["pi"][p]) - _logit(v) for o, v in zip(outs, (0.1, 0.5, 0.9))]
        assert lbf[0] == pytest.approx(lbf[1], abs=1e-7) and lbf[2] == pytest.approx(lbf[1], abs=1e-7)
        assert lbf[1] == pytest.approx(outs[1]["llr"][p] - 0.5 * math.log(max(K[p], 1.0)), abs=1e-7)
        assert outs[0]["pi"][p] < outs[1]["pi"][p] < outs[2]["pi"][p]
        for o in outs:
            assert o["present"][p] == (o["pi"][p] > 0.5)
            if o["present"][p]:
                r, b = orc.intensity_mle(q, h, z[p], int(mu[p]))
                assert (o["refl"][p], o["bg"][p]) == (pytest.approx(r, rel=1e-12), pytest.approx(b, rel=1e-12))
            else:
                assert o["refl"][p] == 0.0 and o["bg"][p] == pytest.approx(K[p] / T, rel=1e-12)
    assert checked >= 8
    assert sum(outs[1]["present"]) not in (0, P)  # both branches taken


def test_detect_limits(orc):
    """No photons: pi = pi0 (no evidence). Faulty: pi = 1/2, r = b = 0. A flat histogram: r = 0, LLR = 0 and
    pi < pi0. Photons only on the template: pi -> 1, b = 0, r = K / sum(h)."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 400
    q = orc.params(T, len(h), peak)
    d = 150
    z = np.zeros((4, T))
    z[1] = 3.0                                               # flat: exactly the background-only model
    z[2, d - peak:d - peak + len(h)] = np.rint(300 * h)      # noiseless template, no background
    z[3] = 2.0
    pi0 = np.array([0.7, 0.5, 0.5, 0.5])
    faulty = np.array([0, 0, 0, 1], np.uint8)
    o = orc.detect(q, h, z, np.full(4, float(d)), pi0=pi0, faulty=faulty)
    assert o["pi"][0] == pytest.approx(0.7, rel=1e-12) and o["llr"][0] == 0.0
    assert o["refl"][0] == 0.0 and o["bg"][0] == 0.0
    assert o["llr"][1] == pytest.approx(0.0, abs=1e-9) and o["pi"][1] < 0.5 and not o["present"][1]
    assert o["refl"][1] == 0.0 and o["bg"][1] == pytest.approx(3.0, rel=1e-12)
    assert o["pi"][2] > 1 - 1e-12 and o["present"][2]
    assert o["bg"][2] == pytest.approx(0.0, abs=1e-9)
    assert o["refl"][2] == pytest.approx(z[2].sum() / float(np.sum(h.astype(np.float64))), rel=1e-9)
    assert o["pi"][3] == 0.5 and not o["present"][3] and o["refl"][3] == 0.0 and o["bg"][3] == 0.0


def test_detect_mode_for_the_test_mean_for_the_estimate(orc):
    """The evidence is taken with the template at the pseudo-posterior mode dmap (the surface's photons there);
    the reported (r, b) of a present pixel use the depth point estimate round(mu), as in Sec. II-E."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 600
    q = orc.params(T, len(h), peak)
    z = np.zeros((1, T))
    z[0] += (np.arange(T) % 37 == 0)                         # a few background photons
    dtrue = 300
    z[0, dtrue - peak:dtrue - peak + len(h)] += np.rint(40 * h)
    mu = np.array([450.0])                                   # a mean pulled away from the surface
    on = orc.detect(q, h, z, mu, dmap=np.array([dtrue]))
    off = orc.detect(q, h, z, mu)                            # test at round(mu): no surface there
    r_m, b_m = orc.intensity_mle(q, h, z[0], dtrue)
    assert on["llr"][0] == pytest.approx(orc.log_lik_ratio(q, h, z[0], dtrue, r_m, b_m), rel=1e-12)
    assert on["llr"][0] > 50 and on["present"][0]
    assert off["llr"][0] < on["llr"][0] and not off["present"][0]
    r, b = orc.intensity_mle(q, h, z[0], 450)
    assert on["refl"][0] == pytest.approx(r, rel=1e-12, abs=1e-12) and on["bg"][0] == pytest.approx(b, rel=1e-12)


def test_detect_occam_term_of_the_depth_marginal(orc):
    """Laplace's method over the depth: a pseudo-posterior of variance var wider than the template costs
    (1/2) log(var / sigma_h^2) nats of evidence; narrower costs nothing. For a box IRF of L taps sigma_h^2 is
    the discrete-uniform variance (L^2 - 1) / 12."""
    L, T, peak = 9, 300, 4
    h = np.full(L, 1.0 / L)
    q = orc.params(T, L, peak)
    rng = _rng(53)
    z = rng.poisson(0.2, size=(1, T)).astype(np.float64)
    z[0, 100 - peak:100 - peak + 3] += 1                  # a weak surface: pi stays well inside (0, 1)
    s2 = (L * L - 1) / 12.0
    mu = np.array([100.0])
    base = orc.detect(q, h, z, mu, pi0=np.array([0.4]))
    x0 = _logit(base["pi"][0])
    assert abs(x0) < 20
    for var, shift in ((0.5 * s2, 0.0), (s2, 0.0), (s2 * math.e ** 2, 1.0), (s2 * math.e ** 5, 2.5)):
        o = orc.detect(q, h, z, mu, var=np.array([var]), pi0=np.array([0.4]))
        assert _logit(o["pi"][0]) == pytest.approx(x0 - shift, abs=1e-9)
        assert o["llr"][0] == base["llr"][0]


def test_detect_llr_is_the_maximum(orc):
    """The LLR at the intensity MLE is >= 0 and >= the ratio at any other (r, b) with r sum(h) + b T = K."""
    h, peak = synth.asymmetric_irf(L=48)
    T = 500
    q = orc.params(T, len(h), peak)
    rng = _rng(47)
    hs = float(np.sum(h.astype(np.float64)))
    for trial in range(10):
        z = rng.poisson(rng.uniform(0.01, 0.3), size=T).astype(np.float64)
        d = int(rng.integers(q.dmin, q.dmax + 1))
        z[d - peak:d - peak + len(h)] += rng.poisson(rng.uniform(0, 3) * h / h.max())
        o = orc.detect(q, h, z[None, :], np.array([float(d)]))
        llr = o["llr"][0]
        assert llr >= -1e-12
        r_hat, _ = orc.intensity_mle(q, h, z, d)
        K = z.sum()
        for r in np.linspace(0.0, 0.999 * K / hs, 17):
            assert orc.log_lik_ratio(q, h, z, d, r, (K - r * hs) / T) <= llr + 1e-9
        if r_hat > 0:
            assert orc.log_lik_ratio(q, h, z, d, r_hat, (K - r_hat * hs) / T) == pytest.approx(llr, abs=1e-12)


# ------------------------------------------------------------------------------------------------------
# Prior probability of presence (Eq. prior_detect)
# ------------------------------------------------------------------------------------------------------


def test_pi_propagation_fixed_points_and_symmetry(orc):
    nu = synth.cross_weights(GOLD["nu0"])
    H, W = 5, 6
    # constant pi with sum(nu) = 1 is a fixed point on interior pixels; 0.5 is a fixed point everywhere
    out = orc.pi_propagate(nu, np.full((H, W), 0.8))
    np.testing.assert_allclose(out[1:-1, 1:-1], 0.8, rtol=1e-12)
    np.testing.assert_allclose(orc.pi_propagate(nu, np.full((H, W), 0.5)), 0.5, rtol=0, atol=1e-15)
    # pi -> 1 - pi maps pi0 -> 1 - pi0 (logit is odd, sigmoid(-a) = 1 - sigmoid(a))
    pi = _rng(15).uniform(0.01, 0.99, size=(H, W))
    np.testing.assert_allclose(orc.pi_propagate(nu, 1 - pi), 1 - orc.pi_propagate(nu, pi), rtol=1e-12)
    # an edge pixel sees out-of-view neighbours as pi = 0.5 (logit 0): constant 0.8 is pulled toward 0.5
    corner = out[0, 0]
    assert 0.5 < corner < 0.8
    # nonlinear averaging of two opposite logits cancels exactly
    nu2 = np.zeros(9)
    nu2[3] = nu2[5] = 0.5
    pi2 = np.full((1, 3), 0.5)
    pi2[0, 0], pi2[0, 2] = 0.9, 0.1
    assert orc.pi_propagate(nu2, pi2)[0, 1] == pytest.approx(0.5, abs=1e-15)
    # faulty pixels are fixed at 0.5
    fa = np.zeros((H, W), np.uint8)
    fa[2, 3] = 1
    assert orc.pi_propagate(nu, pi, faulty=fa)[2, 3] == 0.5


# ------------------------------------------------------------------------------------------------------------
# Differentiable oracle (soft-argmax readout, gradients by autograd)
# ------------------------------------------------------------------------------------------------------------


def _diff_inputs(seed, H=4, W=5, T=90, N=3):
    h, peak = synth.asymmetric_irf(L=16)
    rng = _rng(seed)
    zs, refs = [], []
    for n in range(N):
        z = _cube(seed * 10 + n, H, W, T, h, peak)
        zs.append(z)
        refs.append(rng.uniform(peak + 10, T - 16 + peak - 10, size=(H, W)))
    return h, peak, zs, refs


def test_diff_oracle_forward_equals_c_oracle(orc):
    """The autograd oracle is an independent restatement: its filter states equal the C oracle's, and its
    tau = 1 readout is the posterior mean (the paper's estimator)."""
    from oracle import diff_oracle as dor
    h, peak, zs, refs = _diff_inputs(31)
    nu = NU_ASYM
    T = zs[0].shape[-1]
    out = dor.gradients(h, 0.6, nu, zs, refs, peak, sigma_rw2=2.5, tau=1.0)
    q = orc.params(T, len(h), peak, beta=0.6, sigma_rw2=2.5, nu=nu)
    mu, var = orc.state_init(q, *zs[0].shape[:2])
    for n, z in enumerate(zs):
        e = orc.filter_step(q, h, z, mu, var)
        m2, v2, ds = out["frames"][n]
        np.testing.assert_allclose(m2, e["mu"], rtol=1e-11)
        np.testing.assert_allclose(v2, e["var"], rtol=1e-9)
        np.testing.assert_allclose(ds, m2, rtol=1e-12)
        mu, var = e["mu"], e["var"]


def test_diff_oracle_gradient_matches_finite_differences():
    """Central differences of the loss (float64, steps 1e-6 relative) agree with the autograd gradient for
    every IRF tap, beta and every stencil weight (including weights that are zero)."""
    from oracle import diff_oracle as dor
    h, peak, zs, refs = _diff_inputs(32)
    nu = NU_ASYM
    beta, tau = 0.45, 0.5
    g = dor.gradients(h, beta, nu, zs, refs, peak, sigma_rw2=3.0, tau=tau)
    f = lambda hh, bb, nn: dor.loss_value(hh, bb, nn, zs, refs, peak, sigma_rw2=3.0, tau=tau)
    hd = h.astype(np.float64)
    for j in range(len(h)):
        eps = 1e-6 * max(hd[j], 1e-3)
        hp, hm = hd.copy(), hd.copy()
        hp[j] += eps
        hm[j] -= eps
        fd = (f(hp, beta, nu) - f(hm, beta, nu)) / (2 * eps)
        assert fd == pytest.approx(g["grad_h"][j], rel=1e-5, abs=1e-9 * max(1.0, abs(fd)))
    eps = 1e-7
    fd = (f(hd, beta + eps, nu) - f(hd, beta - eps, nu)) / (2 * eps)
    assert fd == pytest.approx(g["grad_beta"], rel=1e-5)
    for k in range(9):
        up, dn = nu.copy(), nu.copy()
        up[k] += 1e-7
        if nu[k] > 0:   # central difference
            dn[k] -= 1e-7
            fd = (f(hd, beta, up) - f(hd, beta, dn)) / 2e-7
        else:           # a zero weight must stay >= 0: forward difference
            fd = (f(hd, beta, up) - f(hd, beta, nu)) / 1e-7
        assert fd == pytest.approx(g["grad_nu"][k], rel=1e-4, abs=1e-8)


def test_diff_oracle_readout_temperature_limits(orc):
    """The soft readout sum_d d softmax(ell / tau) tends to the maximiser of ell as tau -> 0 and to the mean of the
    candidate grid as tau -> infinity (a temperature that multiplied ell instead would swap the two limits)."""
    import torch
    from oracle import diff_oracle as dor
    h, peak, zs, _ = _diff_inputs(33)
    z = zs[0]
    T, L = z.shape[-1], len(h)
    dmin, dmax = peak, T - L + peak
    q = orc.params(T, L, peak, beta=0.6, sigma_rw2=2.5, nu=NU_ASYM)
    mu0, var0 = orc.state_init(q, *z.shape[:2])
    t = lambda a: torch.as_tensor(a, dtype=torch.float64)
    e = orc.filter_step(q, h, z, mu0, var0, want_ell=True)
    ell = e["ell"].reshape(z.shape[0], z.shape[1], -1)
    srt = np.sort(ell, axis=-1)
    clear = (srt[..., -1] - srt[..., -2]) > 1e-3  # a unique maximiser, by a margin
    assert clear.sum() >= z.shape[0] * z.shape[1] // 2
    _, _, ds_cold = dor.frame(t(h), t(0.6), t(NU_ASYM), t(z), t(mu0), t(var0), peak, dmin, dmax, 2.5, 1e-6)
    np.testing.assert_allclose(ds_cold.numpy()[clear], e["argmax"][clear], atol=1e-9)
    _, _, ds_hot = dor.frame(t(h), t(0.6), t(NU_ASYM), t(z), t(mu0), t(var0), peak, dmin, dmax, 2.5, 1e9)
    np.testing.assert_allclose(ds_hot.numpy(), 0.5 * (dmin + dmax), rtol=1e-6)
