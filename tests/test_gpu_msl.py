"""GPU parity of the multispectral estimate (spl_depth_estimate_msl, Appendix, Eq. div_MSL) against the FP64 oracle.

Tolerances as for the single-band estimate (tests/parity.py): argmax identical except documented near-ties, mu and
var relative 1e-4, and the product M(d) relative 1e-5 with a floor of 1e-6 times its largest value (it is a product
of nbands FP32 ratios, each a sum of at most L products)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close

pytestmark = pytest.mark.gpu
DEV = "cuda"
_DT = {"u16": torch.uint16, "f16": torch.float16, "f32": torch.float32}


def _bands(nb, H, W, T, L, peak, seed, signal=20.0, sbr=0.5, empty_band_pixels=0):
    hb = synth.band_irfs(nb, L, peak)
    rng = np.random.default_rng(seed)
    depth = rng.integers(peak + 4, T - L + peak - 4, size=(H, W))
    z = np.empty((nb, H, W, T))
    for b in range(nb):
        sig = signal * rng.uniform(0.5, 1.5)
        mean = synth.expected_counts(torch.from_numpy(depth), torch.full((H, W), sig, dtype=torch.float64),
                                     sig / (sbr * T), torch.from_numpy(hb[b]), peak, T)
        z[b] = rng.poisson(mean.numpy())
    for k in range(empty_band_pixels):  # pixels whose band k has no photons; the last one has none in any band
        z[k % nb, k // W % H, k % W] = 0.0
    if empty_band_pixels:
        z[:, H - 1, W - 1] = 0.0
    return hb, depth, z


def _gpu(z, fmt):
    nb, H, W, T = z.shape
    pitch = synth.pad_pitch(T) if fmt != "f32" else (T + 3) // 4 * 4
    t = torch.from_numpy(z.reshape(nb * H * W, T).astype(np.float32))
    if fmt == "u16":
        t = t.to(torch.int32).to(torch.uint16)
    else:
        t = t.to(_DT[fmt])
    return synth.pitched(t, pitch).reshape(nb, H * W, pitch).contiguous().to(DEV)


@pytest.mark.parametrize("fmt", ["u16", "f16", "f32"])
@pytest.mark.parametrize("with_prior", [False, True])
def test_msl_matches_oracle(orc, fmt, with_prior):
    nb, H, W, T, L, peak = 4, 9, 13, 320, 24, 8
    hb, depth, z = _bands(nb, H, W, T, L, peak, seed=501, empty_band_pixels=6)
    beta = 0.5
    q = orc.params(T, L, peak, beta=beta)
    prm = spl.make_params(H, W, T, L, peak, beta=beta)
    pm = pv = None
    if with_prior:
        rng = np.random.default_rng(502)
        pm = (depth + rng.normal(0, 6, size=depth.shape)).astype(np.float32)
        pv = rng.uniform(20, 900, size=depth.shape).astype(np.float32)
    e = orc.estimate_msl(q, hb, z, pm, pv, want_ell=True, want_cost=True)
    o = spl.spl_depth_estimate_msl(
        prm, _gpu(z, fmt), torch.from_numpy(hb).to(DEV),
        None if pm is None else torch.from_numpy(pm.reshape(-1)).to(DEV),
        None if pv is None else torch.from_numpy(pv.reshape(-1)).to(DEV), want_cost=True)
    torch.cuda.synchronize()
    check_argmax(o["argmax"].cpu().numpy(), e["argmax"], e["ell"], q.dmin)
    check_close(o["mu"].cpu().numpy(), e["mu"], "mu")
    check_close(o["var"].cpu().numpy(), e["var"], "var", atol=1e-6)
    M = e["M"].reshape(H * W, -1)
    check_close(o["cost"].cpu().numpy(), M, "M", rtol=1e-5, atol=1e-6 * float(M.max()))


def test_msl_one_band_equals_the_single_band_call(orc):
    H, W, T, L, peak = 7, 8, 400, 48, 12
    hb, depth, z = _bands(1, H, W, T, L, peak, seed=503)
    prm = spl.make_params(H, W, T, L, peak, beta=0.35)
    zd = _gpu(z, "u16")
    hd = torch.from_numpy(hb).to(DEV)
    a = spl.spl_depth_estimate_msl(prm, zd, hd)
    s = spl.spl_depth_estimate(prm, zd[0].contiguous(), hd[0].contiguous())
    torch.cuda.synchronize()
    q = orc.params(T, L, peak, beta=0.35)
    e = orc.estimate(q, hb[0], z[0], want_ell=True)
    check_argmax(a["argmax"].cpu().numpy(), e["argmax"], e["ell"], q.dmin)
    check_close(a["mu"].cpu().numpy(), s["mu"].cpu().numpy(), "mu vs single band")
    check_close(a["var"].cpu().numpy(), s["var"].cpu().numpy(), "var vs single band", atol=1e-6)


def test_msl_largest_band_count_and_histogram(orc):
    """SPL_MAX_BANDS bands, L = SPL_MAX_TAPS, T = 2048 (1921 candidates), two pixel rows, against the oracle."""
    nb, H, W, T, L, peak = spl._abi.SPL_MAX_BANDS, 2, 5, 2048, spl._abi.SPL_MAX_TAPS, 30
    hb, depth, z = _bands(nb, H, W, T, L, peak, seed=504, signal=40.0, sbr=0.2)
    q = orc.params(T, L, peak, beta=0.8)
    prm = spl.make_params(H, W, T, L, peak, beta=0.8)
    e = orc.estimate_msl(q, hb, z, want_ell=True)
    o = spl.spl_depth_estimate_msl(prm, _gpu(z, "u16"), torch.from_numpy(hb).to(DEV))
    torch.cuda.synchronize()
    check_argmax(o["argmax"].cpu().numpy(), e["argmax"], e["ell"], q.dmin)
    check_close(o["mu"].cpu().numpy(), e["mu"], "mu")
    check_close(o["var"].cpu().numpy(), e["var"], "var", atol=1e-6)


def test_msl_noiseless_bands_recover_the_depth(orc):
    """Near-noiseless multi-band templates (large integer counts on each band's template, no background): the
    minimum-divergence estimate is the true depth (checked on the oracle too), and the GPU agrees."""
    nb, H, W, T, L, peak = 3, 4, 6, 256, 24, 8
    hb = synth.band_irfs(nb, L, peak)
    rng = np.random.default_rng(505)
    depth = rng.integers(peak, T - L + peak + 1, size=(H, W))
    z = np.zeros((nb, H, W, T))
    for b in range(nb):
        for y in range(H):
            for x in range(W):
                d = depth[y, x]
                z[b, y, x, d - peak:d - peak + L] = np.rint(5000 * hb[b])
    q = orc.params(T, L, peak, beta=0.5)
    e = orc.estimate_msl(q, hb, z, want_ell=True)
    assert np.array_equal(e["argmax"], depth)
    prm = spl.make_params(H, W, T, L, peak, beta=0.5)
    o = spl.spl_depth_estimate_msl(prm, _gpu(z, "f32"), torch.from_numpy(hb).to(DEV))
    torch.cuda.synchronize()
    check_argmax(o["argmax"].cpu().numpy(), e["argmax"], e["ell"], q.dmin)
