"""The uint16 route of the filter step: the data term on the tensor cores with the counts converted to FP16 on
chip (exact below 1024); 128-pixel blocks that hold a larger count, and pixels whose data term exceeds the tensor
cores' accuracy bound, computed again by the FP32 kernel. spl_filter_step_tc takes it at any frame size;
spl_filter_step, spl_filter_step_detect and spl_depth_estimate from one 128-pixel block per SM upward.

Checks: without such counts the uint16 route equals spl_filter_step_tc on FP16 copies of the same frames bit for
bit (the conversion is exact and the kernel the same); a block holding a count of 1024 or more, and a pixel past
the accuracy bound, equal spl_filter_step_fp32 bit for bit (the FP32 kernel computed them), every other block
stays on the tensor cores; a block whose largest count is 1023 stays on the tensor cores and still matches the
oracle; spl_filter_step picks the tensor cores for a large frame and the FP32 kernel for a small one; everything
matches the FP64 oracle at the filter's tolerances (tests/parity.py), including a ragged last block."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close, check_intensity
from test_gpu_parity import DEV, _gpu_hist, _np, video_inputs

pytestmark = pytest.mark.gpu

KEYS = ("mu", "var", "argmax", "refl", "bg")


def _status_clear():
    assert spl.spl_tc_status() == 0, "a bounded wait of the tensor-core kernel ran out"


def _steps(prm, h, zs, T, step, dtype=torch.uint16):
    """The chain of `step` over the frames; returns the outputs of every frame (host copies)."""
    hd = torch.from_numpy(h).to(DEV)
    mu, var = spl.spl_state_init(prm)
    out = []
    for z in zs:
        o = step(prm, _gpu_hist(z, T, dtype), hd, mu, var)
        torch.cuda.synchronize()
        out.append({k: _np(o[k]).copy() for k in KEYS})
        mu, var = o["mu"], o["var"]
    return out


def test_route_equals_the_fp16_kernel_bit_for_bit():
    H, W, N, T = 24, 28, 4, 700
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.02, seed=71)
    assert max(float(z.max()) for z in zs) < 1024
    prm = spl.make_params(H, W, T, len(h), peak, beta=0.4, sigma_rw2=3.0)
    a = _steps(prm, h, zs, T, spl.spl_filter_step_tc)
    b = _steps(prm, h, zs, T, spl.spl_filter_step_tc, torch.float16)
    for n in range(N):
        for k in KEYS:
            assert np.array_equal(a[n][k], b[n][k]), f"frame {n}: {k} differs from the FP16 kernel"
    _status_clear()


def _with_large_counts(zs, H, W, T, cells):
    """Copies of the frames with count c put into bin t of pixel p for each (frame, p, t, c) in cells."""
    out = [z.copy().reshape(H * W, T) for z in zs]
    for n, p, t, c in cells:
        out[n][p, t] = c
    return [z.reshape(H, W, T) for z in out]


def test_blocks_with_large_counts_are_redone_in_fp32(orc):
    """600 pixels (blocks of 128, the last one ragged with 88): frame 1 puts 1025 photons in one bin of a pixel of
    block 1 and 5001 in one of block 4 (the ragged one); frame 2 puts 1023 in block 2 (it stays on the tensor
    cores) and 3001 in block 0. Each frame runs the route and spl_filter_step_fp32 from the same state (the route's
    previous output): redone blocks equal the FP32 kernel bit for bit, the others agree within the tolerances, and
    the route matches the oracle run from that state."""
    H, W, N, T = 20, 30, 3, 400
    P = H * W
    h, peak, sc, zs = video_inputs(H, W, N, T, 0.1, seed=72)
    cells = [(1, 128 + 17, 200, 1025), (1, 4 * 128 + 40, 150, 5001), (2, 2 * 128 + 5, 90, 1023),
             (2, 60, 300, 3001)]
    zs = _with_large_counts(zs, H, W, T, cells)
    beta = 0.5
    prm = spl.make_params(H, W, T, len(h), peak, beta=beta, sigma_rw2=3.0)
    q = orc.params(T, len(h), peak, beta=beta, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    hd = torch.from_numpy(h).to(DEV)
    redone = {1: {1, 4}, 2: {0}}
    mu, var = spl.spl_state_init(prm)
    for n in range(N):
        zt = _gpu_hist(zs[n], T)
        a = spl.spl_filter_step_tc(prm, zt, hd, mu, var)
        f = spl.spl_filter_step_fp32(prm, zt, hd, mu, var)
        e = orc.filter_step(q, h, zs[n], _np(mu).reshape(H, W).astype(np.float64),
                            _np(var).reshape(H, W).astype(np.float64), want_ell=True)
        torch.cuda.synchronize()
        ga = {k: _np(a[k]) for k in KEYS}
        gf = {k: _np(f[k]) for k in KEYS}
        for blk in range((P + 127) // 128):
            sl = slice(128 * blk, min(P, 128 * blk + 128))
            if blk in redone.get(n, set()):
                for k in KEYS:
                    assert np.array_equal(ga[k][sl], gf[k][sl]), f"frame {n} block {blk}: {k} is not the FP32 result"
        check_close(ga["mu"], gf["mu"], f"mu frame {n} route vs FP32 kernel")
        check_close(ga["var"], gf["var"], f"var frame {n} route vs FP32 kernel", atol=1e-6)
        check_argmax(ga["argmax"], e["argmax"], e["ell"], q.dmin, f"argmax frame {n}")
        check_close(ga["mu"], e["mu"], f"mu frame {n}")
        check_close(ga["var"], e["var"], f"var frame {n}", atol=1e-6)
        check_intensity(orc, q, h, zs[n], ga["mu"], e["mu"], ga["refl"], ga["bg"])
        mu, var = a["mu"], a["var"]
    _status_clear()


def test_route_on_a_single_pixel_and_long_histograms(orc):
    """One pixel (one ragged block of 1) and T = SPL_MAX_BINS with a 128-tap IRF, a count of 2000 in frame 0."""
    T = spl._abi.SPL_MAX_BINS
    hh, peak = synth.asymmetric_irf(L=spl._abi.SPL_MAX_TAPS)
    rng = np.random.default_rng(73)
    zs = [rng.poisson(0.02, size=(1, 1, T)).astype(np.float64) for _ in range(2)]
    zs[0][0, 0, 3000] = 2000
    zs[1][0, 0, 5000:5048] += 30
    prm = spl.make_params(1, 1, T, len(hh), peak, beta=0.7, sigma_rw2=3.0)
    q = orc.params(T, len(hh), peak, beta=0.7, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    a = _steps(prm, hh, zs, T, spl.spl_filter_step_tc)
    mu_o, var_o = orc.state_init(q, 1, 1)
    for n in range(2):  # each frame from the route's own previous state
        e = orc.filter_step(q, hh, zs[n], mu_o, var_o, want_ell=True)
        check_argmax(a[n]["argmax"], e["argmax"], e["ell"], q.dmin)
        check_close(a[n]["mu"], e["mu"], "mu")
        check_close(a[n]["var"], e["var"], "var", atol=1e-6)
        mu_o, var_o = a[n]["mu"].reshape(1, 1).astype(np.float64), a[n]["var"].reshape(1, 1).astype(np.float64)
    _status_clear()


def test_bright_pixels_leave_the_tensor_cores(orc):
    """1000 photons in each of 79 consecutive bins at beta = 0.1: the data term lambda log2(e) C is about 8.7e5 bits,
    far past the 1024 the tensor cores keep, so these pixels go to the FP32 kernel and equal it bit for bit (a
    plateau of exactly equal C, which the FP32 kernel's identical operand order reproduces); the photon-starved
    pixels beside them agree with the FP32 kernel within the tolerances. Everything matches the oracle."""
    hh, peak = synth.asymmetric_irf(L=48)
    H, W, T = 4, 8, 600
    rng = np.random.default_rng(74)
    z = rng.poisson(0.01, size=(H, W, T)).astype(np.float64)
    bright = [(0, 1, 100), (1, 3, 250), (2, 6, 400), (3, 2, 130)]
    for y, x, s0 in bright:
        z[y, x, s0:s0 + 79] = 1000.0
    beta = 0.1
    prm = spl.make_params(H, W, T, len(hh), peak, beta=beta, sigma_rw2=3.0)
    q = orc.params(T, len(hh), peak, beta=beta, sigma_rw2=3.0, nu=synth.cross_weights(0.5))
    hd = torch.from_numpy(hh).to(DEV)
    mu, var = spl.spl_state_init(prm)
    zt = _gpu_hist(z, T)
    a = spl.spl_filter_step_tc(prm, zt, hd, mu, var)
    f = spl.spl_filter_step_fp32(prm, zt, hd, mu, var)
    torch.cuda.synchronize()
    ga = {k: _np(a[k]) for k in KEYS}
    gf = {k: _np(f[k]) for k in KEYS}
    for y, x, _ in bright:
        p = y * W + x
        for k in KEYS:
            assert ga[k][p] == gf[k][p], f"pixel {p}: {k} is not the FP32 result"
    check_close(ga["mu"], gf["mu"], "mu route vs FP32 kernel")
    check_close(ga["var"], gf["var"], "var route vs FP32 kernel", atol=1e-6)
    m0, v0 = orc.state_init(q, H, W)
    e = orc.filter_step(q, hh, z, m0, v0, want_ell=True)
    check_argmax(ga["argmax"], e["argmax"], e["ell"], q.dmin)
    check_close(ga["mu"], e["mu"], "mu")
    check_close(ga["var"], e["var"], "var", atol=1e-6)
    _status_clear()


def test_automatic_choice_by_frame_size():
    """spl_filter_step on uint16 frames: from one 128-pixel block per SM upward it is the tensor-core route (equal
    to spl_filter_step_tc bit for bit), below it the FP32 kernel (equal to spl_filter_step_fp32 bit for bit)."""
    hh, peak = synth.asymmetric_irf(L=24)
    T = 160
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for H, W, entry in ((nsm, 128, spl.spl_filter_step_tc), (8, 16, spl.spl_filter_step_fp32)):
        h, peak_, sc, zs = video_inputs(H, W, 2, T, 0.5, seed=75, L=24)
        prm = spl.make_params(H, W, T, len(h), peak_, beta=0.5, sigma_rw2=3.0)
        a = _steps(prm, h, zs, T, spl.spl_filter_step)
        b = _steps(prm, h, zs, T, entry)
        for n in range(2):
            for k in KEYS:
                assert np.array_equal(a[n][k], b[n][k]), f"{H}x{W} frame {n}: {k} differs from {entry.__name__}"
    _status_clear()
