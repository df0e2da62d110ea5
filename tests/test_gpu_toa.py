"""Histograms built on the device from photon time-of-arrival lists (spl_toa_histogram): integer work, so every
element is compared bit for bit with the oracle's histogram of the same lists (oracle.toa_histogram).

Checks: ragged lists (empty pixels, up to a few hundred photons, repeated bins) at frame sizes that leave a partial
CTA, T not a multiple of 8 with a wider pitch, the largest T; every element of every row written (the output starts
as 0xFFFF); the device flags for dropped bins, invalid offsets and saturated counts; an empty frame; and the
histograms of one frame fed to spl_filter_step give the same outputs, bit for bit, as the host-built histograms of
the same photons (on the tensor-core route of a 160 x 128 frame)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from test_gpu_parity import DEV, _gpu_hist

pytestmark = pytest.mark.gpu


def _lists(P, T, seed, max_count=300):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, max_count + 1, size=P)
    counts[rng.random(P) < 0.2] = 0
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    bins = rng.integers(0, T, size=int(off[-1]))
    hot = rng.integers(0, T, size=bins.size // 4)   # repeated bins
    bins[: hot.size] = hot
    return off, bins.astype(np.uint16)


def _run(prm, off, bins, pitch):
    P = prm.H * prm.W
    out = torch.full((P, pitch), 0xFFFF, dtype=torch.int32).to(torch.uint16).to(DEV)
    bd = torch.from_numpy(bins.astype(np.int32)).to(torch.uint16).to(DEV) if bins.size else \
        torch.empty(0, dtype=torch.uint16, device=DEV)
    spl.spl_toa_histogram(prm, torch.from_numpy(off).to(DEV), bd, out=out)
    torch.cuda.synchronize()
    return out.cpu().to(torch.int32).numpy(), spl.spl_toa_status()


@pytest.mark.parametrize("H,W,T,pitch", [(5, 7, 1500, 1504), (9, 13, 61, 104), (3, 3, 8192, 8192),
                                         (1, 1, 1, 8), (33, 31, 4096, 4096)])
def test_histograms_match_the_oracle(orc, H, W, T, pitch):
    assert spl.spl_toa_status() == 0
    off, bins = _lists(H * W, T, seed=H * 1000 + T)
    prm = spl.make_params(H, W, T, 1, 0)
    got, flags = _run(prm, off, bins, pitch)
    z, oflags = orc.toa_histogram(T, off, bins)
    assert oflags == 0 and flags == 0
    np.testing.assert_array_equal(got[:, :T], z)
    assert not got[:, T:].any(), "elements T..pitch-1 must be written as 0"


def test_empty_frame():
    prm = spl.make_params(4, 5, 300, 1, 0)
    got, flags = _run(prm, np.zeros(21, np.int32), np.zeros(0, np.uint16), 304)
    assert flags == 0 and not got.any()


def test_device_flags(orc):
    T = 40
    prm = spl.make_params(2, 2, T, 1, 0)
    # a bin past T is dropped (flag 1); the other photons stay
    off = np.array([0, 3, 3, 5, 6], np.int32)
    bins = np.array([1, 45, 1, 0, 39, 7], np.uint16)
    got, flags = _run(prm, off, bins, 40)
    z, oflags = orc.toa_histogram(T, off, bins)
    assert flags == spl._abi.SPL_TOA_BAD_BIN == oflags
    np.testing.assert_array_equal(got[:, :T], z)
    # decreasing offsets and offsets past nphotons: those rows are zero (flag 4)
    off = np.array([0, 3, 2, 5, 99], np.int32)
    got, flags = _run(prm, off, np.array([1, 2, 3, 4, 5], np.uint16), 40)
    z, oflags = orc.toa_histogram(T, off, [1, 2, 3, 4, 5])
    assert flags == spl._abi.SPL_TOA_BAD_OFFSETS == oflags
    np.testing.assert_array_equal(got[:, :T], z)
    assert not got[1].any() and not got[3].any()
    assert spl.spl_toa_status() == 0, "the status is cleared when read"
    # 70000 photons in one bin: written as 65535 (flag 2), the rest of the row exact
    off = np.array([0, 70003, 70003, 70003, 70003], np.int32)
    bins = np.concatenate([np.full(70000, 5), [6, 6, 7]]).astype(np.uint16)
    got, flags = _run(prm, off, bins, 40)
    z, _ = orc.toa_histogram(T, off, bins)
    assert flags == spl._abi.SPL_TOA_SATURATED
    np.testing.assert_array_equal(got[:, :T], np.minimum(z, 65535))


def test_filter_step_on_device_histograms():
    """The same photons as device-built and as host-built histograms through spl_filter_step: identical outputs."""
    H, W, T, L = 160, 128, 1500, 48
    h, peak = synth.asymmetric_irf(L=L)
    depth = synth.smooth_depth_map(H, W, peak + 30, T - L + peak - 30, 7).round()
    off, bins = synth.toa_lists(depth, np.full((H, W), 3.0), 30.0 / T, h, peak, T, seed=8, max_photons=60)
    prm = spl.make_params(H, W, T, L, peak, beta=0.5, sigma_rw2=3.0)
    hd = torch.from_numpy(h).to(DEV)
    zdev = spl.spl_toa_histogram(prm, torch.from_numpy(off).to(DEV),
                                 torch.from_numpy(bins).to(torch.uint16).to(DEV))
    zhost = _gpu_hist(synth.csr_to_histograms(off, bins, T), T)
    torch.cuda.synchronize()
    assert spl.spl_toa_status() == 0
    assert zdev.shape == zhost.shape
    assert torch.equal(zdev.cpu().to(torch.int32), zhost.cpu().to(torch.int32))
    mu, var = spl.spl_state_init(prm)
    a = spl.spl_filter_step(prm, zdev, hd, mu, var)
    b = spl.spl_filter_step(prm, zhost, hd, mu, var)
    torch.cuda.synchronize()
    assert spl.spl_tc_status() == 0
    for k in ("mu", "var", "argmax", "refl", "bg"):
        assert torch.equal(a[k], b[k]), k


def test_full_size_frame_matches_the_oracle(orc):
    """The video workload's frame size and densest lists (256 x 256 pixels, T = 1500, SBR 0.01: about 300 photons
    per pixel, 20 M in the frame), each pixel's photons in random order, in the launch configuration of the
    benchmark's end-to-end leg: every element equal to the oracle's histogram."""
    H, W, T, L = 256, 256, 1500, 48
    h, peak = synth.asymmetric_irf(L=L)
    depth = synth.smooth_depth_map(H, W, peak + 30, T - L + peak - 30, 11).round()
    g = torch.Generator().manual_seed(11)
    mean = synth.expected_counts(torch.from_numpy(depth), torch.full((H, W), 3.0, dtype=torch.float64),
                                 3.0 / (0.01 * T), torch.from_numpy(h), peak, T)
    z = torch.poisson(mean, generator=g).to(torch.int64).reshape(H * W, T)
    cnt = z.sum(1)
    off = np.concatenate([[0], np.cumsum(cnt.numpy())]).astype(np.int32)
    nz = z.nonzero()
    reps = z[nz[:, 0], nz[:, 1]]
    bins = torch.repeat_interleave(nz[:, 1], reps)
    pix = torch.repeat_interleave(nz[:, 0], reps).to(torch.float64)
    key = pix + torch.rand(pix.numel(), generator=torch.Generator().manual_seed(12), dtype=torch.float64)
    bins = bins[torch.argsort(key)].numpy().astype(np.uint16)  # each pixel's photons in random order
    assert bins.size > 15_000_000
    prm = spl.make_params(H, W, T, L, peak)
    got, flags = _run(prm, off, bins, synth.pad_pitch(T))
    zo, oflags = orc.toa_histogram(T, off, bins)
    assert flags == 0 and oflags == 0
    np.testing.assert_array_equal(got[:, :T], zo)
    np.testing.assert_array_equal(zo, z.numpy())
    assert not got[:, T:].any()
