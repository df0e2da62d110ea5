"""Host logic of bench.py that needs no GPU: the HBM roofline arithmetic and the rule that a captured traffic or
instruction figure is reported only while the kernel's sources hash to the captured version."""
import os
import shutil

import pytest

import bench


def test_hbm_roofline_arithmetic():
    r = bench.hbm_roofline({"hbm_gbs": 6000.0}, 3.0e9, 1.0e-3, 2.5e9, "k", note="x")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert r["achieved"] == pytest.approx(3000.0)
    assert r["frac"] == pytest.approx(0.5)
    assert r["traffic"] == 2.5e9 and r["avg_launch_ms"] == pytest.approx(1.0) and r["note"] == "x"
    assert r["peak_source"].startswith("MEASURED_PEAKS")
    fb = bench.hbm_roofline({}, 6.8e9, 1.0, None, "k")
    assert fb["peak"] == 6800.0 and fb["frac"] == pytest.approx(0.001) and fb["peak_source"].startswith("fallback")


def test_every_capture_names_existing_sources():
    csrc = os.path.join(bench.ROOT, "paper_2004_09211_gb300", "csrc")
    for name, cap in bench.TRAFFIC_CAPTURES.items():
        assert cap["sources"], name
        for f in cap["sources"]:
            assert os.path.isfile(os.path.join(csrc, f)), (name, f)
        assert len(cap["sha256"]) == 64 and cap["bytes_per_pixel"] > 0 and cap["inst_per_pixel"] > 0


def test_changed_source_voids_the_capture(tmp_path, monkeypatch):
    """A capture scales with the pixels while its sources are unchanged and reads None once any of them changes."""
    src = os.path.join(bench.ROOT, "paper_2004_09211_gb300", "csrc")
    dst = tmp_path / "paper_2004_09211_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    live = [k for k in bench.TRAFFIC_CAPTURES if bench.capture_traffic(k, 1) is not None]
    if not live:
        pytest.skip("no capture matches the current sources")
    name = live[0]
    cap = bench.TRAFFIC_CAPTURES[name]
    assert bench.capture_traffic(name, 1000) == pytest.approx(1000 * cap["bytes_per_pixel"])
    assert bench.capture_traffic(name, 1000, "inst_per_pixel") == pytest.approx(1000 * cap["inst_per_pixel"])
    with open(dst / cap["sources"][-1], "a") as fh:
        fh.write("\n// edited\n")
    assert bench.capture_traffic(name, 1000) is None
    assert bench.capture_traffic(name, 1000, "inst_per_pixel") is None


def test_photon_lists_of_a_frame_give_back_its_histograms(orc):
    """The end-to-end leg moves each frame as photon lists built from its histograms (each bin repeated by its
    count): the oracle's histogram of those lists is the frame again, pixel by pixel, including empty pixels."""
    import numpy as np
    import torch
    rng = np.random.default_rng(4)
    P, T, pitch = 37, 61, 64
    z = rng.poisson(0.4, size=(P, T))
    z[[0, 9, 36]] = 0
    z[5, 7] = 300
    zt = torch.zeros((P, pitch), dtype=torch.int32)
    zt[:, :T] = torch.from_numpy(z)
    off, bins = bench.toa_from_histograms(zt.to(torch.uint16), T)
    assert off.dtype == torch.int32 and bins.dtype == torch.uint16 and int(off[-1]) == z.sum()
    got, flags = orc.toa_histogram(T, off.numpy(), bins.to(torch.int32).numpy())
    assert flags == 0
    np.testing.assert_array_equal(got, z)
