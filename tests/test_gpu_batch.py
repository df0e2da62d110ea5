"""GPU parity of the batched photon-list path (spl_batch_*): many sequences of different geometry, IRF and
parameters, photon time-of-arrival lists in CSR form, one persistent launch per frame. The oracle runs the
histogram form on the histograms of the same lists (the photon-list and histogram forms of Eq. beta_div2 are
pinned equal in tests/test_oracle_pins.py)."""
import numpy as np
import pytest
import torch

import paper_2004_09211_gb300 as spl
from paper_2004_09211_gb300 import synth

from parity import check_argmax, check_close, check_intensity

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _seq_specs():
    """(H, W, T, irf, beta, sigma_rw2, nu, signal, bg_photons): uneven sizes, IRFs and parameters."""
    g3 = synth.gaussian_irf(3.0, 12)
    g2 = synth.gaussian_irf(2.0, 8)
    asy = synth.asymmetric_irf(L=48)
    nu_a = np.array([0.05, 0.1, 0.0, 0.15, 0.4, 0.2, 0.0, 0.1, 0.0])
    return [
        (8, 16, 512, g3, 0.5, 3.0, synth.cross_weights(0.5), 3.0, 10.0),
        (16, 8, 300, asy, 0.2, 2.0, synth.cross_weights(0.6), 3.0, 10.0),
        (5, 7, 1024, g2, 1.0, 3.0, nu_a, 4.0, 20.0),
        (12, 12, 700, asy, 0.8, 5.0, synth.cross_weights(0.5), 2.0, 5.0),
        (1, 33, 200, g2, 0.35, 3.0, synth.cross_weights(0.5), 5.0, 3.0),
    ]


def _make_frames(specs, N, seed):
    """Per sequence: params for the oracle/ABI, IRF, and N frames of CSR photon lists (sorted per pixel)."""
    out = []
    for s, (H, W, T, (h, peak), beta, s2, nu, sig, bgp) in enumerate(specs):
        L = len(h)
        sc = synth.moving_scene(H, W, N, peak + 4, T - L + peak - 4, seed + s, n_objects=2)
        frames = []
        for n in range(N):
            off, bins = synth.toa_lists(sc.depth[n], np.full((H, W), sig), bgp / T, h, peak, T, seed * 100 + 10 * s + n)
            frames.append((off, bins))
        out.append(dict(H=H, W=W, T=T, h=h, peak=peak, L=L, beta=beta, s2=s2, nu=np.asarray(nu, np.float64),
                        frames=frames))
    return out


def _alloc_state(H, W, N):
    """One state buffer per frame boundary (frame n reads state n, writes state n+1), so every frame's
    output survives the whole run."""
    P = H * W
    return dict(mu=[torch.empty(P, device=DEV) for _ in range(N + 1)],
                var=[torch.empty(P, device=DEV) for _ in range(N + 1)])


def _run(seqs, N, graph=False, tune=False):
    """Runs N frames through a batch plan (one slot per frame); returns per-frame, per-sequence outputs."""
    prms = [spl.make_params(q["H"], q["W"], q["T"], q["L"], q["peak"], beta=q["beta"], sigma_rw2=q["s2"], nu=q["nu"])
            for q in seqs]
    plan = spl.spl_batch_create(prms, nslots=N)
    try:
        keep = []
        states = [_alloc_state(q["H"], q["W"], N) for q in seqs]
        outs = [[dict() for _ in seqs] for _ in range(N)]
        for n in range(N):
            frames = []
            for i, q in enumerate(seqs):
                st = states[i]
                off, bins = q["frames"][n]
                d = dict(h=torch.from_numpy(q["h"]).to(DEV), offsets=torch.from_numpy(off).to(DEV),
                         bins=torch.from_numpy(bins).to(DEV) if bins.size else torch.zeros(1, dtype=torch.int32,
                                                                                           device=DEV),
                         mu_in=st["mu"][n], var_in=st["var"][n], mu_out=st["mu"][n + 1],
                         var_out=st["var"][n + 1])
                # per-frame output buffers so every frame can be checked after the run
                P = q["H"] * q["W"]
                for k, dt in (("argmax", torch.int32), ("refl", torch.float32), ("bg", torch.float32)):
                    d[k] = torch.empty(P, dtype=dt, device=DEV)
                keep.append(d)
                frames.append(d)
                outs[n][i] = d
            spl.spl_batch_set(plan, n, frames)
        for i, q in enumerate(seqs):
            spl.spl_state_init(prms[i], states[i]["mu"][0], states[i]["var"][0])
        if tune:
            spl.spl_batch_tune(plan, 0)
            for i, q in enumerate(seqs):  # tuning wrote frame 0's outputs; restart from the initial state
                spl.spl_state_init(prms[i], states[i]["mu"][0], states[i]["var"][0])
        results = []
        if graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                spl.spl_batch_step(plan, 0, stream=s)  # warm-up outside capture
            torch.cuda.current_stream().wait_stream(s)
            torch.cuda.synchronize()
            for i, q in enumerate(seqs):
                spl.spl_state_init(prms[i], states[i]["mu"][0], states[i]["var"][0])
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                for n in range(N):
                    spl.spl_batch_step(plan, n)
            g.replay()
            torch.cuda.synchronize()
        else:
            for n in range(N):
                spl.spl_batch_step(plan, n)
            torch.cuda.synchronize()
        for n in range(N):
            fr = []
            for i in range(len(seqs)):
                d = outs[n][i]
                fr.append({k: d[k].cpu().numpy().copy() for k in ("mu_out", "var_out", "argmax", "refl", "bg")})
            results.append(fr)
        flags = spl.spl_batch_status(plan)
        info = spl.spl_batch_info(plan)
        return results, flags, info
    finally:
        spl.spl_batch_destroy(plan)


def test_batch_matches_oracle(orc):
    seqs = _make_frames(_seq_specs(), N=3, seed=7)
    res, flags, info = _run(seqs, 3)
    assert flags == 0
    assert info["units"] > 0
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


def test_batch_size_classes(orc):
    """Sequences whose candidate grids differ by more than a factor of two (T = 4096 against T = 512 and 1000):
    the plan splits them into two size classes with a launch each; the classes partition the work units, the
    second holds only grids of at most half the longest, and both match the oracle, eagerly and replayed from a
    CUDA graph (bit for bit)."""
    asy = synth.asymmetric_irf(L=48)
    specs = [(4, 8, 4096, asy, 0.4, 3.0, synth.cross_weights(0.5), 3.0, 10.0),
             (6, 6, 512, synth.gaussian_irf(3.0, 12), 0.7, 3.0, synth.cross_weights(0.5), 3.0, 10.0),
             (1, 20, 1000, synth.gaussian_irf(2.0, 8), 0.2, 3.0, synth.cross_weights(0.6), 4.0, 5.0)]
    seqs = _make_frames(specs, N=2, seed=12)
    res, flags, info = _run(seqs, 2)
    graph, _, _ = _run(seqs, 2, graph=True)
    assert flags == 0
    cls = info["classes"]
    assert len(cls) == 2, info
    grids = [q["T"] - q["L"] + 1 for q in seqs]
    assert cls[0]["max_candidates"] >= max(grids) and 2 * cls[1]["max_candidates"] <= cls[0]["max_candidates"]
    assert cls[0]["units"] > 0 and cls[1]["units"] > 0 and cls[0]["units"] + cls[1]["units"] == info["units"]
    assert cls[1]["ctas"] * cls[1]["warps_per_cta"] > cls[0]["ctas"] * cls[0]["warps_per_cta"]
    for i, q in enumerate(seqs):
        oq = orc.params(q["T"], q["L"], q["peak"], beta=q["beta"], sigma_rw2=q["s2"], nu=q["nu"])
        mu, var = orc.state_init(oq, q["H"], q["W"])
        for n in range(2):
            off, bins = q["frames"][n]
            z = synth.csr_to_histograms(off, bins, q["T"]).astype(np.float64).reshape(q["H"], q["W"], q["T"])
            e = orc.filter_step(oq, q["h"], z, mu, var, want_ell=True)
            g = res[n][i]
            check_argmax(g["argmax"], e["argmax"], e["ell"], oq.dmin, f"seq {i} frame {n} argmax")
            check_close(g["mu_out"], e["mu"], f"seq {i} frame {n} mu")
            check_close(g["var_out"], e["var"], f"seq {i} frame {n} var", atol=1e-6)
            check_intensity(orc, oq, q["h"], z, g["mu_out"], e["mu"], g["refl"], g["bg"])
            for k in ("mu_out", "var_out", "argmax", "refl", "bg"):
                np.testing.assert_array_equal(graph[n][i][k], g[k])
            mu, var = e["mu"], e["var"]


def test_batch_graph_replay_and_tuning_reproduce_eager():
    seqs = _make_frames(_seq_specs(), N=3, seed=8)
    eager, _, _ = _run(seqs, 3)
    graph, flags, _ = _run(seqs, 3, graph=True)
    tuned, _, info = _run(seqs, 3, tune=True)
    assert flags == 0
    assert info["tile"] in (8, 16, 32, 64, 128)
    for n in range(3):
        for i in range(len(seqs)):
            for k in ("mu_out", "var_out", "argmax", "refl", "bg"):
                np.testing.assert_array_equal(graph[n][i][k], eager[n][i][k])
                np.testing.assert_array_equal(tuned[n][i][k], eager[n][i][k])


def test_batch_equals_histogram_kernel():
    """The photon-list kernel and the FP32 histogram kernel agree on the same data (different summation order)."""
    seqs = _make_frames(_seq_specs()[:3], N=2, seed=9)
    res, _, _ = _run(seqs, 2)
    for i, q in enumerate(seqs):
        prm = spl.make_params(q["H"], q["W"], q["T"], q["L"], q["peak"], beta=q["beta"], sigma_rw2=q["s2"], nu=q["nu"])
        mu, var = spl.spl_state_init(prm)
        hd = torch.from_numpy(q["h"]).to(DEV)
        for n in range(2):
            off, bins = q["frames"][n]
            z = synth.csr_to_histograms(off, bins, q["T"])
            zt = synth.pitched(torch.from_numpy(z.astype(np.int32)).to(torch.uint16), synth.pad_pitch(q["T"])).to(DEV)
            o = spl.spl_filter_step_fp32(prm, zt, hd, mu, var)
            torch.cuda.synchronize()
            check_close(o["mu"].cpu().numpy(), res[n][i]["mu_out"], f"seq {i} frame {n} mu", rtol=1e-5)
            check_close(o["var"].cpu().numpy(), res[n][i]["var_out"], f"seq {i} frame {n} var", rtol=1e-4,
                        atol=1e-6)
            mu, var = o["mu"], o["var"]


def test_batch_reports_out_of_range_bins():
    """A photon bin outside [0, T) is dropped and reported through spl_batch_status; no fault."""
    seqs = _make_frames(_seq_specs()[:1], N=1, seed=10)
    clean, flags0, _ = _run(seqs, 1)
    assert flags0 == 0
    off, bins = seqs[0]["frames"][0]
    P = len(off) - 1
    # append one bad photon (bin T) to pixel 3
    nb = np.insert(bins, off[4], seqs[0]["T"])
    noff = off.copy()
    noff[4:] += 1
    seqs[0]["frames"][0] = (noff, nb.astype(np.int32))
    dirty, flags, _ = _run(seqs, 1)
    assert flags & spl.SPL_BATCH_BAD_BIN
    for k in ("mu_out", "var_out", "argmax"):
        np.testing.assert_array_equal(dirty[0][0][k], clean[0][0][k])
