#!/usr/bin/env python3
"""Benchmark of the online robust depth-reconstruction hot path (one GPU per process).

Workload (the video configuration): 256 x 256 pixels x 50 frames, T = 1500 bins, asymmetric 48-tap IRF
(gamma rise + exponential tail), scene = tilted background plane + 3 moving rectangles/ellipses (1-3 px and
5-20 bins per frame), 1-5 signal photons per pixel-frame, background per sequence for SBR 0.01, 0.1 and 1,
each sequence filtered with beta = 0.2, 0.5 and 1.0 (9 runs), uint16 histograms. One step = the whole job:
9 runs x 50 frames of spl_filter_step (prior from the previous frame, pseudo-posterior, moments,
background/reflectivity) = 29.5 M pixel-frames. Histograms are generated on the device before timing and
stay resident (29.6 GB; every frame is 197 MB, larger than the 129 MB L2, so no flush is needed between
iterations). spl_filter_step takes uint16 frames through the tensor cores (counts converted to FP16 on chip,
exact below 1024); the same job is also timed through spl_filter_step_fp32, the FP32 CUDA-core kernel.

Prints ONE JSON line (rank 0). `--impl reference` times the FP64 CPU oracle instead, on a bounded sample of
the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 256
N_FRAMES = 50
T = 1500
L = 48
SBRS = (0.01, 0.1, 1.0)
BETAS = (0.2, 0.5, 1.0)
SIGMA_RW2 = 3.0
JOB_STREAMS = 3  # streams the video job's independent runs are issued on
E2E_JOBS = 3     # end-to-end legs: whole jobs timed one after another (after one untimed job)
SEED = 2
WORKLOAD = "video 256x256x50 frames, T=1500, 48-tap asymmetric IRF, SBR {0.01,0.1,1} x beta {0.2,0.5,1}"


# DRAM bytes (read + write) and warp-instructions per launch of each workload's dominant kernel (for the filter
# steps: the depth launch plus the intensity launch after it), from ncu captures, scaled by the pixels processed,
# valid only for the exact kernel sources they were taken on: the bench reports null for "traffic" and "issue"
# when the sources' hash differs. Each list names every file of this package the kernel's translation unit
# compiles; the pseudo-posterior code lives in posterior.cuh, apart from the helpers in pixel.cuh, so that a change
# to it voids exactly the captures of the kernels that call it (the depth and photon-list kernels).
TRAFFIC_CAPTURES = {
    # one FP32 filter step of the video job (spl_filter_step_fp32): the depth launch of frame 1 of each of the nine
    # runs (nine captures of one launch each, mean) plus the intensity launch (mean of the same nine frames)
    # (ncu dram__bytes_read.sum + dram__bytes_write.sum and smsp__inst_executed.sum)
    "k_estimate": {"sources": ("estimate.cu", "pixel.cuh", "posterior.cuh", "intensity.cu"),
                   "sha256": "7c03e2392cea9239812429c9c1a41bc18e297fd094372fd196d619374661e66b",
                   "bytes_per_pixel": (201.11e6 + 15.52e6) / 65536,
                   "inst_per_pixel": (368.24e6 + 14.85e6) / 65536},
    # one uint16 filter step of the video job (spl_filter_step): the tensor-core launch, the redo launch and the
    # intensity launch of frame 1 of each of the nine runs (mean)
    "k_filter_tc_u16": {"sources": ("tcfilter.cu", "tc_common.cuh", "intensity.cu", "pixel.cuh", "estimate.cu",
                                    "posterior.cuh", "f32x2.cuh"),
                        "sha256": "0dcc41b054efb2b34239dff8e6cce5d9544c9e2306946b8dc718ba7323729a73",
                        "bytes_per_pixel": (218.70e6 + 3.05e6) / 65536,
                        "inst_per_pixel": 130.80e6 / 65536},
    "k_filter_tc": {"sources": ("tcfilter.cu", "tc_common.cuh", "intensity.cu", "pixel.cuh", "f32x2.cuh"),
                    "sha256": "3a0457eb824d56aecb181436c24d0cec9f94162f04733fdb7316bca9e72ce35e",
                    "bytes_per_pixel": (537.628e6 + 3.699e6 + 17.200e6) / 65536,
                    # warp-instructions of one filter step (tensor-core launch + intensity launch), one capture
                    # of frame 2 of a 256 x 256 run of the mixed workload
                    "inst_per_pixel": (290.46e6 + 14.004e6) / 65536},
    # the two launches (one per size class) of one frame of the photon-list kernel over all 64 sequences of the
    # batched workload (7 050 240 pixels)
    "k_batch": {"sources": ("batch.cu", "pixel.cuh", "posterior.cuh", "photons.cuh"),
                "sha256": "fd666076f64fd9d003440086d9d408245c1461c127b5b3ae82f67e04b7bacf7f",
                "bytes_per_pixel": (160.68e6 + 32.66e6 + 295.12e6 + 71.50e6) / 7050240,
                "inst_per_pixel": (17607.38e6 + 16141.73e6) / 7050240},
    # backward launches of the differentiable filter (128 x 128 frames, T = 1024): mean of three of the 20 launches
    # of one reverse sweep (they differ by 0.04 %)
    "k_diff_backward": {"sources": ("grad.cu", "pixel.cuh"),
                        "sha256": "64352bebe7a4e6a4bbe5d67e3ed6cad8e1956beba898ab517d765fe1f099a408",
                        "bytes_per_pixel": (34.11e6 + 0.0) / 16384,
                        "inst_per_pixel": 260.18e6 / 16384},
}


def capture_traffic(kernel: str, pixels: int, key: str = "bytes_per_pixel"):
    """Traffic (or, key="inst_per_pixel", warp-instructions) per launch of `kernel` over `pixels` pixels from its
    capture, or None if it has none or the sources changed since."""
    import hashlib
    cap = TRAFFIC_CAPTURES.get(kernel)
    if cap is None:
        return None
    h = hashlib.sha256()
    for f in cap["sources"]:
        with open(os.path.join(ROOT, "paper_2004_09211_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return cap[key] * pixels if h.hexdigest() == cap["sha256"] and key in cap else None


def hbm_roofline(peaks, alg_bytes, launch_s, traffic, kernel, **extra):
    """The HBM roof of a launch: `alg_bytes` algorithmic bytes over `launch_s` seconds against the measured copy
    bandwidth; `traffic` is the captured DRAM bytes per launch or None."""
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / launch_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": traffic, "kernel": kernel, "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": launch_s * 1e3,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s", **extra}


# Measured on GB300 (bench.py --workload alu_peaks, with spl_probe_throughput): FP32 FMA instructions issue at
# 124.5 lanes per clock per SM (3.89 warp-instructions per clock per SM, one per scheduler), packed f32x2 FMAs at
# 127.0 operations (no gain: the FMA pipe takes two cycles per packed instruction) and ex2.approx at 31.9.
MEASURED_WARP_ISSUE_PER_CLK_SM = 124.5 / 32


def issue_roofline(dev, peaks, inst, launch_s, source):
    """The instruction-issue roof of a launch: `inst` warp-instructions (from its capture) over `launch_s` seconds
    against the measured FFMA issue rate (3.89 warp-instructions per clock per SM) at the maximum SM clock; None
    without a valid capture."""
    if inst is None:
        return None
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = MEASURED_WARP_ISSUE_PER_CLK_SM * nsm * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    return {"achieved": inst / launch_s, "peak": peak, "unit": "warp-instructions/s",
            "frac": inst / launch_s / peak, "inst_per_launch": inst, "source": source,
            "peak_source": "measured FFMA issue rate (bench.py --workload alu_peaks) x SMs x max SM clock"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--frames", type=int, default=N_FRAMES, help="frames per sequence (default 50)")
    ap.add_argument("--side", type=int, default=None,
                    help="mixed workload only: image side (default 1024; smaller sides for profiling captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="video", choices=["video", "batched", "diff", "mixed", "video_tc", "detect",
                                                              "pd_curves", "fine", "alu_peaks", "msl", "single"],
                    help="video (default, the headline line); batched: 64 photon-list sequences in one launch per "
                         "frame; diff: differentiable filter forward + backward; mixed: 1024x1024 FP16 frames "
                         "through the tensor-core filter step; video_tc: the video job through the tensor-core "
                         "filter step on FP16 copies of its frames, beside the FP32 path; detect: the video job "
                         "with the presence decision on the device (detection surrogate + Eq. prior_detect); "
                         "pd_curves: the single-pixel p_d experiment of Sec. IV-A (Gaussian IRF, five betas); "
                         "fine: single-frame estimates on the sub-bin grid; msl: multispectral estimate (4 bands); "
                         "single: one 32x32 frame, T=1024 (absolute latency); "
                         "alu_peaks: measured FP32 FMA, packed "
                         "FMA and ex2 throughput (the denominators of the ALU rooflines)")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------------------------


def make_sequences(frames: int, device):
    """Three videos (one per SBR), [frames] tensors of [P, pitch] uint16 each, generated on `device`."""
    from paper_2004_09211_gb300 import synth
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(H, W, frames, peak + 8, T - L + peak - 8, SEED)
    hd = torch.from_numpy(h).to(device)
    pitch = synth.pad_pitch(T)
    gen = torch.Generator(device=device).manual_seed(SEED)
    videos = []
    for sbr in SBRS:
        frames_z = []
        for n in range(frames):
            b = float(sc.signal[n].mean()) / (sbr * T)
            mean = synth.expected_counts(torch.from_numpy(sc.depth[n]).to(device),
                                         torch.from_numpy(sc.signal[n]).to(device), b, hd, peak, T)
            z = synth.poisson_histograms(mean, gen).reshape(H * W, T)
            frames_z.append(synth.pitched(z, pitch))
            del mean
        videos.append(frames_z)
    return h, peak, hd, sc, videos


def run_job(spl, prms, hd, videos, states, outs, stream, ev=None, step=None, lanes=None):
    """One step: every (SBR, beta) run over all frames. Returns the number of kernel launches.
    lanes: optional list of (stream, outs) pairs; the runs are independent sequences and are then issued
    round-robin on those streams (each run stays on one stream, in frame order), joined back into `stream`."""
    step = step or spl.spl_filter_step
    launches = 0
    if lanes:
        start = torch.cuda.Event()
        start.record(stream)
        for s_, _ in lanes:
            s_.wait_event(start)
    for r, (vi, bi) in enumerate((vi, bi) for vi in range(len(videos)) for bi in range(len(BETAS))):
        st, o_ = lanes[r % len(lanes)] if lanes else (stream, outs)
        prm = prms[bi]
        mu, var = states[vi][bi]
        spl.spl_state_init(prm, mu[0], var[0], stream=st)
        launches += 1
        for n, z in enumerate(videos[vi]):
            src, dst = n & 1, (n + 1) & 1
            if ev is not None:
                ev[0].append(torch.cuda.Event(enable_timing=True))
                ev[0][-1].record(st)
            step(prm, z, hd, mu[src], var[src], out=dict(mu=mu[dst], var=var[dst], **o_), stream=st)
            if ev is not None:
                ev[1].append(torch.cuda.Event(enable_timing=True))
                ev[1][-1].record(st)
            # spl_filter_step on uint16 frames: tensor-core kernel, redo scan, intensity; otherwise depth, intensity
            launches += 3 if step is spl.spl_filter_step else 2
    if lanes:
        for s_, _ in lanes:
            done = torch.cuda.Event()
            done.record(s_)
            stream.wait_event(done)
    return launches


def depth_rmse(argmax, mu, sc, n: int) -> dict:
    """Depth RMSE (bins) of frame n's estimates against the scene's ground truth, for the argmax and for the posterior
    mean, on every pixel and on three groups: the static background that no object ever covered (where the filter
    converges), the moving objects (which jump 5-20 bins per frame, far beyond the prior's random walk) and the
    background an object has left (the filter keeps tracking the object's depth there: without the detection step
    of Algorithm 1 nothing resets a departed surface)."""
    gt = sc.depth[n].reshape(-1).astype(np.float64)
    a = np.asarray(argmax, np.float64).reshape(-1)
    m = np.asarray(mu, np.float64).reshape(-1)
    static = sc.static_mask(n).reshape(-1)
    objects = sc.object_mask(n).reshape(-1)
    out = {}
    for name, mask in (("all", np.ones(gt.size, bool)), ("static", static), ("objects", objects),
                       ("uncovered", ~static & ~objects)):
        if mask.any():
            out[name] = {"argmax": float(np.sqrt(np.mean((a[mask] - gt[mask]) ** 2))),
                         "mu": float(np.sqrt(np.mean((m[mask] - gt[mask]) ** 2))), "pixels": int(mask.sum())}
    return out


def job_rmse(spl, prms, hd, videos, sc, frames, dev, keep=None, step=None):
    """One untimed pass of the job on the current stream (through `step`, default spl_filter_step): the last
    frame's depth RMSE of every (SBR, beta) run, and, for keep = (run index, frame), that frame's (mu, argmax) of
    that run."""
    step = step or spl.spl_filter_step
    P = H * W
    mu = [torch.empty(P, device=dev) for _ in range(2)]
    var = [torch.empty(P, device=dev) for _ in range(2)]
    outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                bg=torch.empty(P, device=dev))
    runs, kept = [], None
    for r, (vi, bi) in enumerate((vi, bi) for vi in range(len(videos)) for bi in range(len(BETAS))):
        spl.spl_state_init(prms[bi], mu[0], var[0])
        for n, z in enumerate(videos[vi]):
            step(prms[bi], z, hd, mu[n & 1], var[n & 1], out=dict(mu=mu[(n + 1) & 1], var=var[(n + 1) & 1], **outs))
            if keep is not None and keep == (r, n):
                kept = (mu[(n + 1) & 1].cpu().numpy().copy(), outs["argmax"].cpu().numpy().copy())
        last = frames - 1
        runs.append({"sbr": SBRS[vi], "beta": BETAS[bi],
                     **depth_rmse(outs["argmax"].cpu().numpy(), mu[frames & 1].cpu().numpy(), sc, last)})
    return runs, kept


def replica_throughput(ms_local: float, units_per_rank: int, steps: int, world: int, device=None):
    """Whole-job figures of N independent replicas (the path has no data-path collective): the slowest rank's
    time bounds the job (max over ranks, all_reduce on `device` when a process group is initialised), and the
    value counts the units of every rank. Returns (ms_max, units per second)."""
    ms = float(ms_local)
    if world > 1:
        import torch.distributed as td
        t = torch.tensor([ms], device=device if device is not None else "cpu", dtype=torch.float64)
        td.all_reduce(t, op=td.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world * steps / (ms / 1e3)


def native(args):
    import paper_2004_09211_gb300 as spl
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spl.load_library()
    frames = args.frames
    h, peak, hd, sc, videos = make_sequences(frames, dev)
    P = H * W
    prms = [spl.make_params(H, W, T, L, peak, beta=b, sigma_rw2=SIGMA_RW2) for b in BETAS]
    states = [[([torch.empty(P, device=dev) for _ in range(2)], [torch.empty(P, device=dev) for _ in range(2)])
               for _ in BETAS] for _ in SBRS]
    outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                bg=torch.empty(P, device=dev))
    stream = torch.cuda.current_stream(dev)
    units = len(SBRS) * len(BETAS) * frames * P
    # the nine runs are independent sequences: issued round-robin on JOB_STREAMS streams (each with its own
    # output buffers), so one run's launch tail and intensity launch overlap another run's depth launch
    lanes = [(torch.cuda.Stream(dev), dict(argmax=torch.empty(P, dtype=torch.int32, device=dev),
                                           refl=torch.empty(P, device=dev), bg=torch.empty(P, device=dev)))
             for _ in range(JOB_STREAMS)]

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            td.barrier()

    for _ in range(args.warmup):
        run_job(spl, prms, hd, videos, states, outs, stream, lanes=lanes)
    barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        launches = 0
        for _ in range(args.steps):
            launches += run_job(spl, prms, hd, videos, states, outs, stream, lanes=lanes)
        stop.record(stream)
        barrier()
    ms = start.elapsed_time(stop)
    ms, value = replica_throughput(ms, units, args.steps, world, dev if dist else None)

    # the same job on the FP32 CUDA-core kernel (spl_filter_step_fp32), the plain path the route is measured against
    for _ in range(args.warmup):
        run_job(spl, prms, hd, videos, states, outs, stream, lanes=lanes, step=spl.spl_filter_step_fp32)
    barrier()
    start.record(stream)
    for _ in range(args.steps):
        run_job(spl, prms, hd, videos, states, outs, stream, lanes=lanes, step=spl.spl_filter_step_fp32)
    stop.record(stream)
    barrier()
    ms32, value32 = replica_throughput(start.elapsed_time(stop), units, args.steps, world, dev if dist else None)

    # rooflines of one filter step (time per step = job time / steps: the runs' steps overlap on the streams).
    # Algorithmic bytes per pixel-frame: histogram row (2 T) + previous state (mu, var) + outputs (mu, var,
    # argmax, refl, bg).
    alg_bytes = P * (2 * T + 8 + 20)
    n_steps = len(SBRS) * len(BETAS) * frames * args.steps
    peaks = _peaks()
    step_s, step32_s = ms / n_steps / 1e3, ms32 / n_steps / 1e3
    roofline = hbm_roofline(
        peaks, alg_bytes, step_s, capture_traffic("k_filter_tc_u16", P),
        "k_filter_tc<u16> + k_estimate_redo + k_intensity4 (one spl_filter_step; time per step = job time / steps, "
        f"the runs' steps overlapping on {JOB_STREAMS} streams)")
    roofline["issue"] = issue_roofline(dev, peaks, capture_traffic("k_filter_tc_u16", P, "inst_per_pixel"), step_s,
                                       "ncu smsp__inst_executed.sum of the three launches of one filter step, frame 1 "
                                       "of each of the nine runs (mean)")
    roofline32 = hbm_roofline(
        peaks, alg_bytes, step32_s, capture_traffic("k_estimate", P),
        "k_estimate<u16> + k_intensity4 (one spl_filter_step_fp32; time per step = job time / steps)")
    roofline32["issue"] = issue_roofline(dev, peaks, capture_traffic("k_estimate", P, "inst_per_pixel"), step32_s,
                                         "ncu smsp__inst_executed.sum, depth launch of frame 1 of each of the nine "
                                         "runs (mean) plus one intensity launch")

    # depth RMSE of every run's last frame (untimed pass), and the run the oracle checks below: SBR 0.1, beta 0.5
    keep_run = SBRS.index(0.1) * len(BETAS) + BETAS.index(0.5)
    rmse, kept = job_rmse(spl, prms, hd, videos, sc, frames, dev, keep=(keep_run, CROP_FRAMES - 1))
    rmse32, _ = job_rmse(spl, prms, hd, videos, sc, frames, dev, step=spl.spl_filter_step_fp32)

    e2e = e2e_hist = None
    if not args.no_e2e:
        e2e = end_to_end_toa(spl, prms, hd, videos, dev, stream, P)
        e2e_hist = end_to_end(spl, prms, hd, videos, dev, stream, P)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        y0 = (H - CROP) // 2
        zs = [videos[SBRS.index(0.1)][n][:, :T].reshape(H, W, T)[y0:y0 + CROP, y0:y0 + CROP].cpu().numpy()
              .astype(np.float64) for n in range(CROP_FRAMES)]
        cpu = cpu_baseline(h, peak, sc, single_thread_crop=64, zs=zs)
        # the GPU's full-frame results against the oracle's on the crop's interior (after CROP_FRAMES frames a pixel
        # depends only on inputs within that Chebyshev distance, so the crop reproduces the full frame there)
        m = CROP_FRAMES
        g_mu = kept[0].reshape(H, W)[y0 + m:y0 + CROP - m, y0 + m:y0 + CROP - m].astype(np.float64)
        g_am = kept[1].reshape(H, W)[y0 + m:y0 + CROP - m, y0 + m:y0 + CROP - m]
        o_mu = cpu.pop("oracle_mu")[m:CROP - m, m:CROP - m]
        o_am = cpu.pop("oracle_argmax")[m:CROP - m, m:CROP - m]
        cpu["gpu_vs_oracle"] = {"pixels": int(g_mu.size), "frame": CROP_FRAMES - 1, "run": "SBR 0.1, beta 0.5",
                                "rmse_mu_bins": float(np.sqrt(np.mean((g_mu - o_mu) ** 2))),
                                "max_rel_mu": float(np.max(np.abs(g_mu - o_mu) / np.abs(o_mu))),
                                "argmax_equal_frac": float(np.mean(g_am == o_am))}

    if rank == 0:
        line = {
            "metric": "pixel-frames/s", "value": value, "unit": "pixel-frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u16 counts -> f16 on chip (exact below 1024) x f16 hi/lo taps -> f32 (tensor); f32 epilogue",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "pixels": P, "frames": frames, "T": T, "L": L,
                       "sequences": len(SBRS), "betas": list(BETAS), "hist": "uint16",
                       "pixel_frames_per_step": units, "l2": "inputs larger than L2 (197 MB per frame), no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "e2e": e2e, "e2e_histograms": e2e_hist, "gpu_launches": launches,
            "clocks": clk.summary(),
            "fp32_path": {"value": value32, "ms_per_step": ms32 / args.steps, "dtype": "f32",
                          "entry": "spl_filter_step_fp32", "roofline": roofline32,
                          "depth_rmse_last_frame": rmse32},
            "cpu_baseline": cpu, "depth_rmse_last_frame": rmse,
        }
        print(json.dumps(line), flush=True)
    if dist:
        td.destroy_process_group()


def toa_from_histograms(z, T):
    """The photon lists of one frame whose histograms are z ([P, pitch] uint16 on the device): CSR offsets int32
    [P + 1] and bins uint16, each bin repeated by its count, in bin order within a pixel."""
    zi = z[:, :T].to(torch.int32)
    offsets = torch.zeros(zi.shape[0] + 1, dtype=torch.int32, device=z.device)
    offsets[1:] = torch.cumsum(zi.sum(1), 0)
    nz = zi.nonzero()
    bins = torch.repeat_interleave(nz[:, 1], zi[nz[:, 0], nz[:, 1]].to(torch.int64))
    return offsets, bins.to(torch.int32).to(torch.uint16)


def end_to_end_toa(spl, prms, hd, videos, dev, stream, P):
    """Same job through the public API from photon time-of-arrival lists in pinned HOST memory (the ToAs of Sec.
    II-A as CSR lists of uint16 bins, the same photons as the histograms of the device-resident job): inside the
    timed region every frame's lists are copied host -> device (on each lane's copy stream, double-buffered), turned
    into uint16 histograms on the device (spl_toa_histogram) and filtered (spl_filter_step), and every frame's
    outputs (mu, var, argmax, refl, bg) are read back to pinned host buffers. The runs are issued round-robin on
    JOB_STREAMS lanes like the device-resident job."""
    host = []
    maxn = 0
    resident = []  # device lists of the first frames of every video, for the kernel roofline below
    for v in videos:
        hv = []
        for n, z in enumerate(v):
            off, bins = toa_from_histograms(z, T)
            if n < 10:
                resident.append((off, bins))
            ho = torch.empty(off.shape, dtype=off.dtype, pin_memory=True)
            ho.copy_(off)
            hb = torch.empty(bins.shape, dtype=bins.dtype, pin_memory=True)
            hb.copy_(bins)
            hv.append((ho, hb))
            maxn = max(maxn, bins.numel())
        host.append(hv)
    torch.cuda.synchronize(dev)
    pitch = videos[0][0].shape[1]
    frames = len(host[0])

    class Lane:
        def __init__(self):
            self.stream = torch.cuda.Stream(dev)
            self.copy = torch.cuda.Stream(dev)
            self.off = [torch.empty(P + 1, dtype=torch.int32, device=dev) for _ in range(2)]
            self.bins = [torch.empty(max(maxn, 1), dtype=torch.uint16, device=dev) for _ in range(2)]
            self.z = torch.empty(P, pitch, dtype=torch.uint16, device=dev)
            # a frame's five outputs (mu, var, argmax, refl, bg) in one block, read back with one copy; two blocks,
            # since mu and var are also the next frame's input state
            self.blk = [torch.empty(5 * P, dtype=torch.float32, device=dev) for _ in range(2)]
            self.mu = [b[:P] for b in self.blk]
            self.var = [b[P:2 * P] for b in self.blk]
            self.outs = [dict(argmax=b[2 * P:3 * P].view(torch.int32), refl=b[3 * P:4 * P], bg=b[4 * P:])
                         for b in self.blk]
            self.hout = torch.empty(5 * P, dtype=torch.float32).pin_memory()
            self.copied = [torch.cuda.Event() for _ in range(2)]
            self.consumed = [torch.cuda.Event() for _ in range(2)]
            self.i = 0

    lanes = [Lane() for _ in range(JOB_STREAMS)]
    h2d = d2h = 0

    def put(ln, vi, n):  # the frame's lists into the lane's next buffer, on its copy stream
        nonlocal h2d
        s = ln.i & 1
        ho, hb = host[vi][n]
        with torch.cuda.stream(ln.copy):
            ln.copy.wait_event(ln.consumed[s])
            ln.off[s].copy_(ho, non_blocking=True)
            if hb.numel():
                ln.bins[s][:hb.numel()].copy_(hb, non_blocking=True)
            ln.copied[s].record(ln.copy)
        h2d += ho.numel() * 4 + hb.numel() * 2

    def job():
        nonlocal h2d, d2h
        h2d = d2h = 0
        start = torch.cuda.Event()
        start.record(stream)
        for ln in lanes:
            ln.stream.wait_event(start)
            ln.copy.wait_event(start)
            ln.i = 0
        runs = [(vi, bi) for vi in range(len(host)) for bi in range(len(prms))]
        for r, (vi, bi) in enumerate(runs):
            ln = lanes[r % len(lanes)]
            if r < len(lanes):  # a lane's first frame; the later runs' first frames are put by the run before
                put(ln, vi, 0)
            spl.spl_state_init(prms[bi], ln.mu[0], ln.var[0], stream=ln.stream)
            for n in range(frames):
                s = ln.i & 1
                # the next frame of this lane (this run's next frame, or the first frame of its next run)
                nxt = (vi, n + 1) if n + 1 < frames else (runs[r + len(lanes)][0], 0) \
                    if r + len(lanes) < len(runs) else None
                ln.stream.wait_event(ln.copied[s])
                nb = host[vi][n][1].numel()
                spl.spl_toa_histogram(prms[bi], ln.off[s], ln.bins[s][:nb], out=ln.z, stream=ln.stream)
                src, dst = n & 1, (n + 1) & 1
                spl.spl_filter_step(prms[bi], ln.z, hd, ln.mu[src], ln.var[src],
                                    out=dict(mu=ln.mu[dst], var=ln.var[dst], **ln.outs[dst]), stream=ln.stream)
                ln.consumed[s].record(ln.stream)
                with torch.cuda.stream(ln.stream):
                    ln.hout.copy_(ln.blk[dst], non_blocking=True)
                d2h += ln.blk[dst].numel() * 4
                ln.i += 1
                if nxt is not None:
                    put(ln, *nxt)
        for ln in lanes:
            done = torch.cuda.Event()
            done.record(ln.stream)
            stream.wait_event(done)
        return len(runs) * frames

    job()  # warm-up (also primes the events)
    torch.cuda.synchronize(dev)
    assert spl.spl_toa_status() == 0
    times = []
    for _ in range(E2E_JOBS):  # each job timed on its own; the value is over all of them
        t0 = time.perf_counter()
        n = job()
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)

    # the histogram kernel alone on device-resident lists (the first 10 frames of each video, one after another on
    # one stream; each launch writes a 197 MB cube, larger than L2): algorithmic bytes = the rows written
    # (2 pitch per pixel) + the photons (2 B each) and offsets (4 B per pixel) read
    zb = lanes[0].z
    for off, bins in resident[:3]:
        spl.spl_toa_histogram(prms[0], off, bins, out=zb, stream=stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for off, bins in resident:
        spl.spl_toa_histogram(prms[0], off, bins, out=zb, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    assert spl.spl_toa_status() == 0
    launch_s = ev0.elapsed_time(ev1) / 1e3 / len(resident)
    alg = sum(P * pitch * 2 + b.numel() * 2 + (P + 1) * 4 for _, b in resident) / len(resident)
    kern = hbm_roofline(_peaks(), alg, launch_s, None,
                        "k_toa_hist (spl_toa_histogram; mean over the first 10 frames of the three videos)")
    return {"value": n * P / dt, "unit": "pixel-frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "job_seconds": times, "toa_histogram_roofline": kern,
            "note": "photon ToA lists (CSR, uint16 bins; the same photons as the histograms) in pinned host memory, "
                    "copied each frame, histogrammed on the device (spl_toa_histogram) and filtered "
                    "(spl_filter_step) on 3 lanes; outputs read back each frame"}


def end_to_end(spl, prms, hd, videos, dev, stream, P):
    """Same job through the public API with the histograms in pinned HOST memory: every frame is copied
    host -> device inside the timed region (double-buffered on a copy stream) and every frame's outputs
    (mu, var, argmax, refl, bg) are read back to pinned host buffers."""
    host = []
    for v in videos:
        hv = []
        for z in v:
            hz = torch.empty(z.shape, dtype=z.dtype, pin_memory=True)
            hz.copy_(z)
            hv.append(hz)
        host.append(hv)
    pitch = videos[0][0].shape[1]
    dbuf = [torch.empty(P, pitch, dtype=torch.uint16, device=dev) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    hout = {k: torch.empty(P, dtype=dt).pin_memory() for k, dt in
            (("mu", torch.float32), ("var", torch.float32), ("argmax", torch.int32), ("refl", torch.float32),
             ("bg", torch.float32))}
    mu = [torch.empty(P, device=dev) for _ in range(2)]
    var = [torch.empty(P, device=dev) for _ in range(2)]
    outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                bg=torch.empty(P, device=dev))
    frames = len(host[0])
    h2d = d2h = 0
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]

    def job():
        nonlocal h2d, d2h
        h2d = d2h = 0
        seq = [(vi, bi, n) for vi in range(len(host)) for bi in range(len(prms)) for n in range(frames)]
        with torch.cuda.stream(copy_stream):
            dbuf[0].copy_(host[seq[0][0]][seq[0][2]], non_blocking=True)
            copied[0].record(copy_stream)
        for i, (vi, bi, n) in enumerate(seq):
            s = i & 1
            if i + 1 < len(seq):
                nvi, _, nn = seq[i + 1]
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(consumed[1 - s])
                    dbuf[1 - s].copy_(host[nvi][nn], non_blocking=True)
                    copied[1 - s].record(copy_stream)
            h2d += host[vi][n].numel() * 2
            stream.wait_event(copied[s])
            if n == 0:
                spl.spl_state_init(prms[bi], mu[0], var[0], stream=stream)
            src, dst = n & 1, (n + 1) & 1
            o = spl.spl_filter_step(prms[bi], dbuf[s], hd, mu[src], var[src],
                                    out=dict(mu=mu[dst], var=var[dst], **outs), stream=stream)
            consumed[s].record(stream)
            for k in hout:
                hout[k].copy_(o[k], non_blocking=True)
                d2h += o[k].numel() * 4
        return len(seq)

    job()  # warm-up (also primes the events)
    torch.cuda.synchronize(dev)
    times = []
    for _ in range(E2E_JOBS):
        t0 = time.perf_counter()
        n = job()
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    return {"value": n * P / dt, "unit": "pixel-frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "job_seconds": times,
            "note": "histograms in pinned host memory, copied each frame; outputs read back each frame"}


# ---------------------------------------------------------------------------------------------------------
# CPU oracle baseline (the reference arm of this benchmark)
# ---------------------------------------------------------------------------------------------------------

CROP = 128         # oracle sample: a CROP x CROP window of the SBR 0.1 sequence, beta = 0.5
CROP_FRAMES = 3


def cpu_sample_inputs(h, peak, sc, frames=CROP_FRAMES, crop=CROP):
    """The oracle's bounded sample: the first frames of the SBR = 0.1 sequence on a centred crop, generated
    on the host from the same scene (a CPU random stream; the oracle is timed, not compared, here)."""
    from paper_2004_09211_gb300 import synth
    g = torch.Generator().manual_seed(SEED)
    y0 = (H - crop) // 2
    zs = []
    for n in range(frames):
        b = float(sc.signal[n].mean()) / (0.1 * T)
        d = torch.from_numpy(sc.depth[n][y0:y0 + crop, y0:y0 + crop].copy())
        s = torch.from_numpy(sc.signal[n][y0:y0 + crop, y0:y0 + crop].copy())
        mean = synth.expected_counts(d, s, b, torch.from_numpy(h), peak, T)
        zs.append(torch.poisson(mean, generator=g).numpy().astype(np.float64))
    return zs


def cpu_baseline(h, peak, sc, frames=CROP_FRAMES, crop=CROP, single_thread_crop=0, zs=None):
    """The oracle's filter steps (+ intensity) on a crop of the video job, OpenMP over pixels on every host core;
    with single_thread_crop > 0, also one frame of a smaller crop on one thread. zs: the crop's histograms (the
    GPU's own frames, copied to the host); default: drawn on the host from the same scene."""
    from oracle import oracle as orc
    from paper_2004_09211_gb300 import synth
    q = orc.params(T, L, peak, beta=0.5, sigma_rw2=SIGMA_RW2, nu=synth.cross_weights(0.5))

    last = {}

    def run(zs, c):
        mu, var = orc.state_init(q, c, c)
        t0 = time.perf_counter()
        for z in zs:
            e = orc.filter_step(q, h, z, mu, var)
            mu, var = e["mu"], e["var"]
            orc.intensity(q, h, z, mu)
        dt_ = time.perf_counter() - t0
        last.update(mu=mu, argmax=e["argmax"])
        return dt_

    cores = orc.set_threads(os.cpu_count() or 1)
    dt = run(zs if zs is not None else cpu_sample_inputs(h, peak, sc, frames, crop), crop)
    out = {"value": crop * crop * frames / dt, "unit": "pixel-frames/s", "cores": cores, "kind": "oracle",
           "sample": f"{crop}x{crop} crop x {frames} frames of the SBR 0.1 sequence, beta 0.5 "
                     f"(filter step + intensity, FP64, OpenMP over pixels)", "seconds": dt,
           "oracle_mu": last["mu"], "oracle_argmax": last["argmax"]}
    if single_thread_crop > 0:
        c = single_thread_crop
        one = orc.set_threads(1)
        try:
            dt1 = run(cpu_sample_inputs(h, peak, sc, 1, c), c)
        finally:
            orc.set_threads(cores)
        out["single_thread"] = {"value": c * c / dt1, "unit": "pixel-frames/s", "cores": one,
                                "sample": f"{c}x{c} crop x 1 frame, same sequence", "seconds": dt1}
    return out


def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2004_09211_gb300 import synth
    h, peak = synth.asymmetric_irf(L=L)
    sc = synth.moving_scene(H, W, CROP_FRAMES, peak + 8, T - L + peak - 8, SEED)
    for _ in range(args.warmup):
        cpu_baseline(h, peak, sc, frames=1, crop=32)
    secs = []
    vals = []
    for _ in range(max(1, args.steps)):
        r = cpu_baseline(h, peak, sc, frames=1)
        secs.append(r["seconds"])
        vals.append(r["value"])
    value = statistics.mean(vals)
    units = CROP * CROP
    line = {"impl": "reference", "metric": "pixel-frames/s", "value": value, "unit": "pixel-frames/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{CROP}x{CROP} crop x 1 frame per step"},
            "cpu_baseline": {"value": value, "unit": "pixel-frames/s", "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": "pixel-frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "units_per_step": units}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------------
# secondary workloads (one JSON line each; the default run prints the video line only)
# ---------------------------------------------------------------------------------------------------------

BATCH_SEQS = 64
BATCH_FRAMES = 10


def batched(args):
    """64 independent sequences, sides {32..512} (square or 2:1), T in {512..4096}, per-sequence Gaussian
    (sigma 2-6 bins, taps +-4 sigma) or 48-tap asymmetric IRF and beta in [0.1, 1]; photon lists (0-30 photons
    per pixel: Poisson(3) signal + Poisson(10) background, truncated); 10 frames per step, captured in one CUDA
    graph of 10 persistent launches. Also timed: the same sequences stepped one plan (one launch) per sequence."""
    import paper_2004_09211_gb300 as spl
    from paper_2004_09211_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    rng = np.random.default_rng(4)
    gen = torch.Generator(device=dev).manual_seed(4)
    seqs = []
    for s in range(BATCH_SEQS):
        side = int(rng.choice([32, 64, 128, 256, 512]))
        Hs, Ws = side, side * (2 if rng.random() < 0.5 else 1)
        T = int(rng.choice([512, 1024, 2048, 4096]))
        if rng.random() < 0.5:
            sig = rng.uniform(2.0, 6.0)
            h, peak = synth.gaussian_irf(sig, int(math.ceil(4 * sig)))
        else:
            h, peak = synth.asymmetric_irf(L=48)
        beta = float(rng.uniform(0.1, 1.0))
        L = len(h)
        sc = synth.moving_scene(Hs, Ws, BATCH_FRAMES, peak + 8, T - L + peak - 8, 400 + s)
        hd = torch.from_numpy(h).to(dev)
        frames = [synth.toa_lists_torch(torch.from_numpy(sc.depth[n]).to(dev), torch.tensor(3.0, device=dev), 10.0,
                                        hd, peak, T, gen) for n in range(BATCH_FRAMES)]
        prm = spl.make_params(Hs, Ws, T, L, peak, beta=beta, sigma_rw2=SIGMA_RW2)
        P = Hs * Ws
        st_mu = [torch.empty(P, device=dev) for _ in range(BATCH_FRAMES + 1)]
        st_var = [torch.empty(P, device=dev) for _ in range(BATCH_FRAMES + 1)]
        outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                    bg=torch.empty(P, device=dev))
        seqs.append(dict(prm=prm, h=hd, frames=frames, mu=st_mu, var=st_var, outs=outs, P=P, sc=sc, T=T))
    units = sum(q["P"] for q in seqs) * BATCH_FRAMES
    photons = sum(int(f[1].numel()) for q in seqs for f in q["frames"])

    def frame_dicts(n):
        return [dict(h=q["h"], offsets=q["frames"][n][0], bins=q["frames"][n][1], mu_in=q["mu"][n],
                     var_in=q["var"][n], mu_out=q["mu"][n + 1], var_out=q["var"][n + 1], **q["outs"]) for q in seqs]

    def init_states():
        for q in seqs:
            spl.spl_state_init(q["prm"], q["mu"][0], q["var"][0])

    plan = spl.spl_batch_create([q["prm"] for q in seqs], nslots=BATCH_FRAMES)
    for n in range(BATCH_FRAMES):
        spl.spl_batch_set(plan, n, frame_dicts(n))
    init_states()
    spl.spl_batch_tune(plan, 0)
    info = spl.spl_batch_info(plan)
    launches_per_frame = sum(1 for c in info["classes"] if c["units"] > 0)
    init_states()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        for n in range(BATCH_FRAMES):
            spl.spl_batch_step(plan, n, stream=s)
    torch.cuda.current_stream(dev).wait_stream(s)
    torch.cuda.synchronize(dev)
    with torch.cuda.graph(g):
        for n in range(BATCH_FRAMES):
            spl.spl_batch_step(plan, n)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    flags = spl.spl_batch_status(plan)
    # baseline: one single-sequence plan per sequence, stepped one after the other
    plans = [spl.spl_batch_create([q["prm"]], nslots=BATCH_FRAMES) for q in seqs]
    for i, q in enumerate(seqs):
        for n in range(BATCH_FRAMES):
            spl.spl_batch_set(plans[i], n, [frame_dicts(n)[i]])
    for _ in range(2):
        for n in range(BATCH_FRAMES):
            for pl in plans:
                spl.spl_batch_step(pl, n)
    torch.cuda.synchronize(dev)
    e0.record()
    for n in range(BATCH_FRAMES):
        for pl in plans:
            spl.spl_batch_step(pl, n)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_unbatched = e0.elapsed_time(e1)
    for pl in plans:
        spl.spl_batch_destroy(pl)
    spl.spl_batch_destroy(plan)

    # depth RMSE of the batched step at the last frame (the graph replays left every sequence's last state), and
    # the same sequences through the plain FP32 histogram path: histograms built from the same photon lists
    # (outside the timed region), one spl_filter_step_fp32 per sequence and frame, timed frame by frame
    def pooled(parts):
        out = {}
        for k in ("all", "static", "objects", "uncovered"):
            n = sum(p_[k]["pixels"] for p_ in parts if k in p_)
            if n:
                out[k] = {m: float(np.sqrt(sum(p_[k][m] ** 2 * p_[k]["pixels"] for p_ in parts if k in p_) / n))
                          for m in ("argmax", "mu")}
                out[k]["pixels"] = n
        return out

    last = BATCH_FRAMES - 1
    per_seq = [depth_rmse(q["outs"]["argmax"].cpu().numpy(), q["mu"][BATCH_FRAMES].cpu().numpy(), q["sc"], last)
               for q in seqs]
    low_beta = [i for i, q in enumerate(seqs) if q["prm"].beta <= 0.5]
    rmse_batched = {"all_sequences": pooled(per_seq), "beta_le_0.5": pooled([per_seq[i] for i in low_beta]),
                    "beta_le_0.5_sequences": len(low_beta)}
    batched_mu = [q["mu"][BATCH_FRAMES].clone() for q in seqs]
    plain_mu = [[torch.empty(q["P"], device=dev) for _ in range(2)] for q in seqs]
    plain_var = [[torch.empty(q["P"], device=dev) for _ in range(2)] for q in seqs]
    for i, q in enumerate(seqs):
        spl.spl_state_init(q["prm"], plain_mu[i][0], plain_var[i][0])
    ms_plain = 0.0
    hist_bytes = 0
    for n in range(BATCH_FRAMES):
        hists = []
        for q in seqs:
            off, bins = q["frames"][n]
            pitch = synth.pad_pitch(q["T"])
            cnt = (off[1:] - off[:-1]).to(torch.int64)
            pix = torch.repeat_interleave(torch.arange(q["P"], device=dev), cnt)
            zz = torch.zeros(q["P"] * pitch, dtype=torch.int32, device=dev)
            zz.index_add_(0, pix * pitch + bins.to(torch.int64), torch.ones_like(pix, dtype=torch.int32))
            hists.append(zz.to(torch.uint16).reshape(q["P"], pitch))
            del zz, pix, cnt
        hist_bytes = sum(z_.numel() * 2 for z_ in hists)
        torch.cuda.synchronize(dev)
        e0.record()
        for i, q in enumerate(seqs):
            spl.spl_filter_step_fp32(q["prm"], hists[i], q["h"], plain_mu[i][n & 1], plain_var[i][n & 1],
                                     out=dict(mu=plain_mu[i][(n + 1) & 1], var=plain_var[i][(n + 1) & 1],
                                              **q["outs"]))
        e1.record()
        torch.cuda.synchronize(dev)
        ms_plain += e0.elapsed_time(e1)
        del hists
    fin = BATCH_FRAMES & 1
    per_plain = [depth_rmse(q["outs"]["argmax"].cpu().numpy(), plain_mu[i][fin].cpu().numpy(), q["sc"], last)
                 for i, q in enumerate(seqs)]
    rmse_plain = {"all_sequences": pooled(per_plain), "beta_le_0.5": pooled([per_plain[i] for i in low_beta])}
    rel = max(float(((plain_mu[i][fin] - batched_mu[i]).abs() / batched_mu[i].abs()).max()) for i in range(len(seqs)))
    plain = {"value": units / (ms_plain / 1e3), "ms_per_step": ms_plain,
             "histogram_bytes_per_frame": hist_bytes, "depth_rmse_last_frame": rmse_plain,
             "max_rel_mu_vs_batched": rel,
             "note": "the same 64 sequences and photons as uint16 histograms through spl_filter_step_fp32 (one launch "
                     "pair per sequence and frame, 640 per step), histograms built outside the timed region"}
    # roofline of k_batch: algorithmic bytes per frame of every sequence = 4 B per photon (bin index) + 32 B per
    # pixel (list offset, previous state, new state, argmax, refl, bg); its time = the graph's time over its 10
    # frames (each frame's nodes are an 8-byte memset and one launch per size class)
    peaks = _peaks()
    P_all = units // BATCH_FRAMES
    launch_s = ms / BATCH_FRAMES / 1e3
    roofline = hbm_roofline(
        peaks, 4 * photons // BATCH_FRAMES + 32 * P_all, launch_s, capture_traffic("k_batch", P_all),
        "k_batch (one frame of all 64 sequences: one launch per size class)",
        issue=issue_roofline(dev, peaks, capture_traffic("k_batch", P_all, "inst_per_pixel"), launch_s,
                             "ncu smsp__inst_executed.sum of the launches of one frame of this workload"),
        note="latency-bound: up to 4049 candidates per pixel from at most 30 photons")
    line = {"metric": "pixel-frames/s", "value": units / (ms / 1e3), "unit": "pixel-frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched: 64 photon-list sequences x 10 frames, sides 32-512, T 512-4096",
                       "pixels": units // BATCH_FRAMES, "frames": BATCH_FRAMES, "photons_per_step": photons,
                       "tile": info["tile"], "size_classes": info["classes"],
                       "graph": f"{launches_per_frame * BATCH_FRAMES} persistent launches (one per size class and "
                                "frame) captured in one CUDA graph"},
            "unbatched": {"value": units / (ms_unbatched / 1e3), "ms_per_step": ms_unbatched,
                          "note": "same sequences, one single-sequence plan per sequence, 640 launches"},
            "plain_fp32_histograms": plain, "depth_rmse_last_frame": rmse_batched,
            "status_flags": flags, "gpu_launches": launches_per_frame * BATCH_FRAMES * args.steps,
            "clocks": clk.summary(),
            "roofline": roofline}
    print(json.dumps(line), flush=True)


def diff(args):
    """Differentiable filter: 128 x 128 pixels x 20 frames, T = 1024, 48-tap asymmetric IRF, soft-argmax readout
    (tau = 0.5), loss = MSE to the ground-truth depth, gradients for h, beta and the 3x3 weights. One step =
    forward (states, readouts, loss) + backward (gradients)."""
    import paper_2004_09211_gb300 as spl
    from paper_2004_09211_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    Hd = Wd = 128
    N, Td, Ld = 20, 1024, 48
    h, peak = synth.asymmetric_irf(L=Ld)
    sc = synth.moving_scene(Hd, Wd, N, peak + 8, Td - Ld + peak - 8, 5)
    gen = torch.Generator(device=dev).manual_seed(5)
    hd = torch.from_numpy(h).to(dev)
    pitch = synth.pad_pitch(Td)
    zs = []
    for n in range(N):
        mean = synth.expected_counts(torch.from_numpy(sc.depth[n]).to(dev), torch.from_numpy(sc.signal[n]).to(dev),
                                     float(sc.signal[n].mean()) / (0.1 * Td), hd, peak, Td)
        zs.append(synth.pitched(synth.poisson_histograms(mean, gen).reshape(-1, Td), pitch))
    z = torch.stack(zs).contiguous()
    d_ref = torch.from_numpy(sc.depth.reshape(N, -1).astype(np.float32)).to(dev)
    prm = spl.make_params(Hd, Wd, Td, Ld, peak, beta=0.5, sigma_rw2=SIGMA_RW2)
    P = Hd * Wd
    mu_s = torch.empty(N + 1, P, device=dev)
    var_s = torch.empty(N + 1, P, device=dev)
    scratch = torch.empty(spl.spl_diff_scratch_size(prm), dtype=torch.uint8, device=dev)

    def step(ev=None):
        spl.spl_state_init(prm, mu_s[0], var_s[0])
        fw = spl.spl_diff_forward(prm, z, hd, 0.5, d_ref=d_ref, mu_states=mu_s, var_states=var_s, scratch=scratch)
        if ev is not None:
            ev[0].record()
        bw = spl.spl_diff_backward(prm, z, hd, 0.5, d_ref, mu_s, var_s, scratch=scratch)
        if ev is not None:
            ev[1].record()
        return fw, bw

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(0) as clk:
        e0.record()
        for i in range(args.steps):
            fw, bw = step(bev[i])
        e1.record()
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    # roofline of the dominant kernel, k_diff_backward (65 % of the step): algorithmic bytes per launch = the
    # frame's rows (2 T per pixel) + the previous states and this state's adjoints (16 B) + d_ref (4 B) + the
    # 9 x 2 neighbour-state adjoints written (72 B); its average launch time = spl_diff_backward's event time
    # over its N launches (the call's 19 gather launches and one finalize launch, about 1 % of it, included)
    peaks = _peaks()
    bw_s = sum(a.elapsed_time(b) for a, b in bev) / args.steps / N / 1e3
    roofline = hbm_roofline(
        peaks, P * (2 * Td + 92), bw_s, capture_traffic("k_diff_backward", P),
        "k_diff_backward (one frame of the reverse sweep)",
        issue=issue_roofline(dev, peaks, capture_traffic("k_diff_backward", P, "inst_per_pixel"), bw_s,
                             "ncu smsp__inst_executed.sum, mean of the 20 backward launches of one step"),
        note="latency-bound at 12 resident warps per SM (register and shared-memory limits)")
    line = {"metric": "pixel-frames/s", "value": P * N / (ms / 1e3), "unit": "pixel-frames/s (forward+backward)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "differentiable 128x128x20 frames, T=1024, L=48, tau=0.5", "pixels": P,
                       "frames": N},
            "loss": float(fw["loss"].item()), "grad_beta": float(bw["grad_beta"].item()),
            "gpu_launches": (1 + N + 1 + N + (N - 1) + 1) * args.steps, "clocks": clk.summary(),
            "roofline": roofline}
    print(json.dumps(line), flush=True)


def video_tc(args):
    """The video job (the headline workload) through spl_filter_step_tc on FP16 copies of its uint16 frames (the
    counts are small integers, exact in FP16), timed like the headline (the runs on JOB_STREAMS streams), beside
    spl_filter_step_fp32 on the original frames. Also reported: the depth RMSE of both paths against the ground truth at every run's last frame."""
    import paper_2004_09211_gb300 as spl
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    frames = args.frames
    h, peak, hd, sc, videos = make_sequences(frames, dev)
    videos16 = [[z.to(torch.int32).to(torch.float16) for z in v] for v in videos]
    P = H * W
    prms = [spl.make_params(H, W, T, L, peak, beta=b, sigma_rw2=SIGMA_RW2) for b in BETAS]
    states = [[([torch.empty(P, device=dev) for _ in range(2)], [torch.empty(P, device=dev) for _ in range(2)])
               for _ in BETAS] for _ in SBRS]
    outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                bg=torch.empty(P, device=dev))
    stream = torch.cuda.current_stream(dev)
    units = len(SBRS) * len(BETAS) * frames * P
    # the runs on JOB_STREAMS streams, as in the headline job (two tensor-core CTAs fill an SM's shared memory, so a
    # CTA of another launch never waits there for tensor memory)
    lanes = [(torch.cuda.Stream(dev), dict(argmax=torch.empty(P, dtype=torch.int32, device=dev),
                                           refl=torch.empty(P, device=dev), bg=torch.empty(P, device=dev)))
             for _ in range(JOB_STREAMS)]

    def timed(step, vids):
        for _ in range(args.warmup):
            run_job(spl, prms, hd, vids, states, outs, stream, step=step, lanes=lanes)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            run_job(spl, prms, hd, vids, states, outs, stream, step=step, lanes=lanes)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps, job_rmse(spl, prms, hd, vids, sc, frames, dev, step=step)[0]

    with ClockSampler(0) as clk:
        ms_tc, rmse_tc = timed(spl.spl_filter_step_tc, videos16)
    flags = spl.spl_tc_status()
    ms_32, rmse_32 = timed(spl.spl_filter_step_fp32, videos)
    runs = [f"SBR {sb} beta {b}" for sb in SBRS for b in BETAS]
    # roofline of one filter step (tensor-core depth launch + intensity launch): FP16 row (2 T) + previous state
    # (8 B) + outputs (20 B) per pixel; time per step = job time / steps (no capture of this workload)
    roofline = hbm_roofline(_peaks(), P * (2 * T + 8 + 20), ms_tc / 1e3 / (len(SBRS) * len(BETAS) * frames), None,
                            "k_filter_tc + k_intensity4 (one spl_filter_step_tc)",
                            note="traffic not captured for this workload")
    line = {"metric": "pixel-frames/s", "value": units / (ms_tc / 1e3), "unit": "pixel-frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_tc, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 x f16 -> f32 (tensor), f32 epilogue",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + ", FP16 copies of the counts", "pixels": P, "frames": frames,
                       "pixel_frames_per_step": units},
            "fp32_path": {"value": units / (ms_32 / 1e3), "ms_per_step": ms_32, "speedup_tc_over_fp32": ms_32 / ms_tc},
            "depth_rmse_last_frame": {r: {"tc": {k: a[k] for k in ("all", "static", "objects", "uncovered") if k in a},
                                             "fp32": {k: b[k] for k in ("all", "static", "objects", "uncovered")
                                                      if k in b}}
                                      for r, a, b in zip(runs, rmse_tc, rmse_32)},
            "status_flags": flags, "gpu_launches": len(SBRS) * len(BETAS) * (2 * frames + 1) * args.steps,
            "clocks": clk.summary(), "roofline": roofline, "e2e": None}
    print(json.dumps(line), flush=True)


def detect(args):
    """The video job with the presence decision of Algorithm 1 on the device: per frame spl_filter_step_detect
    (depth, moments and the detection surrogate with the intensity rule) and spl_pi_propagate (Eq. prior_detect
    for the next frame), the decision feeding the next frame's present_in. Timed like the headline, beside the
    plain spl_filter_step job (the same depth arithmetic). Every pixel of this scene has a surface, so the fraction declared present at each
    run's last frame is the detection rate; the false-alarm rate is measured on one background-only frame per
    SBR (same background level, pi0 = 0.5)."""
    import paper_2004_09211_gb300 as spl
    from paper_2004_09211_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    frames = args.frames
    h, peak, hd, sc, videos = make_sequences(frames, dev)
    P = H * W
    prms = [spl.make_params(H, W, T, L, peak, beta=b, sigma_rw2=SIGMA_RW2) for b in BETAS]
    states = [[([torch.empty(P, device=dev) for _ in range(2)], [torch.empty(P, device=dev) for _ in range(2)])
               for _ in BETAS] for _ in SBRS]
    outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                bg=torch.empty(P, device=dev))
    stream = torch.cuda.current_stream(dev)
    units = len(SBRS) * len(BETAS) * frames * P

    def lane_buffers():
        return dict(pi=[torch.empty(P, device=dev) for _ in range(2)],
                    pres=[torch.empty(P, dtype=torch.uint8, device=dev) for _ in range(2)],
                    pi0=torch.empty(P, device=dev),
                    outs=dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                              bg=torch.empty(P, device=dev)))

    # the nine runs are independent sequences: issued round-robin on JOB_STREAMS streams, each with its own
    # buffers, as in the headline job
    lanes = [(torch.cuda.Stream(dev), lane_buffers()) for _ in range(JOB_STREAMS)]
    plain_lanes = [(st, lb["outs"]) for st, lb in lanes]

    def run(vi, bi, st=None, lb=None):
        """One (SBR, beta) run over all frames on stream st with lane buffers lb; returns the last frame's
        decisions."""
        st = st if st is not None else stream
        lb = lb if lb is not None else lanes[0][1]
        prm = prms[bi]
        mu, var = states[vi][bi]
        spl.spl_state_init(prm, mu[0], var[0], stream=st)
        pi0 = pres = None
        for n, z in enumerate(videos[vi]):
            src, dst = n & 1, (n + 1) & 1
            o = spl.spl_filter_step_detect(prm, z, hd, mu[src], var[src], present_in=pres, pi0=pi0,
                                           out=dict(mu=mu[dst], var=var[dst], pi=lb["pi"][n & 1],
                                                    present=lb["pres"][n & 1], **lb["outs"]), stream=st)
            pi0 = spl.spl_pi_propagate(prm, o["pi"], pi_out=lb["pi0"], stream=st)
            pres = o["present"]
        return pres

    def job():
        start = torch.cuda.Event()
        start.record(stream)
        for st, _ in lanes:
            st.wait_event(start)
        runs = [(vi, bi) for vi in range(len(SBRS)) for bi in range(len(BETAS))]
        for r, (vi, bi) in enumerate(runs):
            st, lb = lanes[r % len(lanes)]
            run(vi, bi, st, lb)
        for st, _ in lanes:
            done = torch.cuda.Event()
            done.record(st)
            stream.wait_event(done)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / args.steps

    with ClockSampler(0) as clk:
        ms_det = timed(job)
    launches = len(SBRS) * len(BETAS) * (1 + 4 * frames) * args.steps  # state init; depth, redo scan, intensity, pi
    p_d = {f"SBR {SBRS[vi]} beta {BETAS[bi]}": float(run(vi, bi).float().mean())
           for vi in range(len(SBRS)) for bi in range(len(BETAS))}
    p_fa = {}
    gen = torch.Generator(device=dev).manual_seed(SEED + 7)
    for vi, sbr in enumerate(SBRS):
        b = float(sc.signal[0].mean()) / (sbr * T)
        zbg = synth.pitched(synth.poisson_histograms(torch.full((P, T), b, device=dev), gen).reshape(P, T),
                            synth.pad_pitch(T))
        for bi, prm in enumerate(prms):
            mu, var = states[vi][bi]
            o = spl.spl_filter_step_detect(prm, zbg, hd, mu[frames & 1], var[frames & 1], stream=stream)
            p_fa[f"SBR {sbr} beta {BETAS[bi]}"] = float(o["present"].float().mean())
    ms_plain = timed(lambda: run_job(spl, prms, hd, videos, states, outs, stream, lanes=plain_lanes))
    # roofline of one detect step (tensor-core depth launch + redo scan + detecting intensity launch + pi
    # propagation): uint16 row (2 T) + previous state (8 B) + present_in (1 B) + pi0 (4 B) + outputs mu, var, argmax,
    # refl, bg, pi, present (25 B) + the propagation's pi read and pi0 write (8 B) per pixel; time per step = job
    # time / steps
    roofline = hbm_roofline(_peaks(), P * (2 * T + 46), ms_det / 1e3 / (len(SBRS) * len(BETAS) * frames), None,
                            "k_filter_tc<u16> + k_estimate_redo + k_intensity4<detect> + k_pi_propagate (one frame)",
                            note="traffic not captured for this workload")
    line = {"metric": "pixel-frames/s", "value": units / (ms_det / 1e3), "unit": "pixel-frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_det, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u16 counts -> f16 on chip (exact below 1024) x f16 hi/lo taps -> f32 (tensor); f32 epilogue",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + ", presence decided on the device (detection surrogate)",
                       "pixels": P, "frames": frames, "pixel_frames_per_step": units},
            "plain_path": {"value": units / (ms_plain / 1e3), "ms_per_step": ms_plain,
                           "detection_overhead": ms_det / ms_plain - 1.0},
            "detection_rate_last_frame": p_d, "false_alarm_rate_background_frame": p_fa,
            "gpu_launches": launches, "clocks": clk.summary(), "roofline": roofline, "e2e": None}
    print(json.dumps(line), flush=True)


def fine(args):
    """Sub-bin depth (spl_depth_estimate_fine): single-frame estimates of the video frames (SBR 1 sequence, beta
    0.5, uniform prior) on the fine grid with S = 1, 2, 4, 8 steps per bin, beside spl_depth_estimate on the
    integer grid. Throughput in pixel-estimates/s per S."""
    import paper_2004_09211_gb300 as spl
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    frames = min(args.frames, 4)
    h, peak, hd, sc, videos = make_sequences(frames, dev)
    P = H * W
    prm = spl.make_params(H, W, T, L, peak, beta=0.5)
    zs = videos[SBRS.index(1.0)]

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            for z in zs:
                fn(z)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            for z in zs:
                fn(z)
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / (args.steps * len(zs))

    res = {}
    with ClockSampler(0) as clk:
        ms_int = timed(lambda z: spl.spl_depth_estimate(prm, z, hd, intensity=False))
        for S in (1, 2, 4, 8):
            ms = timed(lambda z: spl.spl_depth_estimate_fine(prm, S, z, hd))
            res[f"S={S}"] = {"ms_per_frame": ms, "pixel_estimates_per_s": P / (ms / 1e3),
                             "candidates_per_pixel": (prm.dmax - prm.dmin) * S + 1}
    # roofline of k_estimate_fine at S = 4: algorithmic bytes per launch = the uint16 row (2 T) + argmax_k, mu,
    # var (12 B) per pixel (the uniform prior reads nothing)
    peaks = _peaks()
    launch_s = res["S=4"]["ms_per_frame"] / 1e3
    roofline = hbm_roofline(peaks, P * (2 * T + 12), launch_s, None, "k_estimate_fine<u16> (S = 4, one frame)",
                            note="traffic not captured for this workload; every one of the 4 (D - 1) + 1 "
                                 "candidates is evaluated exactly (no pruning)")
    line = {"metric": "pixel-estimates/s", "value": res["S=4"]["pixel_estimates_per_s"],
            "unit": "pixel-estimates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["S=4"]["ms_per_frame"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sub-bin single-frame estimate, S = 4, video frames 256x256, T=1500, SBR 1, "
                                   "beta 0.5, uniform prior", "frames": frames},
            "by_S": res, "integer_grid": {"ms_per_frame": ms_int, "pixel_estimates_per_s": P / (ms_int / 1e3)},
            "gpu_launches": (4 + 1) * args.steps * len(zs), "clocks": clk.summary(), "roofline": roofline,
            "e2e": None}
    print(json.dumps(line), flush=True)


PD_T, PD_FWHM, PD_PRIOR_MU, PD_PRIOR_VAR, PD_ETA, PD_NMC = 1500, 28.0, 600.0, 2500.0, 28.0, 2000
PD_BETAS = (0.1, 0.3, 0.5, 0.7, 0.9)


def pd_inputs(sbr, msc, n_mc, seed, device):
    """The single-pixel experiment of Sec. IV-A with the Gaussian IRF (FWHM 28 bins, taps +-4 sigma, unit sum):
    n_mc histograms per (SBR, MSC) cell, depth drawn from N(600, 2500) and rounded to the bin grid (kept inside
    the full-support range), z ~ Poisson(MSC s_d + MSC / (SBR T)) (Eq. lik_bg_poisson). Returns (h, peak,
    depth [cells * n_mc] int, z [cells * n_mc, pitch] uint16) with cells = len(sbr) * len(msc), SBR fastest."""
    from paper_2004_09211_gb300 import synth
    sigma = PD_FWHM / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    h, peak = synth.gaussian_irf(sigma, int(math.ceil(4 * sigma)))
    hd = torch.from_numpy(h).to(device)
    gen = torch.Generator(device=device).manual_seed(seed)
    pitch = synth.pad_pitch(PD_T)
    lo, hi = peak, PD_T - len(h) + peak
    depth, zs = [], []
    for m in msc:
        d = torch.randn(len(sbr) * n_mc, generator=gen, device=device) * math.sqrt(PD_PRIOR_VAR) + PD_PRIOR_MU
        d = d.round().clamp(lo, hi).to(torch.int64)
        b = torch.tensor([m / (s * PD_T) for s in sbr], device=device).repeat_interleave(n_mc)
        mean = synth.expected_counts(d, torch.full_like(b, m), b, hd, peak, PD_T)
        zs.append(synth.pitched(synth.poisson_histograms(mean, gen), pitch))
        depth.append(d)
        del mean
    return h, peak, torch.cat(depth), torch.cat(zs)


def pd_curves(args):
    """Curves of satisfactory detection (Sec. IV-A, Fig. MMSE_synth, Gaussian-IRF half, the PB estimator only):
    p_d = fraction of |d_hat - d| < 28 with d_hat the pseudo-posterior mean under the prior N(600, 2500), over a
    25 x 13 grid of SBR in [1e-4, 1e2] and mean signal count in [10, 1000], 2000 histograms per cell, for five
    values of beta. Reports, per beta and MSC, the smallest SBR on the grid from which p_d >= 0.85, and the
    estimate throughput (one spl_depth_estimate launch over all cells per beta)."""
    import paper_2004_09211_gb300 as spl
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    sbr = np.logspace(-4, 2, 25)
    msc = np.logspace(1, 3, 13)
    h, peak, depth, z = pd_inputs(sbr, msc, PD_NMC, SEED + 11, dev)
    hd = torch.from_numpy(h).to(dev)
    P = z.shape[0]
    W_ = 1000
    assert P % W_ == 0
    pm = torch.full((P,), PD_PRIOR_MU, device=dev)
    pv = torch.full((P,), PD_PRIOR_VAR, device=dev)
    out = {}
    ms_all = []
    with ClockSampler(0) as clk:
        for beta in PD_BETAS:
            prm = spl.make_params(P // W_, W_, PD_T, len(h), peak, beta=beta)
            o = dict(mu=torch.empty(P, device=dev), var=torch.empty(P, device=dev),
                     argmax=torch.empty(P, dtype=torch.int32, device=dev))
            for _ in range(max(args.warmup, 1)):
                spl.spl_depth_estimate(prm, z, hd, pm, pv, intensity=False, out=o)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                spl.spl_depth_estimate(prm, z, hd, pm, pv, intensity=False, out=o)
            e1.record()
            torch.cuda.synchronize(dev)
            ms_all.append(e0.elapsed_time(e1) / args.steps)
            ok = ((o["mu"] - depth.float()).abs() < PD_ETA).float().view(len(msc), len(sbr), PD_NMC).mean(-1).cpu()
            limit = {}
            for i, m in enumerate(msc):
                good = [j for j in range(len(sbr)) if bool((ok[i, j:] >= 0.85).all())]
                limit[f"{m:.4g}"] = float(sbr[good[0]]) if good else None
            out[f"beta {beta}"] = {"limiting_sbr_by_msc": limit, "pd_grid": ok.numpy().round(4).tolist()}
    ms = sum(ms_all)
    # roofline of k_estimate on this workload: algorithmic bytes per launch = the uint16 row (2 T) + the Gaussian
    # prior (8 B) + mu, var, argmax (12 B) per pixel; average launch time over the five betas' launches
    peaks = _peaks()
    launch_s = ms / len(PD_BETAS) / 1e3
    roofline = hbm_roofline(peaks, P * (2 * PD_T + 8 + 12), launch_s, None,
                            "k_filter_tc<u16> + k_estimate_redo (one spl_depth_estimate over all cells of one beta)",
                            note="traffic not captured for this workload")
    line = {"metric": "pixel-estimates/s", "value": P * len(PD_BETAS) / (ms / 1e3), "unit": "pixel-estimates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u16 counts -> f16 on chip (exact below 1024) x f16 hi/lo taps -> f32 (tensor); f32 epilogue",
            "data": "synthetic",
            "config": {"workload": "single-pixel p_d experiment (Sec. IV-A, Gaussian IRF FWHM 28, T=1500, prior "
                                   "N(600, 2500), eta 28): 25 SBR x 13 MSC x 2000 histograms per beta",
                       "sbr_grid": sbr.tolist(), "msc_grid": msc.tolist(), "betas": list(PD_BETAS), "pixels": P},
            # per call: the tensor-core depth launch and the redo scan (no intensity)
            "curves": out, "gpu_launches": 2 * len(PD_BETAS) * args.steps, "clocks": clk.summary(),
            "roofline": roofline, "e2e": None}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------------
# mixed precision: the filter step with the data term on the tensor cores
# ---------------------------------------------------------------------------------------------------------

MIX_HW, MIX_FRAMES, MIX_T, MIX_L, MIX_SBR, MIX_SEED = 1024, 20, 4096, 64, 0.05, 3
MIX_CROP, MIX_CROP_FRAMES = 48, 2


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def mixed(args):
    """Mixed precision: 1024 x 1024 pixels x 20 frames, T = 4096, the asymmetric IRF stretched to 64 taps, the
    video scene generator (1-5 signal photons per pixel-frame) at SBR 0.05 (about 60 background photons per
    pixel-frame), beta = 0.5, FP16 counts (exact up to 2048). One step = the 20 frames through
    spl_filter_step_tc. Every frame is generated on the device (seeded per frame) before its filter step; CUDA
    events bracket each step and the step time is their sum, so generation is outside the timed region (each
    frame is 8.6 GB, far larger than L2). Also measured: spl_filter_step_fp32 (FP32 CUDA cores) on the same FP16
    frames, the depth RMSE of both against the ground truth, the tensor-core data term against an FP64
    evaluation of its definition on a crop, and (CPU baseline leg) the FP64 oracle on crops with the
    tensor-core filter's depths compared to it."""
    import paper_2004_09211_gb300 as spl
    from paper_2004_09211_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    Hm = Wm = args.side or MIX_HW
    N = args.frames if args.frames != N_FRAMES else MIX_FRAMES
    Tm, Lm = MIX_T, MIX_L
    P = Hm * Wm
    h, peak = synth.stretched_irf(synth.asymmetric_irf(L=48)[0], Lm)
    sc = synth.moving_scene(Hm, Wm, N, peak + 8, Tm - Lm + peak - 8, MIX_SEED)
    hd = torch.from_numpy(h).to(dev)
    pitch = synth.pad_pitch(Tm)
    prm = spl.make_params(Hm, Wm, Tm, Lm, peak, beta=0.5, sigma_rw2=SIGMA_RW2)
    depth = [torch.from_numpy(sc.depth[n]).to(dev) for n in range(N)]
    signal = [torch.from_numpy(sc.signal[n]).to(dev) for n in range(N)]
    bgs = [float(sc.signal[n].mean()) / (MIX_SBR * Tm) for n in range(N)]
    gen = torch.Generator(device=dev)
    zbuf = torch.zeros(P, pitch, dtype=torch.float16, device=dev)

    def gen_frame(n):
        gen.manual_seed(MIX_SEED * 1000 + n)
        synth.frame_histograms(depth[n], signal[n], bgs[n], hd, peak, Tm, gen, pitch, out=zbuf)

    mu = [torch.empty(P, device=dev) for _ in range(2)]
    var = [torch.empty(P, device=dev) for _ in range(2)]
    outs = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), refl=torch.empty(P, device=dev),
                bg=torch.empty(P, device=dev))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    split = {}

    def run(step_fn):
        """The 20-frame sequence; returns (summed step ms, per-frame depth RMSE against the ground truth); the last
        frame's split RMSE goes to split[step_fn]."""
        spl.spl_state_init(prm, mu[0], var[0])
        total, rmse = 0.0, []
        for n in range(N):
            gen_frame(n)
            src, dst = n & 1, (n + 1) & 1
            e0.record()
            step_fn(prm, zbuf, hd, mu[src], var[src], out=dict(mu=mu[dst], var=var[dst], **outs))
            e1.record()
            torch.cuda.synchronize(dev)
            total += e0.elapsed_time(e1)
            rmse.append(float(((mu[dst] - depth[n].reshape(-1).float()) ** 2).mean().sqrt()))
        split[step_fn] = depth_rmse(outs["argmax"].cpu().numpy(), mu[N & 1].cpu().numpy(), sc, N - 1)
        return total, rmse

    for _ in range(args.warmup):
        run(spl.spl_filter_step_tc)
    with ClockSampler(0) as clk:
        runs = [run(spl.spl_filter_step_tc) for _ in range(args.steps)]
    ms = statistics.mean(r[0] for r in runs)
    rmse_tc = runs[-1][1]
    flags = spl.spl_tc_status()
    ms_fp32, rmse_fp32 = run(spl.spl_filter_step_fp32)

    # data term against an FP64 evaluation of its definition (C(d) = sum_j h_j^beta z[d - peak + j]) on a crop
    gen_frame(0)
    cz = 32
    crop = zbuf.reshape(Hm, Wm, pitch)[:cz, :cz, :].contiguous().reshape(cz * cz, pitch)
    pc = spl.make_params(cz, cz, Tm, Lm, peak, beta=0.5, sigma_rw2=SIGMA_RW2)
    ctc, _ = spl.spl_depth_cost_tc(pc, crop, hd)
    g64 = torch.where(hd > 0, hd.double().clamp(min=1e-300) ** 0.5, torch.zeros_like(hd, dtype=torch.float64))
    win = crop[:, :Tm].double().unfold(1, Lm, 1)[:, pc.dmin - peak:pc.dmax - peak + 1, :]
    cref = win @ g64
    cerr = (ctc.double() - cref).abs()
    cost_error = {"max_abs_over_max_C": float(cerr.max() / cref.max()),
                  "rms_rel": float(((cerr / cref.clamp(min=1e-30)) ** 2).mean().sqrt()),
                  "crop": f"{cz}x{cz} pixels of frame 0, all {pc.dmax - pc.dmin + 1} candidates"}

    # roofline of the fused kernel: algorithmic bytes = FP16 row + previous state + outputs per pixel-frame;
    # tensor work = the issued MMAs (hi and lo Toeplitz tiles, count MMAs)
    peaks = _peaks()
    kw = ((64 + Lm - 1) + 15) & ~15
    ntiles = (prm.dmax - prm.dmin + 1 + 63) // 64
    npt = (P + 127) // 128
    slabs = max(ntiles + (kw + 63) // 64 - 1, (Tm + 63) // 64)
    flops = npt * (ntiles * 2 * (2 * 128 * 64 * kw) + slabs * 2 * 128 * 16 * 64)
    frame_s = ms / N / 1e3
    alg_bytes = P * (2 * Tm + 8 + 20)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    roofline = {"bound": "hbm", "achieved": alg_bytes / frame_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": alg_bytes / frame_s / 1e9 / hbm_peak, "traffic": capture_traffic("k_filter_tc", P),
                "kernel": "k_filter_tc + k_intensity4 (one spl_filter_step_tc, timed as a whole)",
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": frame_s * 1e3,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s",
                "tensor": {"achieved": flops / frame_s / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                           "frac": flops / frame_s / 1e12 / tc_peak, "flops_per_launch": flops,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops (FP16 runs at the BF16 rate)"},
                "note": "epilogue-bound on this workload: broad posteriors leave nothing to prune, so every "
                        "candidate's mixture prior is evaluated"}

    cpu = None
    if not args.no_cpu:
        cpu = mixed_cpu_baseline(spl, synth, h, hd, peak, sc, dev)

    rt, rf = statistics.mean(rmse_tc), statistics.mean(rmse_fp32)
    inst = capture_traffic("k_filter_tc", P, "inst_per_pixel")
    if inst is not None:
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        issue_peak = MEASURED_WARP_ISSUE_PER_CLK_SM * nsm * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
        roofline["issue"] = {"achieved": inst / frame_s, "peak": issue_peak, "unit": "warp-instructions/s",
                             "frac": inst / frame_s / issue_peak, "inst_per_step": inst,
                             "source": "ncu smsp__inst_executed.sum of one 256 x 256 step, scaled by the pixels"}
    line = {"metric": "pixel-frames/s", "value": P * N / (ms / 1e3), "unit": "pixel-frames/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 x f16 -> f32 (tensor), f32 epilogue",
            "data": "synthetic",
            "config": {"workload": f"mixed precision {Hm}x{Wm}x{N} frames, T=4096, 64-tap IRF, SBR 0.05, FP16 counts",
                       "pixels": P, "frames": N, "T": Tm, "L": Lm, "beta": 0.5,
                       "l2": "inputs larger than L2 (8.6 GB per frame), generated between timed steps"},
            "fp32_path": {"value": P * N / (ms_fp32 / 1e3), "ms_per_step": ms_fp32,
                          "speedup_tc_over_fp32": ms_fp32 / ms},
            "depth_rmse_bins": {"tc_mean_over_frames": rt, "fp32_mean_over_frames": rf,
                                "tc_last_frame": rmse_tc[-1], "fp32_last_frame": rmse_fp32[-1],
                                "equal": abs(rt - rf) <= max(0.01, 0.01 * rf),
                                "last_frame_split": {"tc": split[spl.spl_filter_step_tc],
                                                     "fp32": split[spl.spl_filter_step_fp32]}},
            "cost_error_vs_fp64": cost_error, "status_flags": flags, "roofline": roofline,
            "gpu_launches": 2 * N * args.steps, "clocks": clk.summary(), "cpu_baseline": cpu, "e2e": None}
    print(json.dumps(line), flush=True)


def mixed_cpu_baseline(spl, synth, h, hd, peak, sc, dev):
    """The FP64 oracle on a MIX_CROP x MIX_CROP crop of the mixed workload for MIX_CROP_FRAMES frames (host
    cores, timed), and the tensor-core filter on the same crop as its own image, compared with it."""
    from oracle import oracle as orc
    c = MIX_CROP
    pitch = synth.pad_pitch(MIX_T)
    gen = torch.Generator(device=dev)
    zs = []
    for n in range(MIX_CROP_FRAMES):
        gen.manual_seed(MIX_SEED * 7000 + n)
        zs.append(synth.frame_histograms(torch.from_numpy(sc.depth[n][:c, :c].copy()).to(dev),
                                         torch.from_numpy(sc.signal[n][:c, :c].copy()).to(dev),
                                         float(sc.signal[n].mean()) / (MIX_SBR * MIX_T), hd, peak, MIX_T, gen, pitch))
    q = orc.params(MIX_T, MIX_L, peak, beta=0.5, sigma_rw2=SIGMA_RW2, nu=synth.cross_weights(0.5))
    threads = orc.set_threads(os.cpu_count() or 1)
    m, v = orc.state_init(q, c, c)
    t0 = time.perf_counter()
    for z in zs:
        e = orc.filter_step(q, h, z[:, :MIX_T].double().cpu().numpy().reshape(c, c, MIX_T), m, v)
        m, v = e["mu"], e["var"]
    dt = time.perf_counter() - t0
    prm = spl.make_params(c, c, MIX_T, MIX_L, peak, beta=0.5, sigma_rw2=SIGMA_RW2)
    mu, var = spl.spl_state_init(prm)
    for z in zs:
        o = spl.spl_filter_step_tc(prm, z, hd, mu, var)
        mu, var = o["mu"], o["var"]
    d = mu.double().cpu().numpy().reshape(c, c) - m
    return {"value": c * c * MIX_CROP_FRAMES / dt, "unit": "pixel-frames/s", "cores": threads, "kind": "oracle",
            "sample": f"{c}x{c} crop x {MIX_CROP_FRAMES} frames of the mixed workload (T={MIX_T}, L={MIX_L})",
            "tc_vs_fp64_depth": {"rms_bins": float(np.sqrt((d ** 2).mean())), "max_abs_bins": float(np.abs(d).max()),
                                 "max_rel": float((np.abs(d) / np.abs(m)).max())}}


MSL_BANDS, MSL_SEED, MSL_SBR = 4, 7, 0.2


def msl(args):
    """Multispectral estimate (Appendix, Eq. div_MSL): 256 x 256 pixels, 4 bands, T = 1500, 48-tap band IRFs of
    different widths and tails (maxima aligned), beta = 0.5, the video scene's first frame (tilted plane + 3
    objects), 5-25 signal photons per pixel in each band (the video scene's 1-5, times 5, times per-band gains 0.8-1.2)
    and the same SBR, 0.2, in every band (the paper's multispectral experiment uses the same SBR and signal level in
    all bands; at this photon level one band alone often misses the surface). One step = one
    spl_depth_estimate_msl launch over the frame, without a prior (the minimum-divergence estimate of the paper's
    multispectral experiment); the histograms (4 x 197 MB) stay resident. Also reported: the depth RMSE of the
    4-band estimate and of band 0 alone (spl_depth_estimate) against the ground truth."""
    import paper_2004_09211_gb300 as spl
    from paper_2004_09211_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    nb, peak = MSL_BANDS, 12
    hb = synth.band_irfs(nb, L, peak)
    sc = synth.moving_scene(H, W, 1, peak + 8, T - L + peak - 8, MSL_SEED)
    gen = torch.Generator(device=dev).manual_seed(MSL_SEED)
    pitch = synth.pad_pitch(T)
    P = H * W
    gains = (0.8, 1.0, 1.2, 0.9)
    z = torch.empty(nb, P, pitch, dtype=torch.uint16, device=dev)
    depth = torch.from_numpy(sc.depth[0]).to(dev)
    for b in range(nb):
        sig = torch.from_numpy(sc.signal[0]).to(dev) * (5.0 * gains[b])
        mean = synth.expected_counts(depth, sig, float(sig.mean()) / (MSL_SBR * T), torch.from_numpy(hb[b]).to(dev),
                                     peak, T)
        z[b] = synth.pitched(synth.poisson_histograms(mean, gen).reshape(P, T), pitch)
    hd = torch.from_numpy(hb).to(dev)
    prm = spl.make_params(H, W, T, L, peak, beta=0.5)
    out = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), mu=torch.empty(P, device=dev),
               var=torch.empty(P, device=dev))
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        spl.spl_depth_estimate_msl(prm, z, hd, out=out)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            spl.spl_depth_estimate_msl(prm, z, hd, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    gt = depth.reshape(-1).float()
    rmse = float((out["argmax"].float() - gt).pow(2).mean().sqrt())
    one = spl.spl_depth_estimate(prm, z[0].contiguous(), hd[0].contiguous())
    torch.cuda.synchronize(dev)
    rmse1 = float((one["argmax"].float() - gt).pow(2).mean().sqrt())
    peaks = _peaks()
    alg = P * (nb * 2 * T + 12)
    line = {"metric": "pixel-estimates/s", "value": P / (ms / 1e3), "unit": "pixel-estimates/s (4 bands each)",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"multispectral {H}x{W}, {nb} bands, T={T}, L={L}, 5-25 signal photons, "
                                   f"SBR {MSL_SBR}, beta 0.5, no prior",
                       "pixels": P, "bands": nb, "l2": f"inputs larger than L2 ({nb} x 197 MB), no flush"},
            "rmse_bins": {"msl_argmax": rmse, "band0_alone_argmax": rmse1},
            "roofline": hbm_roofline(peaks, alg, ms / 1e3, None, "k_estimate_msl<u16> (one launch)"),
            "gpu_launches": args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def single(args):
    """The single-frame workload: 32 x 32 pixels, T = 1024, Gaussian IRF (sigma 3 bins, taps -12..12), depth = a
    smooth random surface (4 Gaussians) in bins 100-900, Poisson signal mean 10 at the template plus a uniform
    background of mean 50 over the histogram, beta = 0.5, uint16, no prior (the minimum-divergence estimate and its
    pseudo-posterior moments), with the intensity estimate. 2 MB of input sits in L2: the figure is the absolute
    time of one spl_depth_estimate call (a depth launch and an intensity launch), back to back. The FP64 oracle runs
    the same frame in full on the host cores, and every pixel is compared with it."""
    import paper_2004_09211_gb300 as spl
    from paper_2004_09211_gb300 import synth
    from oracle import oracle as orc
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    spl.load_library()
    Hs = Ws = 32
    Ts = 1024
    h, peak = synth.gaussian_irf(3.0, 12)
    Ls = len(h)
    depth = synth.smooth_depth_map(Hs, Ws, 100, 900, 1)
    g = torch.Generator().manual_seed(1)
    mean = synth.expected_counts(torch.from_numpy(depth), torch.full((Hs, Ws), 10.0, dtype=torch.float64), 50.0 / Ts,
                                 torch.from_numpy(h), peak, Ts)
    z = torch.poisson(mean, generator=g)
    zd = synth.pitched(z.reshape(-1, Ts).to(torch.int32).to(torch.uint16), synth.pad_pitch(Ts)).to(dev)
    hd = torch.from_numpy(h).to(dev)
    P = Hs * Ws
    prm = spl.make_params(Hs, Ws, Ts, Ls, peak, beta=0.5)
    out = dict(argmax=torch.empty(P, dtype=torch.int32, device=dev), mu=torch.empty(P, device=dev),
               var=torch.empty(P, device=dev), refl=torch.empty(P, device=dev), bg=torch.empty(P, device=dev))
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        spl.spl_depth_estimate(prm, zd, hd, out=out)
    torch.cuda.synchronize(dev)
    # 100 calls captured in one CUDA graph (the device time of the calls, without the host's per-call cost), and
    # the same calls issued eagerly from the host
    G = 100
    gs_ = torch.cuda.Stream(dev)
    gs_.wait_stream(stream)
    with torch.cuda.stream(gs_):
        spl.spl_depth_estimate(prm, zd, hd, out=out, stream=gs_)
    stream.wait_stream(gs_)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(G):
            spl.spl_depth_estimate(prm, zd, hd, out=out)
    graph.replay()
    torch.cuda.synchronize(dev)
    steps = max(args.steps, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(steps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    reps = steps * G
    ms = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for _ in range(reps):
        spl.spl_depth_estimate(prm, zd, hd, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_eager = e0.elapsed_time(e1) / reps
    # the oracle on the same frame, in full (every host core), and every pixel compared
    q = orc.params(Ts, Ls, peak, beta=0.5)
    zh = z.numpy().astype(np.float64)
    cores = orc.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    e = orc.estimate(q, h, zh)
    r_o, b_o = orc.intensity(q, h, zh, e["mu"])
    dt = time.perf_counter() - t0
    one = orc.set_threads(1)
    t1 = time.perf_counter()
    orc.estimate(q, h, zh)
    orc.intensity(q, h, zh, e["mu"])
    dt1 = time.perf_counter() - t1
    orc.set_threads(cores)
    mu = out["mu"].cpu().numpy().reshape(Hs, Ws).astype(np.float64)
    am = out["argmax"].cpu().numpy().reshape(Hs, Ws)
    gt = depth.astype(np.float64)
    line = {"metric": "ms per frame", "value": ms, "unit": "ms", "n_gpus": 1, "steps": reps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "single frame 32x32, T=1024, Gaussian IRF sigma 3 (25 taps), signal 10, "
                                   "background 50, beta 0.5, uint16, no prior", "pixels": P,
                       "l2": "input L2-resident (2 MB): launch-latency bound"},
            "pixel_frames_per_s": P / (ms / 1e3), "eager_ms_per_frame": ms_eager,
            "timing": "100 calls per CUDA graph replay; eager_ms_per_frame: the same calls issued from the host",
            "depth_rmse_bins": {"argmax": float(np.sqrt(np.mean((am - gt) ** 2))),
                                "mu": float(np.sqrt(np.mean((mu - gt) ** 2)))},
            "vs_oracle": {"pixels": P, "argmax_equal_frac": float(np.mean(am == e["argmax"])),
                          "max_rel_mu": float(np.max(np.abs(mu - e["mu"]) / np.abs(e["mu"]))),
                          "max_rel_var": float(np.max(np.abs(out["var"].cpu().numpy().reshape(Hs, Ws) - e["var"]) /
                                                      np.maximum(np.abs(e["var"]), 1e-6)))},
            "cpu_baseline": {"value": dt * 1e3, "unit": "ms per frame", "cores": cores, "kind": "oracle",
                             "sample": "the whole frame (estimate + intensity, FP64)",
                             "single_thread": {"value": dt1 * 1e3, "unit": "ms per frame", "cores": one}},
            "gpu_launches": 2 * reps, "clocks": clk.summary(), "e2e": None}
    print(json.dumps(line), flush=True)


def alu_peaks(args):
    """Measured arithmetic throughput of this GPU: FFMA, packed f32x2 FMA and MUFU ex2 (spl_probe_throughput),
    as operations per clock per SM (from the blocks' own clock64 counts) and per second (CUDA events), at 4 and 8
    resident blocks of 256 threads per SM, under the sampled clocks. Prints one JSON line."""
    import ctypes as ct
    from paper_2004_09211_gb300 import _abi
    lib = _abi.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    kinds = {"ffma": 0, "ffma2": 1, "ex2": 2}
    iters = {"ffma": 4096, "ffma2": 2048, "ex2": 1024}
    out = {}
    with ClockSampler(dev.index or 0) as clk:
        for name, kind in kinds.items():
            for bps in (4, 8):
                nb, opt = ct.c_int(0), ct.c_longlong(0)
                _abi.check(lib.spl_probe_throughput(kind, bps, iters[name], None, None, ct.byref(nb), ct.byref(opt),
                                                    None))
                sink = torch.empty(nb.value * 256, device=dev)
                cyc = torch.zeros(nb.value, dtype=torch.int64, device=dev)
                res = []
                for rep in range(args.warmup + args.steps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize(dev)
                    e0.record(stream)
                    _abi.check(lib.spl_probe_throughput(kind, bps, iters[name], ct.c_void_p(sink.data_ptr()),
                                                        ct.c_void_p(cyc.data_ptr()), ct.byref(nb), ct.byref(opt),
                                                        ct.c_void_p(stream.cuda_stream)))
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    if rep >= args.warmup:
                        ops = float(nb.value) * 256 * opt.value
                        cy = cyc.double()
                        res.append({"ops_per_s": ops / (e0.elapsed_time(e1) / 1e3),
                                    "ops_per_clk_sm": ops / nsm / float(cy.mean()),
                                    "cycles_spread": float(cy.max() / cy.min())})
                best = max(res, key=lambda r: r["ops_per_s"])
                out[f"{name}_bps{bps}"] = {"ops_per_s_best": best["ops_per_s"],
                                           "per_block_clock64_ops_per_clk_sm":
                                               round(statistics.median(r["ops_per_clk_sm"] for r in res), 2)}
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz") or float(_peaks().get("sm_max_mhz", 2070.0))
    for v in out.values():  # per clock per SM at the SM clock sampled during the runs
        v["ops_per_clk_sm"] = round(v["ops_per_s_best"] / nsm / (mhz * 1e6), 2)
    line = {"metric": "arithmetic throughput (operations per clock per SM, per second)", "workload": "alu_peaks",
            "n_sm": nsm, "results": out, "clocks": clocks, "steps": args.steps, "warmup": args.warmup,
            "note": "an FMA counts as one operation (two flops); an f32x2 instruction as two operations; "
                    "ops_per_clk_sm divides the event-timed rate by the sampled SM clock (the per-block clock64 "
                    "figure counts each block's own cycles, which start and end at different times)"}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
    elif args.workload == "batched":
        batched(args)
    elif args.workload == "diff":
        diff(args)
    elif args.workload == "mixed":
        mixed(args)
    elif args.workload == "video_tc":
        video_tc(args)
    elif args.workload == "detect":
        detect(args)
    elif args.workload == "pd_curves":
        pd_curves(args)
    elif args.workload == "fine":
        fine(args)
    elif args.workload == "alu_peaks":
        alu_peaks(args)
    elif args.workload == "msl":
        msl(args)
    elif args.workload == "single":
        single(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
