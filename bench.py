#!/usr/bin/env python3
"""Throughput / latency benchmark of the cross-correlation tracking hot path.

Workload (frame stream): 10,000 uint16 128x128 frames of a Gaussian spot
(sigma 2.5 px, peak 2000 photons, background 20, Poisson noise) on a reflected
2-D Brownian trajectory (step 0.3 px), tracked against one noise-free reference
with u = 100, CC-U, in 256-frame batches (the last batch has 16 frames), one
CUDA-graph launch per batch. One step = one pass over the whole stream: its 40
batches (39 x 256 + 16), batch b on CUDA stream b mod 3. The stream (328 MB) is
larger than L2 and is staged in HBM before timing; each step reads all of it once.

Prints one JSON line: the contract keys (metric, value, unit, n_gpus, steps, warmup,
ms_per_step, config, roofline, cpu_baseline, e2e, clocks, gpu_launches), the headline's
latency percentiles and oracle parity, and one object per extra leg (plain per-frame
launch, latency under offered load, real-time, offline, uneven ROIs, serving, adjoint).
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 128
U = 100
N_FRAMES = 10_000
BATCH = 256
SM_COUNT = 148
FP32_LANES_PER_SM = 128          # FFMA lanes per SM (4 SMSPs x 32)
MAX_SM_MHZ = 2032.0
PROFILE_FILE = os.path.join(ROOT, "profiles", "track_kernel_128x128_u100.txt")
KERNEL_SOURCES = ["paper_2310_08770_b300/csrc/ccst_kernels.cuh", "paper_2310_08770_b300/csrc/ccst_device.cuh",
                  "paper_2310_08770_b300/csrc/ccst_dfloat.cuh", "paper_2310_08770_b300/csrc/ccst_fft.cuh",
                  "paper_2310_08770_b300/csrc/ccst_tc.cuh", "paper_2310_08770_b300/csrc/ccst_track_h128.cu"]


def grid_size(u):
    return (3 * u + 1) // 2


def flop_per_frame(h=H, w=W, u=U):
    """Algorithmic FP32 flops of one frame in the folded formulation the kernel computes:
    the contraction exploits the Hermitian symmetry of the real-input spectrum in both
    stages (ky folded into P/Q planes, +-t and +-tx pairs from one product)."""
    m = grid_size(u)
    h0 = m // 2
    wc = w // 2 + 1
    fft = 2 * 2.5 * h * w * math.log2(h * w)           # R2C forward + C2R inverse
    product = 6 * h * wc                                 # X = F[a] conj F[b]
    stage_a = h0 * wc * (h // 2) * 8                     # U', V: 4 FMA per (t, kx, m)
    stage_b = m * m * wc * 2                             # one FMA per (grid point, kx)
    g_row = (h0 + 1) * wc * 4
    return fft + product + stage_a + stage_b + g_row


def scope_flop_per_frame(h=H, w=W, u=U):
    """Algorithmic flops of one frame as the scope table counts them (real input and
    output, Hermitian half in kx only): the two FFTs, the product and the integer-peak
    phase (6 flop per half-spectrum bin each), stage A as a complex contraction over all
    H rows (8 flop per (grid row, ky, kx)) and stage B over the half spectrum (4 flop per
    (grid point, kx)). 17.1 MFLOP at 128 x 128, u = 100."""
    m = grid_size(u)
    wc = w // 2 + 1
    fft = 2 * 2.5 * h * w * math.log2(h * w)
    return fft + 12 * h * wc + 8 * m * h * wc + 4 * m * m * wc


def scope_contraction_flop(h=H, w=W, u=U):
    """The upsampled-DFT contraction's share of scope_flop_per_frame (stages A and B)."""
    m = grid_size(u)
    wc = w // 2 + 1
    return 8 * m * h * wc + 4 * m * m * wc


def kernel_source_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel."""
    try:
        with open(PROFILE_FILE) as f:
            kv = dict(line.split(":", 1) for line in f if ":" in line and not line.startswith("#"))
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        if kv.get("kernel_source_hash") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch_full_batch"])
    except (OSError, KeyError, ValueError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        mx = np.array([num(r[2]) for r in rows])
        pw = np.array([num(r[3]) for r in rows])
        load = pw >= np.nanmax(pw) * 0.6 if np.isfinite(pw).any() else np.ones_like(sm, bool)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.nanmedian(sm[load])), "sm_max_mhz": float(np.nanmax(mx)),
                "power_w_max": float(np.nanmax(pw)), "samples": int(len(rows)), "reasons": reasons}


# ---------------------------------------------------------------- distributed plumbing
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_seed(rank: int) -> int:
    """Each rank tracks its own independent stream (weak scaling); rank 0 is the seed-0 workload."""
    return rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weighted_percentile(values, weights, q):
    order = np.argsort(values)
    v = np.asarray(values, float)[order]
    w = np.asarray(weights, float)[order]
    c = np.cumsum(w)
    return float(v[np.searchsorted(c, q / 100.0 * c[-1])])


# ---------------------------------------------------------------- CPU baseline (oracle)
def _oracle_chunk(args):
    import oracle
    frames, ref = args
    return oracle.track_batch(frames, ref, u=U)


def cpu_baseline(frames, ref, budget_s=15.0):
    """The FP64 oracle, as it stands, over all host cores on a bounded sample of the stream."""
    import multiprocessing as mp
    import oracle
    t0 = time.perf_counter()
    oracle.track_one(frames[0], ref, u=U)
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    n = int(min(len(frames), max(cores, budget_s * cores / max(t1, 1e-3))))
    n = max(1, min(n, 4096))
    ctx = mp.get_context("spawn")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_chunk, [(frames[:1], ref)] * cores)          # start-up outside the timing
        chunks = [(c, ref) for c in np.array_split(frames[:n], cores) if len(c)]
        t0 = time.perf_counter()
        parts = pool.map(_oracle_chunk, chunks)
        dt = time.perf_counter() - t0
    res = [r for p in parts for r in p]
    return res, {"value": n / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
                 "sample": f"first {n} frames of the 128x128 stream, FP64 numpy oracle, "
                           f"{cores} spawn workers with one BLAS thread each"}


WORKLOAD = ("frame stream: 10000 uint16 128x128 Gaussian-spot frames (sigma 2.5, peak 2000, bg 20, Poisson), "
            "Brownian trajectory step 0.3 px, u=100, CC-U, 256-frame CUDA-graph batches, consecutive batches on "
            "alternating streams")
RT_FRAMES = 1024                 # real-time leg: frames after frame 0
RT_A0 = 0.05                     # its filter, a0 = 1 - exp(-T/tau)
RT_ORACLE_FRAMES = 48


def realtime_leg(C, torch, s, stream, rt_frames=RT_FRAMES):
    """Real-time reference mode (Sec. III B): frames of the same stream tracked one after
    another, the reference updated after each (Eq. (9)). Throughput over one call of
    rt_frames frames; latency from one call per frame."""
    n = rt_frames + 1
    frames = torch.from_numpy(s.frames[:n].view(np.int16)).cuda().view(torch.uint16)
    t = C.Tracker(s.ref, upsample=U, method="ccu", in_dtype="u16", max_batch=1, stream=stream)
    out = t.empty_results(n - 1)
    ev = lambda: torch.cuda.Event(enable_timing=True)          # noqa: E731
    with torch.cuda.stream(stream):
        C.ccst_rt_begin(t.ctx, frames[0], 0, RT_A0, 1 - RT_A0)
        C.ccst_rt_track(t.ctx, frames[1:9], 8, 0, out[:8])       # warm-up
        torch.cuda.synchronize()
        C.ccst_rt_begin(t.ctx, frames[0], 0, RT_A0, 1 - RT_A0)
        e0, e1 = ev(), ev()
        e0.record(stream)
        C.ccst_rt_track(t.ctx, frames[1:], n - 1, 0, out)
        e1.record(stream)
        torch.cuda.synchronize()
        thr_ms = e0.elapsed_time(e1)
        res = C.decode(out)
        C.ccst_rt_begin(t.ctx, frames[0], 0, RT_A0, 1 - RT_A0)
        k = min(256, n - 1)
        starts, ends = [ev() for _ in range(k)], [ev() for _ in range(k)]
        for i in range(k):
            starts[i].record(stream)
            C.ccst_rt_track(t.ctx, frames[1 + i:2 + i], 1, 0, out[i:i + 1])
            ends[i].record(stream)
        torch.cuda.synchronize()
        lat_us = np.array([a.elapsed_time(b) * 1e3 for a, b in zip(starts, ends)])
    again = C.decode(out)[:k]
    t.close()
    return {"workload": f"frames 0..{n - 1} of the same stream, u={U}, CC-U, a0={RT_A0}, b1={1 - RT_A0}",
            "value": (n - 1) / (thr_ms / 1e3), "unit": "frames/s", "frames": n - 1,
            "p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
            "same_records_per_frame_calls": bool(again.tobytes() == res[:k].tobytes()),
            "gpu_launches_per_frame": 2, "memsets_per_call": 1}, res


def realtime_cpu_baseline(frames, res):
    """The FP64 real-time oracle, as it stands, on the first RT_ORACLE_FRAMES frames: its
    rate, and parity of the GPU records with it."""
    from oracle import rt_oracle
    t0 = time.perf_counter()
    orc = rt_oracle.rt_track(frames[:RT_ORACLE_FRAMES + 1].astype(np.float64), u=U, a0=RT_A0)
    dt = time.perf_counter() - t0
    mism = sum(1 for a, o in zip(res, orc)
               if (int(a["ipy"]), int(a["ipx"])) != (o["ipy"], o["ipx"])
               or abs(float(a["dx"]) - o["dx32"]) > 1e-3 or abs(float(a["dy"]) - o["dy32"]) > 1e-3)
    return ({"value": len(orc) / dt, "unit": "frames/s", "cores": 1, "kind": "oracle",
             "sample": f"first {len(orc)} frames after frame 0, FP64 numpy real-time oracle, one process"},
            {"frames": len(orc), "mismatches": mism, "tolerance_px": 1e-3})


OFF_PASSES = 5                   # offline leg: reference updates (the paper's fifth reference)
OFF_ORACLE_FRAMES = 32
FP64_PEAK_TFLOPS = 1.25          # nominal B300 FP64 rate (no measured figure on this machine)


def off_flop_per_frame(h=H, w=W):
    """FP64 flop of one frame's share of the Eq. (8) sum: a real 2-D FFT (2.5 HW log2 HW)
    plus the phase product and the accumulation over the half spectrum (8 per bin)."""
    return 2.5 * h * w * math.log2(h * w) + 8 * h * (w // 2 + 1)


def offline_leg(C, torch, s, frames_dev, n, stream):
    """Offline method (Sec. III A) over the whole stream: reference from frame 0, then
    OFF_PASSES rounds of track-all + Eq. (8) update, and a last track-all."""
    t = C.Tracker(s.ref, upsample=U, method="ccu", in_dtype="u16", max_batch=BATCH, stream=stream)
    out = t.empty_results(n)
    ev = lambda: torch.cuda.Event(enable_timing=True)          # noqa: E731
    with torch.cuda.stream(stream):
        C.ccst_offline_track(t.ctx, frames_dev, min(n, 1024), 0, 1, out[:min(n, 1024)])     # warm-up
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        C.ccst_offline_track(t.ctx, frames_dev, n, 0, OFF_PASSES, out)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms = e0.elapsed_time(e1)
        reps = 3
        u0, u1 = ev(), ev()
        u0.record(stream)
        for _ in range(reps):
            C.ccst_offline_update(t.ctx, frames_dev, n, 0, out)
        u1.record(stream)
        torch.cuda.synchronize()
        upd_ms = u0.elapsed_time(u1) / reps
    stale = C.ccst_reference_status(t.ctx)
    t.close()
    achieved = off_flop_per_frame() * n / (upd_ms / 1e3) / 1e12
    return {"workload": f"all {n} frames of the stream, u={U}, CC-U, reference from frame 0, {OFF_PASSES} Eq. (8) "
                        f"passes, {OFF_PASSES + 1} track-all passes",
            "value": n * (OFF_PASSES + 1) / (total_ms / 1e3), "unit": "frame-trackings/s",
            "ms_total": total_ms, "ms_per_pass": total_ms / (OFF_PASSES + 1), "update_ms": upd_ms,
            "update_share": OFF_PASSES * upd_ms / total_ms, "stale": stale,
            "roofline_update": {"bound": "fp64-equivalent", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                                "kernel": "off_accumulate + rt_update", "flop_per_frame": off_flop_per_frame(),
                                "peak_basis": "nominal B300 FP64 1.25 TFLOP/s (not measured); the transforms run "
                                              "in double-float on the FP32 pipes, so the FP64-equivalent rate is "
                                              "compared with what the FP64 pipe could give"}}


def offline_cpu_baseline(C, torch, s, stream):
    """The FP64 offline oracle, as it stands, on the first OFF_ORACLE_FRAMES frames with two
    passes: its rate, and parity of the GPU's last-pass records on the same sample."""
    from oracle import offline_oracle
    fr = s.frames[:OFF_ORACLE_FRAMES]
    t0 = time.perf_counter()
    ores, _ = offline_oracle.offline_track(fr.astype(np.float64), u=U, passes=2)
    dt = time.perf_counter() - t0
    t = C.Tracker(s.ref, upsample=U, method="ccu", in_dtype="u16", max_batch=BATCH, stream=stream)
    with torch.cuda.stream(stream):
        got = t.offline_track(torch.from_numpy(fr.view(np.int16)).cuda().view(torch.uint16), passes=2)
    t.close()
    mism = sum(1 for a, o in zip(got, ores[2])
               if (int(a["ipy"]), int(a["ipx"])) != (o["ipy"], o["ipx"])
               or abs(float(a["dx"]) - o["dx32"]) > 1e-3 or abs(float(a["dy"]) - o["dy32"]) > 1e-3)
    return ({"value": 3 * len(fr) / dt, "unit": "frame-trackings/s", "cores": 1, "kind": "oracle",
             "sample": f"first {len(fr)} frames, 2 Eq. (8) passes (3 track-all passes), FP64 numpy offline "
                       "oracle, one process"},
            {"frames": len(fr), "passes": 2, "mismatches": mism, "tolerance_px": 1e-3})


ADJ_PAIRS = 1024                 # adjoint leg: 64 x 64 FP32 pairs
ADJ_REPS = 20
ADJ_ORACLE_PAIRS = 32


def adj_flop_per_pair(h=64, w=64, newton_steps=4):
    """FP64 flop of one pair, forward + backward: three real 2-D transforms (the frame's
    spectrum in each pass, the complex-to-real return of dL/dI) at 2.5 HW log2 HW, and
    2 x newton_steps Newton steps at 16 flop per half-spectrum bin."""
    return 3 * 2.5 * h * w * math.log2(h * w) + 2 * newton_steps * 16 * h * (w // 2 + 1)


def adjoint_leg(C, torch, stream):
    """Continuous peak and its adjoint (ccst_peak_continuous, ccst_backward) over 1024 pairs:
    forward = tracking + Newton refinement, backward = the VJP into frames and reference."""
    from paper_2310_08770_b300 import synth
    p = synth.adjoint_pairs(seed=0, n=ADJ_PAIRS)
    n, H, W = p.frames.shape
    t = C.Tracker(p.ref, upsample=U, method="ccu", in_dtype="f32", max_batch=n, stream=stream)
    fr = torch.from_numpy(p.frames).cuda()
    rec = t.empty_results(n)
    peak = torch.empty((n, 2), dtype=torch.float64, device="cuda")
    status = torch.empty((n,), dtype=torch.int32, device="cuda")
    g = torch.ones((n, 2), dtype=torch.float32, device="cuda")
    gI = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    gE = torch.empty((H, W), dtype=torch.float32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)          # noqa: E731

    def fwd():
        C.ccst_track(t.ctx, fr, n, 0, rec)
        C.ccst_peak_continuous(t.ctx, fr, n, 0, rec, peak, status)

    def bwd():
        C.ccst_backward(t.ctx, fr, n, 0, rec, g, gI, gE)
    times = {}
    with torch.cuda.stream(stream):
        for _ in range(3):
            fwd()
            bwd()
        torch.cuda.synchronize()
        for name, fn in (("forward", fwd), ("backward", bwd)):
            a, b = ev(), ev()
            a.record(stream)
            for _ in range(ADJ_REPS):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            times[name] = a.elapsed_time(b) / ADJ_REPS
        bad = int((status != 0).sum().item())
        # Poisson-propagated spread of s* at the expected frames: sum_r (ds*/dI(r))^2 mu(r)
        mu = torch.from_numpy(p.mu).cuda()
        C.ccst_track(t.ctx, mu, n, 0, rec)
        sd = []
        for gv in ((1.0, 0.0), (0.0, 1.0)):
            g.copy_(torch.tensor(gv, dtype=torch.float32).expand(n, 2))
            C.ccst_backward(t.ctx, mu, n, 0, rec, g, gI, None)
            sd.append(torch.sqrt((gI.double() ** 2 * mu.double()).sum(dim=(1, 2))).cpu().numpy())
        torch.cuda.synchronize()
    t.close()
    flop = adj_flop_per_pair(H, W)
    achieved = flop * n / ((times["forward"] + times["backward"]) / 1e3) / 1e12
    return {"workload": f"{n} pairs, 64x64 FP32, noise-free reference (sigma 3, peak 1000, bg 10), Poisson frames "
                        "shifted uniformly in [-2, 2] px, u=100, CC-U; dL/dd = 1",
            "value": n / ((times["forward"] + times["backward"]) / 1e3), "unit": "pairs/s (forward + backward)",
            "forward_ms": times["forward"], "backward_ms": times["backward"], "status_nonzero": bad,
            "roofline": {"bound": "latency", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "flop_per_pair": flop,
                         "kernel": "adj_kernel (+ track_kernel in forward)",
                         "peak_basis": "nominal B300 FP64 1.25 TFLOP/s (not measured): the rate FP64-precision "
                                       "flops would have on the FP64 pipe; the kernel runs most of them as "
                                       "double-float on the FP32 pipes, so frac can exceed 1",
                         "bound_basis": "ncu: the FP64 pipe 36% busy, the first stall the barriers between the "
                                        "kernel's phases (profiles/adj_kernel_64x64_1024pairs.txt)"}}, (p, sd)


def adjoint_cpu_baseline(C, torch, stream, p, sd):
    """The FP64 adjoint oracle on the first ADJ_ORACLE_PAIRS pairs: its rate, parity of the
    GPU's s* and dL/dI there, and the propagated spread against the Cramer-Rao bound."""
    from oracle import adjoint_oracle, cc_oracle
    from paper_2310_08770_b300 import synth
    k = ADJ_ORACLE_PAIRS
    ref = p.ref.astype(np.float64)
    t = C.Tracker(p.ref, upsample=U, method="ccu", in_dtype="f32", max_batch=k, stream=stream)
    fr = torch.from_numpy(p.frames[:k]).cuda()
    rec = t.empty_results(k)
    peak = torch.empty((k, 2), dtype=torch.float64, device="cuda")
    gI = torch.empty((k, 64, 64), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        C.ccst_track(t.ctx, fr, k, 0, rec)
        C.ccst_peak_continuous(t.ctx, fr, k, 0, rec, peak, None)
        C.ccst_backward(t.ctx, fr, k, 0, rec, torch.ones((k, 2), dtype=torch.float32, device="cuda"), gI, None)
        torch.cuda.synchronize()
    recs, pk_gpu, gI_gpu = C.decode(rec), peak.cpu().numpy(), gI.cpu().numpy()
    t.close()
    t0 = time.perf_counter()
    ds, dg = 0.0, 0.0
    for i in range(k):
        f = p.frames[i].astype(np.float64)
        orec = cc_oracle.track_one(f, ref, U)
        pk, a, _ = adjoint_oracle.peak_and_vjp(f, ref, orec, (1.0, 1.0))
        ds = max(ds, abs(pk["s"][1] - pk_gpu[i, 0]), abs(pk["s"][0] - pk_gpu[i, 1]))
        dg = max(dg, float(np.max(np.abs(a - gI_gpu[i])) / np.abs(a).max()))
    dt = time.perf_counter() - t0
    ratio = []
    for i in range(k):
        h = 1e-4
        d = p.d_true[i]

        def spot(dy, dx):
            return synth.gaussian_spot(64, 64, 32 + d[1] + dy, 32 + d[0] + dx, 3.0, 1000.0, 10.0)
        b = adjoint_oracle.crlb(p.mu[i].astype(np.float64), (spot(h, 0) - spot(-h, 0)) / (2 * h),
                                (spot(0, h) - spot(0, -h)) / (2 * h))
        ratio.append((sd[0][i] / b[1], sd[1][i] / b[0]))
    ratio = np.array(ratio)
    del recs
    return ({"value": k / dt, "unit": "pairs/s (forward + backward)", "cores": 1, "kind": "oracle",
             "sample": f"first {k} pairs: FP64 oracle tracking, Newton peak and VJP, one process"},
            {"pairs": k, "max_abs_ds_px": ds, "max_rel_dLdI": dg},
            {"pairs": k, "propagated_std_over_crlb_x": float(ratio[:, 0].mean()),
             "propagated_std_over_crlb_y": float(ratio[:, 1].mean()),
             "min_ratio": float(ratio.min())})


REFINE_CAL = 512                 # template refinement leg: calibration frames (known shifts)
REFINE_TEST = 512                # held-out frames
REFINE_STEPS = 30
REFINE_STEP_REL = 0.01
REFINE_ORACLE = (16, 3)          # oracle parity sample: frames, steps


def refine_workload(seed=0, n_cal=REFINE_CAL, n_test=REFINE_TEST, H=64, W=64, sigma=3.0, amp=1000.0, bg=10.0):
    """64 x 64 FP32 spot frames (sigma 3, peak 1000, bg 10, Poisson): calibration frame 0 at
    the centre (it is also the noisy starting template E_0 = I_0), the other calibration and
    all held-out frames at shifts uniform in [-2, 2]^2 px."""
    from paper_2310_08770_b300 import synth
    rng = np.random.default_rng(seed)
    d = rng.uniform(-2.0, 2.0, size=(n_cal + n_test, 2))
    d[0] = 0.0
    fr = np.array([rng.poisson(synth.gaussian_spot(H, W, H / 2 + p[1], W / 2 + p[0], sigma, amp, bg))
                   for p in d]).astype(np.float32)
    truth = synth.gaussian_spot(H, W, H / 2, W / 2, sigma, amp, bg).astype(np.float32)
    return fr[:n_cal], d[:n_cal], fr[n_cal:], d[n_cal:], truth


def refine_leg(C, torch, stream):
    """Reference refinement by the adjoint (ccst_refine_reference) against the paper's Eq. (8)
    offline mean, judged by the displacement error on held-out frames."""
    fc, dc, ft, dt, truth = refine_workload()
    fc_d, ft_d = torch.from_numpy(fc).cuda(), torch.from_numpy(ft).cuda()
    dc_d = torch.from_numpy(dc).cuda()
    n_cal, n_test = len(fc), len(ft)
    ev = lambda: torch.cuda.Event(enable_timing=True)          # noqa: E731

    def test_error(t):
        rec = t.empty_results(n_test)
        peak = torch.empty((n_test, 2), dtype=torch.float64, device="cuda")
        status = torch.empty((n_test,), dtype=torch.int32, device="cuda")
        C.ccst_track(t.ctx, ft_d, n_test, 0, rec)
        C.ccst_peak_continuous(t.ctx, ft_d, n_test, 0, rec, peak, status)
        C.ccst_sync(t.ctx)
        r = C.decode(rec)
        grid = np.stack([r["dx"], r["dy"]], 1).astype(np.float64)
        pk = peak.cpu().numpy()
        return {"rms_px": float(np.sqrt(np.mean(np.sum((grid - dt) ** 2, 1)))),
                "rms_continuous_px": float(np.sqrt(np.mean(np.sum((pk - dt) ** 2, 1)))),
                "bias_px": [float(x) for x in np.mean(grid - dt, 0)]}

    def tracker(ref):
        return C.Tracker(ref, upsample=U, method="ccu", in_dtype="f32", max_batch=n_cal, stream=stream)

    out = {"workload": f"64x64 FP32 spot frames (sigma 3, peak 1000, bg 10, Poisson), {n_cal} calibration frames "
                       f"(frame 0 at the centre, the rest shifted U(-2,2)^2 px, shifts known) and {n_test} held-out "
                       f"frames; u={U}, CC-U; noisy start E_0 = calibration frame 0; {REFINE_STEPS} steps, first "
                       f"step {REFINE_STEP_REL} |E|",
           "loss": "mean over calibration frames of |s* - d|^2 (continuous peak), px^2",
           "metric": "rms displacement error on the held-out frames (grid records and continuous peaks)"}
    with torch.cuda.stream(stream):
        t = tracker(truth)
        out["noise_free_template"] = test_error(t)
        t.close()
        t = tracker(fc[0])
        out["noisy_start"] = test_error(t)
        hist = torch.empty((REFINE_STEPS + 1, 2), dtype=torch.float64, device="cuda")
        C.ccst_refine_reference(t.ctx, fc_d, n_cal, 0, dc_d, 1, REFINE_STEP_REL, hist)     # warm-up
        t.close()
        t = tracker(fc[0])
        a, b = ev(), ev()
        a.record(stream)
        C.ccst_refine_reference(t.ctx, fc_d, n_cal, 0, dc_d, REFINE_STEPS, REFINE_STEP_REL, hist)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        h = hist.cpu().numpy()
        out["adjoint_from_noisy_start"] = test_error(t)
        out["adjoint_from_noisy_start"].update({"loss_first": float(h[0, 0]), "loss_last_accepted": float(
            min(h[:, 0])), "rejected_steps": int(np.sum(np.diff(h[:, 1]) < 0)), "ms_total": ms,
            "ms_per_step": ms / (REFINE_STEPS + 1)})
        t.close()
        t = tracker(fc[0])
        C.ccst_offline_track(t.ctx, fc_d, n_cal, 0, 5, t.empty_results(n_cal))          # Eq. (8), 5 passes
        out["eq8_offline_mean"] = test_error(t)
        C.ccst_refine_reference(t.ctx, fc_d, n_cal, 0, dc_d, REFINE_STEPS, REFINE_STEP_REL, hist)
        h = hist.cpu().numpy()
        out["adjoint_from_eq8"] = test_error(t)
        out["adjoint_from_eq8"].update({"loss_first": float(h[0, 0]), "loss_last_accepted": float(min(h[:, 0])),
                                        "rejected_steps": int(np.sum(np.diff(h[:, 1]) < 0))})
        t.close()
    return out


def refine_cpu_baseline(C, torch, stream):
    """The FP64 refinement oracle on a small sample: its rate and parity of the GPU's loss
    history and template with it."""
    from oracle import refine_oracle
    n, steps = REFINE_ORACLE
    fc, dc, _, _, _ = refine_workload()
    fc, dc = fc[:n], dc[:n]
    t = C.Tracker(fc[0], upsample=U, method="ccu", in_dtype="f32", max_batch=n, stream=stream)
    hist = torch.empty((steps + 1, 2), dtype=torch.float64, device="cuda")
    E = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        C.ccst_refine_reference(t.ctx, torch.from_numpy(fc).cuda(), n, 0, torch.from_numpy(dc).cuda(), steps,
                                REFINE_STEP_REL, hist, E)
        torch.cuda.synchronize()
    t.close()
    t0 = time.perf_counter()
    E_o, h_o = refine_oracle.refine(fc.astype(np.float64), fc[0].astype(np.float64), dc, steps, REFINE_STEP_REL, U)
    dt = time.perf_counter() - t0
    h = hist.cpu().numpy()
    return ({"value": n * (steps + 1) / dt, "unit": "frame-evaluations/s", "cores": 1, "kind": "oracle",
             "sample": f"first {n} calibration frames, {steps} steps, FP64 refinement oracle, one process"},
            {"frames": n, "steps": steps, "same_steps": bool(np.array_equal(h[:, 1], h_o[:, 1])),
             "max_rel_loss": float(np.max(np.abs(h[:, 0] - h_o[:, 0]) / np.abs(h_o[:, 0]))),
             "max_template_diff_rel": float(np.max(np.abs(E.cpu().numpy() - E_o)) / np.abs(E_o).max())})


ROIS_N = 4096                    # uneven-ROI leg
ROIS_SIDES = (32, 48, 64, 96, 128)   # 48 and 96 run on the FP32 general-size kernel
ROIS_POW2_SIDES = (32, 64, 128)      # the power-of-two kernel alone, for context
ROIS_REPS = 10
ROIS_ORACLE = 48


def rois_leg(C, torch, stream, n_rois=ROIS_N, sides=ROIS_SIDES, plain=True):
    """Uneven batch: FP32 ROIs of mixed sizes, each against its own reference, in one
    ccst_track_rois call (the power-of-two kernel and the general-size kernels side by side),
    after ccst_autotune, replayed as one captured CUDA graph (the reported value). Beside it:
    the same call launched directly, the same ROIs as one batched call per size class (the
    per-size form), and (context) one call per ROI."""
    import ctypes
    from paper_2310_08770_b300 import synth
    r = synth.uneven_rois(seed=0, n=n_rois, sides=sides)
    n = len(r.frames)
    frames = [torch.from_numpy(f).cuda() for f in r.frames]
    ev = lambda: torch.cuda.Event(enable_timing=True)          # noqa: E731
    needs_tune = any(x not in (16, 32, 64, 128) for x in sides)

    def make(graphs):
        t = C.Tracker(r.refs[0], upsample=U, method="ccu", in_dtype="f32", stream=stream, graphs=graphs)
        t0 = time.perf_counter()
        ids = [0] + [C.ccst_add_reference(t.ctx, ref, ref.shape[0], ref.shape[1]) for ref in r.refs[1:]]
        return t, C.make_rois(frames, ids), time.perf_counter() - t0

    def timed(fn, reps=ROIS_REPS):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    with torch.cuda.stream(stream):
        # direct launches
        t, rois, setup_s = make(False)
        out = t.empty_results(n)
        default_ms = timed(lambda: C.ccst_track_rois(t.ctx, rois, n, out))
        t0 = time.perf_counter()
        tuned = C.ccst_autotune(t.ctx, 3, rois, n) if needs_tune else []
        tune_s = time.perf_counter() - t0
        direct_ms = timed(lambda: C.ccst_track_rois(t.ctx, rois, n, out)) if tuned else default_ms
        res = C.decode(out)
        # per-size form: one batched call per size class, one after another
        groups = {}
        for i, f in enumerate(r.frames):
            groups.setdefault(f.shape[0], []).append(i)
        per = [(C.make_rois([frames[i] for i in idx], [rois[i].ref_id for i in idx]), len(idx),
                t.empty_results(len(idx)), idx) for _, idx in sorted(groups.items())]
        per_size_ms = timed(lambda: [C.ccst_track_rois(t.ctx, rr, m, oo) for rr, m, oo, _ in per])
        per_same = all(C.decode(oo).tobytes() == res[idx].tobytes() for _, _, oo, idx in per)
        plain_ms = None
        if plain:
            a, b = ev(), ev()
            a.record(stream)
            for i in range(n):                                  # one call per ROI
                C.ccst_track_rois(t.ctx, ctypes.byref(rois[i]), 1, out[i:i + 1])
            b.record(stream)
            torch.cuda.synchronize()
            plain_ms = a.elapsed_time(b)
        same = bool(C.decode(out).tobytes() == res.tobytes())
        t.close()
        # the same work list captured as one graph and replayed (the product path)
        tg, rois_g, _ = make(True)
        if needs_tune:
            C.ccst_autotune(tg.ctx, 3, rois_g, n)
        out_g = tg.empty_results(n)
        graph_ms = timed(lambda: C.ccst_track_rois(tg.ctx, rois_g, n, out_g))
        gstats = C.ccst_graph_stats(tg.ctx)
        graph_same = bool(C.decode(out_g).tobytes() == res.tobytes())
        tg.close()
    flop = sum(scope_flop_per_frame(f.shape[0], f.shape[1], U) for f in r.frames)
    flop_folded = sum(flop_per_frame(f.shape[0], f.shape[1], U) for f in r.frames)
    fma = C.ccst_fp32_fma_peak(stream.cuda_stream)
    peak = fma["tflops"]
    achieved = flop / (graph_ms / 1e3) / 1e12
    achieved_folded = flop_folded / (graph_ms / 1e3) / 1e12
    sizes = {s_: int(sum(1 for f in r.frames if f.shape[0] == s_)) for s_ in sides}
    line = {"workload": f"{n} FP32 square ROIs, sides uniform over {list(sides)} ({sizes}), per-ROI noise-free "
                        "reference (sigma U(1.5,4), peak U(200,5000), bg U(5,50)), Poisson frames shifted U(-3,3)^2 px, "
                        f"u={U}, CC-U",
            "value": n / (graph_ms / 1e3), "unit": "ROIs/s", "ms_per_batch": graph_ms,
            "form": "one ccst_track_rois work list captured as one CUDA graph (all its kernels) and replayed",
            "graphs": gstats, "records_equal_to_direct": graph_same,
            "direct_launch": {"value": n / (direct_ms / 1e3), "ms": direct_ms},
            "per_size_batched": {"value": n / (per_size_ms / 1e3), "ms": per_size_ms, "calls": len(per),
                                 "records_equal": bool(per_same),
                                 "form": "one batched ccst_track_rois call per side, one after another"},
            "speedup_vs_per_size_batched": per_size_ms / graph_ms,
            "reference_setup_s": setup_s,
            "autotune": {"ms_per_batch_default_schedule": default_ms, "seconds": tune_s,
                         "plans": [{k: x[k] for k in ("H", "W", "H1", "W1", "threads", "us_per_frame")}
                                   for x in tuned]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "kernel": "track_rois_kernel + mix_track_kernel (+ track_generic_kernel on its fallback "
                                   "list)", "flop_total": flop,
                         "flop_basis": "the scope table's flops for every ROI (FFTs, product and phase, stage A over "
                                       "all H rows, stage B over the half spectrum; 17.1 M at 128 x 128), as the "
                                       "headline counts them",
                         "peak_basis": "of measured: FP32 FMA rate of this GPU (ccst_fp32_fma_peak)",
                         "folded": {"flop_total": flop_folded, "achieved": achieved_folded,
                                    "frac": achieved_folded / peak,
                                    "basis": "the flops the kernels' folded formulation performs (Hermitian "
                                             "symmetry in both contraction stages; the guard levels come on top)"}}}
    if plain:
        line.update({"plain_per_roi_call": {"value": n / (plain_ms / 1e3), "unit": "ROIs/s", "ms": plain_ms},
                     "speedup_vs_plain": plain_ms / graph_ms, "records_equal_to_plain": same})
    return line, (r, res)


# The paper's Table I (CC-SN images/s, CUDA on an RTX 3080): context for the same shapes and
# upsampling factors on this GPU, not a target (other hardware, unstated workload).
TABLE1_CUDA = {(256, 128): {128: 1636, 256: 811}, (256, 256): {128: 981, 256: 432}}
TABLE1_FRAMES = 2048
TABLE1_ORACLE = 4


def table1_leg(C, torch, stream):
    """CC-SN on noise-free-reference / Poisson spot frames of the paper's Table I shapes
    (256 x 128 and 256 x 256, uint16) at u = 128 and 256: batched images/s through ccst_track
    (the FP32 general-size kernel), with the first frames checked against the FP64 oracle."""
    import oracle
    from paper_2310_08770_b300 import synth
    out = []
    rng = np.random.default_rng(11)
    for (h, w), paper in TABLE1_CUDA.items():
        ref = synth.gaussian_spot(h, w, h / 2, w / 2, 3.0, 2000.0, 20.0).astype(np.float32)
        d = rng.uniform(-3, 3, size=(64, 2))
        pool = np.array([rng.poisson(synth.gaussian_spot(h, w, h / 2 + p[0], w / 2 + p[1], 3.0, 2000.0, 20.0))
                         for p in d]).astype(np.uint16)
        frames = np.concatenate([pool] * (TABLE1_FRAMES // len(pool)))
        dev = torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
        for u in sorted(paper):
            with torch.cuda.stream(stream):
                t = C.Tracker(ref, upsample=u, method="ccsn", in_dtype="u16", max_batch=len(frames), stream=stream)
                o = t.empty_results(len(frames))
                for _ in range(2):
                    C.ccst_track(t.ctx, dev, len(frames), 0, o)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(3):
                    C.ccst_track(t.ctx, dev, len(frames), 0, o)
                b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / 3
                res = C.decode(o)
                t.close()
            bad = 0
            for i in range(TABLE1_ORACLE):
                q = oracle.track_one(frames[i].astype(np.float64), ref.astype(np.float64), u, oracle.CC_SN)
                if (int(res["ipy"][i]), int(res["ipx"][i])) != (q["ipy"], q["ipx"]) or \
                        abs(float(res["dx"][i]) - q["dx32"]) > 1e-3 or abs(float(res["dy"][i]) - q["dy32"]) > 1e-3:
                    bad += 1
            out.append({"shape": f"{h}x{w}", "u": u, "images_per_s": len(frames) / (ms / 1e3),
                        "fp32_records": int(np.sum((res["flags"] & C.R_FP32_GENERAL) != 0)),
                        "frames": len(frames), "oracle_checked": TABLE1_ORACLE, "oracle_mismatches": bad,
                        "paper_cuda_images_per_s": paper[u]})
    return {"workload": "the paper's Table I shapes, CC-SN, uint16 Poisson spot frames (sigma 3, peak 2000, bg 20, "
                        f"shifts U(-3,3)^2) against a noise-free reference, batches of {TABLE1_FRAMES} frames",
            "context": "paper_cuda_images_per_s: Table I, CUDA on an RTX 3080 (another GPU, workload unstated); "
                       "not a target", "runs": out}


def rois_cpu_baseline(r, res):
    """The FP64 oracle on the first ROIS_ORACLE ROIs: its rate and parity with the batch."""
    import oracle
    k = ROIS_ORACLE
    t0 = time.perf_counter()
    orc = [oracle.track_one(r.frames[i].astype(np.float64), r.refs[i].astype(np.float64), U) for i in range(k)]
    dt = time.perf_counter() - t0
    mism = sum(1 for a, o in zip(res[:k], orc)
               if (int(a["ipy"]), int(a["ipx"])) != (o["ipy"], o["ipx"])
               or abs(float(a["dx"]) - o["dx32"]) > 1e-3 or abs(float(a["dy"]) - o["dy32"]) > 1e-3)
    return ({"value": k / dt, "unit": "ROIs/s", "cores": 1, "kind": "oracle",
             "sample": f"first {k} ROIs of the uneven batch, FP64 numpy oracle, one process"},
            {"rois": k, "mismatches": mism, "tolerance_px": 1e-3})


SERVE_TRUE_SIDES = (64, 96, 128, 192, 256, 64, 128, 256)
SERVE_SIDES = (64, 64, 128, 128, 128, 64, 128, 128)   # power-of-two stand-ins for the sides above
SERVE_TRUE_SECONDS = 2.0
SERVE_RATES_HZ = (1e3, 2e3, 5e3, 10e3, 20e3, 50e3, 100e3, 100e3)
SERVE_POOL = 512
SERVE_SECONDS = 5.0


def serving_leg(C, torch, sides=SERVE_SIDES, seconds=SERVE_SECONDS, slots=4096, note=""):
    """8 simulated cameras at Poisson rates of 1-100 kHz for `seconds` through one server
    (continuous batching over the uneven-ROI and general-size kernels); host-clock
    submit-to-result latency."""
    from paper_2310_08770_b300 import synth
    pools = [synth.camera_pool(seed=k, n=SERVE_POOL, N=N) for k, N in enumerate(sides)]
    t = C.Tracker(pools[0][0], upsample=U, method="ccu", in_dtype="u16")
    ids = [0] + [C.ccst_add_reference(t.ctx, ref, ref.shape[0], ref.shape[1]) for ref, _ in pools[1:]]
    srv = C.ccst_server_create(t.ctx, slots, 1024)
    try:
        C.ccst_server_loadgen(srv, ids, SERVE_RATES_HZ, [f for _, f in pools], 0.2, seed=99)     # warm-up
        st = C.ccst_server_loadgen(srv, ids, SERVE_RATES_HZ, [f for _, f in pools], seconds, seed=0)
    finally:
        C.ccst_server_destroy(srv)
        t.close()
    return {"workload": f"8 cameras, sides {list(sides)}{note}, "
                        f"uint16 spot frames (sigma 3, peak 2000, bg 20, shifts U(-3,3)^2), pools of {SERVE_POOL} "
                        f"frames, Poisson arrivals at {[int(r) for r in SERVE_RATES_HZ]} Hz for {seconds} s, "
                        f"u=100, CC-U; {slots} device slots, batches of up to 1024",
            "offered_hz": sum(SERVE_RATES_HZ), "value": st["completed"] / seconds, "unit": "frames/s",
            "refused_fraction": st["rejected"] / max(1, st["submitted"] + st["rejected"]),
            "p50_us": st["p50_us"], "p99_us": st["p99_us"], "max_us": st["max_us"],
            "submitted": st["submitted"], "rejected": st["rejected"], "batches": st["batches"],
            "mean_batch": st["mean_batch"],
            "latency": "host clock, submit call to the worker seeing the batch's completion event"}


LOAD_RATES_HZ = (5e3, 15e3, 30e3, 100e3, 300e3)
LOAD_SECONDS = 1.0
LOAD_POOL = 4096
LOAD_BUDGET = LOAD_POOL * H * W * 2          # admission arena: 4096 frames of 128 x 128 uint16


def load_latency_leg(C, torch, s):
    """Latency under offered load: one 128 x 128 uint16 camera (frames of the stream) with
    Poisson arrivals at each rate, through the server twice: served (continuous batching, up
    to 1024 frames per launch, 4 batches in flight) and plain (one launch per frame, each
    after the previous one finished: max_batch 1, 1 in flight). Same admission budget, same
    host-clock latency (submit to the worker seeing the result), same load generator."""
    pool = np.ascontiguousarray(s.frames[:LOAD_POOL])
    t = C.Tracker(s.ref, upsample=U, method="ccu", in_dtype="u16")
    forms = {"served": (1024, 4), "plain": (1, 1)}
    rows = []
    try:
        for rate in LOAD_RATES_HZ:
            row = {"offered_hz": rate}
            for name, (mb, depth) in forms.items():
                srv = C.ccst_server_create_ex(t.ctx, mb, depth, LOAD_BUDGET)
                try:
                    C.ccst_server_loadgen(srv, [0], [min(rate, 20e3)], [pool], 0.05, seed=98)     # warm-up
                    st = C.ccst_server_loadgen(srv, [0], [rate], [pool], LOAD_SECONDS, seed=1)
                finally:
                    C.ccst_server_destroy(srv)
                row[name] = {"frames_per_s": st["completed"] / LOAD_SECONDS,
                             "refused_fraction": st["rejected"] / max(1, st["submitted"] + st["rejected"]),
                             "p50_us": st["p50_us"], "p99_us": st["p99_us"], "mean_batch": st["mean_batch"]}
            rows.append(row)
    finally:
        t.close()
    wins = [r["offered_hz"] for r in rows
            if r["served"]["p99_us"] < r["plain"]["p99_us"] and r["served"]["frames_per_s"] >= r["plain"]["frames_per_s"]]
    return {"workload": f"one 128x128 uint16 camera (frames of the stream, pool of {LOAD_POOL}), Poisson arrivals "
                        f"for {LOAD_SECONDS} s per rate, u={U}, CC-U; admission budget {LOAD_BUDGET >> 20} MiB",
            "forms": {"served": "continuous batching: up to 1024 frames per launch, 4 batches in flight",
                      "plain": "one launch per frame, each after the previous finished (max_batch 1, 1 in flight)"},
            "latency": "host clock, submit call to the worker seeing the frame's completion event",
            "rates": rows, "served_beats_plain_on_p99_and_rate_at_hz": wins}


PLAIN_FRAMES = 1024


def plain_leg(C, torch, s, frames_dev, stream):
    """The plain form: one direct launch per frame (no batching, no graph) on one stream, for
    the first PLAIN_FRAMES frames; each frame's latency is its own launch (CUDA events)."""
    t = C.Tracker(s.ref, upsample=U, method="ccu", in_dtype="u16", max_batch=1, stream=stream)
    out = t.empty_results(PLAIN_FRAMES)
    n = min(PLAIN_FRAMES, frames_dev.shape[0])
    with torch.cuda.stream(stream):
        for i in range(8):
            C.ccst_track(t.ctx, frames_dev[i:i + 1], 1, 0, out[i:i + 1])
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(n):
            ev[i][0].record(stream)
            C.ccst_track(t.ctx, frames_dev[i:i + 1], 1, 0, out[i:i + 1])
            ev[i][1].record(stream)
        b.record(stream)
        torch.cuda.synchronize()
    lat = np.array([e0.elapsed_time(e1) * 1e3 for e0, e1 in ev])
    total_ms = a.elapsed_time(b)
    t.close()
    return {"workload": f"frames 0..{n} of the stream, one ccst_track launch per frame (no graph), one stream",
            "value": n / (total_ms / 1e3), "unit": "frames/s", "p50_us": float(np.percentile(lat, 50)),
            "p99_us": float(np.percentile(lat, 99)), "gpu_launches": n}


# ---------------------------------------------------------------- our arm
TIE_MARGIN = 1e-12               # oracle top-2 margin (relative) below which a frame is a genuine tie


def batch_bounds(n_frames, batch=BATCH):
    """The stream's batches: 39 x 256 frames and a last batch of 16 at 10,000 frames."""
    return [(lo, min(n_frames, lo + batch)) for lo in range(0, n_frames, batch)]


def headline_config(world):
    """config of the headline line; the reference arm prints the same dictionary."""
    return {"workload": WORKLOAD, "global_batch": BATCH * world, "frames_per_rank": N_FRAMES,
            "frames_per_step": N_FRAMES * world, "batches_per_step": len(batch_bounds(N_FRAMES)),
            "upsample": U, "streams": 3, "parallelism": f"replicas x{world} (independent streams)",
            "l2": "inputs larger than L2 (the 328 MB stream per rank is read once per step)"}


def parity_with_ties(gpu, orc, u=U):
    """Frame-by-frame comparison with the oracle: integer peaks identical and |d| within 1e-3
    px, except where the oracle's own top-2 margin shows a genuine tie (< TIE_MARGIN relative),
    where a one-bin difference is allowed and counted. Lists every mismatch and tie."""
    mism, ties = [], []
    for i, (a, o) in enumerate(zip(gpu, orc)):
        int_same = (int(a["ipy"]), int(a["ipx"])) == (o["ipy"], o["ipx"])
        close = abs(float(a["dx"]) - o["dx32"]) <= 1e-3 and abs(float(a["dy"]) - o["dy32"]) <= 1e-3
        if int_same and close:
            continue
        one_bin = (abs(float(a["dx"]) - o["dx32"]) <= 1.0 / u + 1e-6 and abs(float(a["dy"]) - o["dy32"]) <= 1.0 / u + 1e-6)
        item = {"frame": i, "gpu": [float(a["dx"]), float(a["dy"]), int(a["ipy"]), int(a["ipx"])],
                "oracle": [o["dx32"], o["dy32"], o["ipy"], o["ipx"]],
                "int_margin": o["int_margin"], "sub_margin": o["sub_margin"]}
        tie = ((not int_same and o["int_margin"] < TIE_MARGIN) or
               (int_same and one_bin and o["sub_margin"] < TIE_MARGIN))
        (ties if tie else mism).append(item)
    return {"frames": len(orc), "mismatches": len(mism), "genuine_ties": len(ties), "tolerance_px": 1e-3,
            "tie_rule": f"one bin allowed where the oracle's top-2 margin < {TIE_MARGIN} of sum|X|/HW",
            "mismatch_list": mism[:20], "tie_list": ties[:20]}


def run_ours(args):
    import torch
    from paper_2310_08770_b300 import ccst as C
    from paper_2310_08770_b300 import synth

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n_frames = args.frames
    s = synth.frame_stream(seed=shard_seed(rank), n=N_FRAMES, count=n_frames)
    frames_dev = torch.from_numpy(s.frames.view(np.int16)).cuda().view(torch.uint16)
    bounds = batch_bounds(n_frames)
    nb = len(bounds)
    outs = torch.empty((n_frames, 24), dtype=torch.uint8, device="cuda")
    # batch b runs on stream b % streams: the next batch's CTAs start on the SMs the previous
    # batch's last frames leave idle; each cached graph (one per stream and batch) owns its
    # frame counter
    streams = [torch.cuda.Stream() for _ in range(args.streams)]
    stream = streams[0]
    t = C.Tracker(s.ref, upsample=U, method="ccu", in_dtype="u16", max_batch=BATCH, stream=stream, graphs=True)
    lat_passes = min(args.steps, 50)                # per-batch latency events for the first passes

    # each batch's stream handle and device addresses, computed once: the host loop that
    # issues a step's 40 launches then costs a few microseconds per batch, below the
    # device's time per batch (the loop is otherwise the bound on a slow host)
    lib = C.lib()
    fbase, obase = frames_dev.data_ptr(), outs.data_ptr()
    issue = [(streams[b % len(streams)], streams[b % len(streams)].cuda_stream, fbase + lo * H * W * 2, hi - lo,
              obase + lo * 24) for b, (lo, hi) in enumerate(bounds)]

    def one_pass(ev=None):
        for b, (si, sh, fp, m, op) in enumerate(issue):
            if ev is not None:
                ev[b][0].record(si)
            if lib.ccst_set_stream(t.ctx, sh) or lib.ccst_track(t.ctx, fp, m, 0, op):
                raise C.CcstError(-1, lib.ccst_last_error(t.ctx).decode())
            if ev is not None:
                ev[b][1].record(si)

    fma = C.ccst_fp32_fma_peak(stream.cuda_stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):                # the first pass captures every batch's graph
            one_pass()
        torch.cuda.synchronize()
        outs.fill_(0xFF)                            # sentinel: every record must be rewritten
        stats0 = C.ccst_graph_stats(t.ctx)
        lat_ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in bounds]
                  for _ in range(lat_passes)]
        t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local)
        clocks.start()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_begin.record(stream)
        for st in streams[1:]:
            st.wait_event(t_begin)
        h0 = time.perf_counter()
        for i in range(args.steps):
            one_pass(lat_ev[i] if i < lat_passes else None)
        host_issue_s = time.perf_counter() - h0
        for st in streams[1:]:
            e = torch.cuda.Event()
            e.record(st)
            stream.wait_event(e)
        t_end.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clk = clocks.stop()
    stats1 = C.ccst_graph_stats(t.ctx)
    lat_us = np.array([[a.elapsed_time(b) * 1e3 for a, b in row] for row in lat_ev])
    lat_w = np.array([[hi - lo for lo, hi in bounds]] * lat_passes, dtype=float)
    total_ms = t_begin.elapsed_time(t_end)
    total_ms_max = max_over_ranks(total_ms, world, device="cuda")
    frames_step = n_frames
    value = frames_step * args.steps * world / (total_ms_max / 1e3)
    raw = outs.cpu().numpy()
    unwritten = int(np.sum((raw == 0xFF).all(axis=1)))
    assert unwritten == 0, f"{unwritten} records not written in the timed region"
    res_all = C.decode(outs)
    flags = res_all["flags"]

    # roofline of the dominant kernel (FP32 ALU bound, the FMA rate measured above). The timed
    # region holds only its launches (40 graph replays per step); with three batches in flight
    # their spans overlap, so a launch's average duration is the region's time per launch
    launches = args.steps * nb
    ms_per_launch = total_ms / launches
    fpf_s, fpf_f, fpf_c = scope_flop_per_frame(), flop_per_frame(), scope_contraction_flop()
    rate = frames_step * args.steps / (total_ms / 1e3)
    peak = fma["tflops"]
    peaks = load_peaks()
    tensor_peak = peaks.get("bf16_tflops")

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e_steps = 0 if args.no_e2e else args.steps
    pinned_t = torch.from_numpy(s.frames.view(np.int16)).pin_memory()
    pinned = pinned_t.numpy().view(np.uint16)
    # pipelined: up to DEPTH batches in flight, each with its own host result area; a
    # batch's host->device copy overlaps the tracking of the one before
    DEPTH = 3
    host_outs = [torch.empty((BATCH * 24,), dtype=torch.uint8).pin_memory() for _ in range(DEPTH + 1)]
    host_views = [h.numpy().view(C.RESULT_DTYPE) for h in host_outs]

    def e2e_run(passes):
        pending, done_frames, i = [], 0, 0
        for _ in range(passes):
            for lo, hi in bounds:
                pending.append(C.ccst_submit_host(t.ctx, pinned[lo:hi], hi - lo, 0, host_views[i % (DEPTH + 1)]))
                done_frames += hi - lo
                i += 1
                if len(pending) >= DEPTH:
                    while not C.ccst_poll(t.ctx, pending.pop(0), 100000):
                        pass
        for tk in pending:
            while not C.ccst_poll(t.ctx, tk, 100000):
                pass
        return done_frames, i
    C.ccst_set_stream(t.ctx, stream.cuda_stream)
    if e2e_steps:
        e2e_run(1)
    t0 = time.perf_counter()
    e2e_frames, e2e_batches = e2e_run(e2e_steps)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
    # the results of the last batch, read back through the pipelined path, match the device path
    if e2e_steps:
        lo, hi = bounds[-1]
        got = host_views[(e2e_batches - 1) % (DEPTH + 1)][:hi - lo]
        ref = res_all[lo:hi]
        assert got.tobytes() == ref.tobytes(), "e2e results differ"
    e2e = {"value": e2e_frames * world / e2e_s if e2e_frames else None, "unit": "frames/s",
           "h2d_bytes_per_step": n_frames * H * W * 2, "d2h_bytes_per_step": n_frames * 24,
           "api": f"ccst_submit_host + ccst_poll, one step = the {nb} batches of the stream (pinned host frames "
                  f"in, host results out; {DEPTH} batches in flight over 4 staging slots and 2 streams, so copies "
                  "overlap tracking)"}

    line = {
        "metric": "frames/s and p50/p99 per-frame latency (us) at 128x128, <=1e-3 px vs FP64 oracle",
        "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "p50_us": weighted_percentile(lat_us.ravel(), lat_w.ravel(), 50),
        "p99_us": weighted_percentile(lat_us.ravel(), lat_w.ravel(), 99),
        "latency_basis": "frame-weighted percentiles of each batch's end event - start event on its stream, "
                         f"first {lat_passes} timed passes, three batches in flight",
        "config": headline_config(world),
        "roofline": {"bound": "alu", "achieved": fpf_s * rate / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": fpf_s * rate / 1e12 / peak, "traffic": profiled_traffic(),
                     "kernel": "track_kernel", "flop_per_frame": fpf_s, "frames_per_launch": frames_step / nb,
                     "ms_per_launch": ms_per_launch, "launches_timed": launches,
                     "achieved_basis": "scope-table flops per frame (17.1 M at 128x128, u=100: FFTs, product and "
                                       "phase, stage A over all H rows, stage B over the half spectrum) x frames / "
                                       "timed region (CUDA events on the launching streams)",
                     "peak_basis": "of measured: FP32 FMA rate of this GPU (ccst_fp32_fma_peak, independent FMA "
                                   "chains on every SM, best of 3 launches), "
                                   f"nominal {fma['nominal_tflops']:.1f} TFLOP/s from the device attributes",
                     "folded": {"flop_per_frame": fpf_f, "achieved": fpf_f * rate / 1e12,
                                "frac": fpf_f * rate / 1e12 / peak,
                                "basis": "the flops the kernel's folded formulation performs (Hermitian symmetry "
                                         "in both contraction stages)"},
                     "contraction_tensor_pipe": {
                         "flop_per_frame": fpf_c, "achieved": fpf_c * rate / 1e12,
                         "peak": tensor_peak / 3 if tensor_peak else None,
                         "frac": fpf_c * rate / 1e12 / (tensor_peak / 3) if tensor_peak else None,
                         "basis": "stages A and B run as fp16 hi/lo MMAs (3 products each) on the tensor pipe: "
                                  "their scope-table flops against the measured dense bf16/fp16 rate / 3 "
                                  "(the pool's measured bf16 GEMM rate, burst)"},
                     "ingest": {"achieved": rate * (H * W * 2 + 24) / 1e9, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                                "frac": (rate * (H * W * 2 + 24) / 1e9 / peaks["hbm_gbs"]
                                         if peaks.get("hbm_gbs") else None),
                                "basis": "algorithmic HBM bytes per frame (uint16 input + 24-byte record) x "
                                         "frames/s per GPU, against the measured copy bandwidth"}},
        "fp32_fma_peak": fma,
        "graphs": {"instantiations": stats1["instantiations"], "distinct_batches": nb,
                   "instantiated_in_timed_region": stats1["instantiations"] - stats0["instantiations"],
                   "replays_timed": stats1["replays"] - stats0["replays"]},
        "records_written": {"frames": n_frames, "unwritten_after_timed_region": unwritten,
                            "check": "outputs filled with 0xFF before the timed region"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,                       # one tracking kernel per batch
        "host_issue": {"ms_per_step": host_issue_s * 1e3 / args.steps, "gpu_ms_per_step": total_ms / args.steps,
                       "basis": "wall time of the host loop that issues a step's launches (and its latency "
                                "events), against the device time of a step: near equal means host-bound"},
        "guard": {"frames": int(len(flags)), "int": int(np.sum((flags & C.R_INT_GUARD) != 0)),
                  "sub": int(np.sum((flags & C.R_SUB_GUARD) != 0)), "df64": int(np.sum((flags & C.R_DF64) != 0)),
                  "overflow": int(np.sum((flags & C.R_OVERFLOW) != 0))},
    }
    rt_line = rt_res = None
    if world == 1:
        line["plain_per_frame_launch"] = plain_leg(C, torch, s, frames_dev, stream)
    if world == 1 and not args.no_serving:
        line["latency_under_load"] = load_latency_leg(C, torch, s)
    if world == 1 and not args.no_realtime:         # the extra legs are single-GPU measurements
        rt_line, rt_res = realtime_leg(C, torch, s, stream, args.rt_frames)
        line["realtime"] = rt_line
    if world == 1 and not args.no_offline:
        line["offline"] = offline_leg(C, torch, s, frames_dev, n_frames, stream)
    if world == 1 and not args.no_serving:
        line["serving"] = serving_leg(C, torch, note=" (power-of-two stand-ins for 64, 96, 128, 192, 256, 64, "
                                                     "128, 256)")
        # the workload's own sides: 96, 192 and 256 run on the FP32 general-size kernel
        line["serving"]["true_sides"] = serving_leg(C, torch, SERVE_TRUE_SIDES, SERVE_TRUE_SECONDS, 2048,
                                                    " (96, 192, 256 on the FP32 general-size kernel)")
    rois_extra = None
    if world == 1 and not args.no_table1:
        line["table1"] = table1_leg(C, torch, stream)
    if world == 1 and not args.no_rois:
        sides = tuple(int(x) for x in args.rois_sides.split(",")) if args.rois_sides else ROIS_SIDES
        line["rois"], rois_extra = rois_leg(C, torch, stream, args.rois_n, sides, plain=sides == ROIS_SIDES)
        if sides == ROIS_SIDES:
            line["rois"]["power_of_two_sides_only"] = rois_leg(C, torch, stream, args.rois_n, ROIS_POW2_SIDES,
                                                               plain=False)[0]
    adj_extra = None
    if world == 1 and not args.no_adjoint:
        line["adjoint"], adj_extra = adjoint_leg(C, torch, stream)
        line["refine"] = refine_leg(C, torch, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if rois_extra is not None:
            line["rois"]["cpu_baseline"], line["rois"]["parity"] = rois_cpu_baseline(*rois_extra)
        if adj_extra is not None:
            (line["adjoint"]["cpu_baseline"], line["adjoint"]["parity"],
             line["adjoint"]["cramer_rao"]) = adjoint_cpu_baseline(C, torch, stream, *adj_extra)
            line["refine"]["cpu_baseline"], line["refine"]["parity"] = refine_cpu_baseline(C, torch, stream)
        if "offline" in line:
            line["offline"]["cpu_baseline"], line["offline"]["parity"] = offline_cpu_baseline(C, torch, s, stream)
        if rt_res is not None:
            rt_line["cpu_baseline"], rt_line["parity"] = realtime_cpu_baseline(s.frames, rt_res)
        orc, cb = cpu_baseline(s.frames, s.ref)
        line["cpu_baseline"] = cb
        line["parity"] = parity_with_ties(res_all[:len(orc)], orc)
    t.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    """The FP64 oracle as it stands, on the host cores, on the headline's config: each step
    tracks a bounded sample of the step's 10,000 frames (the same frames every step)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    from paper_2310_08770_b300 import synth
    s = synth.frame_stream(seed=0, n=N_FRAMES)
    t0 = time.perf_counter()
    oracle.track_one(s.frames[0], s.ref, u=U)
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    budget = 150.0
    per_step = int(max(1, budget * cores / ((args.steps + args.warmup) * max(t1, 1e-3))))
    per_step = min(per_step, N_FRAMES)
    use_pool = per_step >= cores
    pool = None
    if use_pool:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        pool = mp.get_context("spawn").Pool(cores)
        pool.map(_oracle_chunk, [(s.frames[:1], s.ref)] * cores)
    # the sample: frames spread evenly over the stream
    pick = np.linspace(0, N_FRAMES - 1, per_step).astype(int)
    fr = s.frames[pick]

    def step():
        if pool:
            pool.map(_oracle_chunk, [(c, s.ref) for c in np.array_split(fr, cores) if len(c)])
        else:
            oracle.track_batch(fr, s.ref, u=U)
        return len(fr)

    for _ in range(args.warmup):
        step()
    lat, sizes = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sizes.append(step())
        lat.append(time.perf_counter() - t0)
    dt = time.perf_counter() - t_all
    if pool:
        pool.close()
    value = sum(sizes) / dt
    sample = (f"{per_step} of the 10000 frames per step (evenly spaced), FP64 numpy oracle (naive separable DFTs), "
              f"{cores if use_pool else 1} process(es)")
    print(json.dumps({
        "impl": "reference",
        "metric": "frames/s and p50/p99 per-frame latency (us) at 128x128, <=1e-3 px vs FP64 oracle",
        "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "p50_us": float(np.median(lat)) * 1e6 / max(1, per_step), "p99_us": float(np.percentile(lat, 99)) * 1e6 / max(1, per_step),
        "latency_basis": "time per sample step / frames in it",
        "config": headline_config(world),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": cores if use_pool else 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-realtime", action="store_true")
    ap.add_argument("--no-offline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-rois", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-table1", action="store_true")
    ap.add_argument("--rois-n", type=int, default=ROIS_N)
    ap.add_argument("--rois-sides", default="", help="comma-separated ROI sides of the uneven-ROI leg "
                    "(default: the survey's mix); e.g. 96 to profile one kernel")
    ap.add_argument("--streams", type=int, default=3)
    ap.add_argument("--rt-frames", type=int, default=RT_FRAMES)
    ap.add_argument("--frames", type=int, default=N_FRAMES,
                    help="frames of the stream to stage (the workload is 10000; smaller only for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2310_08770_b300 import build
        build.build()
        run_ours(args)


if __name__ == "__main__":
    main()
