#!/usr/bin/env python
"""Benchmark: 640x480 frame-to-keyframe alignments per second (plain FP32 path).

Workload: the seeded synthetic 300-frame 640x480 room sequence (30 Hz, <= 0.5 m/s,
<= 30 deg/s; fx = fy = 525, cx = 319.5, cy = 239.5), tracked frame to keyframe
on a 4-level pyramid with [10, 5, 5, 5] Gauss-Newton iterations (coarsest
first), every frame fused into the keyframe, keyframe switch every 20 frames.
One step = one frame through the whole hot path: the frame's pyramid, the
constant-velocity guess, the IRLS alignment (robust scale + fused sweep + solve
per iteration), the keyframe fusion (or switch) and the keyframe pyramid.

value      frames (= 640x480 alignments) per second over all ranks, inputs
           resident in HBM, each step timed with CUDA events on the tracker's
           stream; L2 is flushed (a 512 MiB write) between steps, outside the
           timed intervals.
e2e        the same with every step's frame copied from pinned host memory and
           its result struct read back to pinned host memory inside the step.
roofline   the dominant kernel by share of its timed region: each alignment
           kernel is timed live (CUDA events around each of its launches, on the
           tracker's stream) over its own pass of 60 device-resident steps, since
           events between launches break the programmatic dependent launches and
           would slow the value pass; achieved = 16 B x units per launch / launch
           time (units: level pixels for the sweep, systematic-sample pixels for
           the robust-scale kernel).  The other kernel is reported under
           roofline_other_kernels.

Multi-GPU: every rank tracks its own independent sequence (seed = rank), no
collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "640x480 alignments/s at <=1e-5 rad pose err vs plain GPU form; % HBM roofline"
UNIT = "alignments/s"
W, H = 640, 480
LEVELS, ITERS = 4, (5, 5, 5, 10)
KF_EVERY = 20
N_FRAMES = 300
# algorithmic bytes per pixel (or sample) per launch: I_A, W_A, I_B, W_B each read
# once -- 4 B each as float32 planes, 2 B each in the reduced-precision form
BYTES_PER_UNIT = {"f32": 16, "bf16": 8}

# FP32 operations (FMA, multiply or add, each counted once) per pixel-iteration of the
# sweep: warp 20, bilinear taps and transfer 18, gradients/Jacobians/lambda_n 45,
# weights 10, accumulation of both residuals 2 x 35, counts 2
OPS_PER_PIXEL = 165
# FP32 lanes x SMs x maximum SM clock of GB300 (the recipe's unit counts and clock)
ALU_PEAK_GOPS = 128 * 152 * 2.07


def alu_roofline(kernel: str, units_per_launch: float, ms_per_launch: float) -> dict:
    achieved = OPS_PER_PIXEL * units_per_launch / (ms_per_launch / 1000.0) / 1e9 if ms_per_launch > 0 else 0.0
    return {"bound": "alu", "kernel": kernel, "ops_per_unit": OPS_PER_PIXEL, "achieved": achieved,
            "peak": ALU_PEAK_GOPS, "peak_kind": "nominal (128 FP32 lanes x 152 SMs x 2.07 GHz)",
            "unit": "Gop/s", "frac": achieved / ALU_PEAK_GOPS}


# DRAM bytes (read + write) per unit (level pixel for the sweep, sample pixel for
# the robust-scale kernel, level pixel x iteration for the level kernel) from one ncu
# capture of each kernel on this workload (the sweep and robust-scale kernels at
# level 0, the level kernel's 80x60 launch, the one it gets in a frame; cold caches);
# set to None whenever those kernels change.
TRAFFIC_PER_UNIT = {"robust_kernel": None, "sweep_kernel": 4847616 / 307200,
                    "level_kernel": 169472 / (4800 * 10), "split_kernel": None}


# ----------------------------------------------------------------------------- ranks
def ranks_from_env():
    """(rank, world size, local rank) from the launcher's environment; one process: (0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_ranks(world: int, backend: str, device=None):
    """The process group when world > 1, else None.  Every rank works on its own,
    independent data (weak scaling); the group carries only the barriers around the
    timed region and the timing reduction, never data."""
    if world <= 1:
        return None
    import torch.distributed as dist
    kw = {"device_id": device} if device is not None else {}
    dist.init_process_group(backend, **kw)
    return dist


def max_over_ranks(values, dist, device) -> list:
    """Each timing's maximum over the ranks: the slowest rank bounds the whole job."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / (ms / 1000.0)


def pose_err(Ta, Tb):
    """(rotation angle, translation norm) of Ta^-1 Tb.  The angle is
    atan2(|axial part|, (tr - 1)/2) of the relative rotation, which stays exact
    for tiny angles; arccos((tr - 1)/2) alone turns a 1e-10 departure from
    orthonormality of an FP64 pose into ~1e-5 rad."""
    import numpy as np
    E = np.linalg.inv(np.asarray(Ta, dtype=np.float64)) @ np.asarray(Tb, dtype=np.float64)
    Rm = E[:3, :3]
    ax = 0.5 * np.array([Rm[2, 1] - Rm[1, 2], Rm[0, 2] - Rm[2, 0], Rm[1, 0] - Rm[0, 1]])
    ang = float(np.arctan2(np.linalg.norm(ax), 0.5 * (np.trace(Rm) - 1.0)))
    return ang, float(np.linalg.norm(E[:3, 3]))


GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden(name: str):
    """A stored oracle result (written by the scripts beside it, which call only the
    oracle), or None when absent."""
    try:
        with open(os.path.join(GOLDEN, name)) as f:
            return json.load(f)
    except OSError:
        return None


def err_stats(errs) -> dict:
    import numpy as np
    e = np.asarray(errs, dtype=np.float64).reshape(-1, 2)
    return {"n": int(e.shape[0]), "max_rad": float(e[:, 0].max()), "p99_rad": float(np.percentile(e[:, 0], 99)),
            "max_m": float(e[:, 1].max()), "p99_m": float(np.percentile(e[:, 1], 99))}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=240)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extensions", action="store_true",
                    help="leave out the batched, bf16 and learned forms that the default line summarises")
    ap.add_argument("--workload", choices=["sequence", "batch", "learned"], default="sequence",
                    help="sequence: the 640x480 tracking sequence (default); batch: 64 uneven loop-closure "
                         "pairs in one persistent launch; learned: held-out 640x480 pairs with the learned "
                         "start against the plain start")
    ap.add_argument("--precision", choices=["f32", "bf16"], default="f32",
                    help="plane storage: f32, or the reduced-precision form (bf16 I, fp16 W)")
    ap.add_argument("--no-level-kernel", action="store_true",
                    help="run every level by the per-iteration kernels (no persistent level kernel)")
    ap.add_argument("--keyframes", choices=["every20", "covisibility"], default="every20",
                    help="sequence workload: a new keyframe every 20 frames (default), or when the dense covisibility "
                         "ratio of the aligned frame with the keyframe falls below 0.7 (decided on the device)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------- CPU baseline
CPU_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O
from paper_1807_08271_gb300 import synth
seq = synth.render_sequence(0, n_frames={N})
if {warm} > 0:      # untimed warm-up: the same tracker over the first frames
    O.track_sequence(seq["I"], seq["W"], seq["K"], levels={levels}, iters={iters}, kf_every={kf},
                     n_frames={warm} + 1, reduced={reduced})
t0 = time.perf_counter()
r = O.track_sequence(seq["I"], seq["W"], seq["K"], levels={levels}, iters={iters}, kf_every={kf}, n_frames={nf},
                     reduced={reduced})
dt = time.perf_counter() - t0
print(json.dumps({{"frames": {nf} - 1, "seconds": dt, "T_world": r["T_world"].tolist()}}))
"""


def run_oracle_sample(n_frames: int, reduced: bool = False, warmup: int = 0) -> dict:
    """Time the FP64 oracle (one thread) on frames 0..n_frames-1 of the sequence, after
    `warmup` untimed frames of the same tracker."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    code = CPU_SNIPPET.format(root=ROOT, N=N_FRAMES, nf=n_frames, levels=LEVELS, iters=tuple(ITERS), kf=KF_EVERY,
                              reduced=reduced, warm=int(warmup))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------- reference arm
def reference(args):
    if ranks_from_env()[0] != 0:      # rank 0 alone runs the reference arm
        return
    n_timed = max(1, min(args.steps, 24))
    n_warm = max(3, min(args.warmup, 8))
    r = run_oracle_sample(n_timed + 1, reduced=(args.precision == "bf16"), warmup=n_warm)
    value = r["frames"] / r["seconds"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": r["frames"], "warmup": n_warm, "ms_per_step": 1000.0 * r["seconds"] / r["frames"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict("oracle frames 1..%d of the sequence" % r["frames"],
                                                    precision=args.precision),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"frames 1..{r['frames']} of the 300-frame sequence after {n_warm} untimed "
                                   "warm-up frames, one thread (numpy float64)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


KF_COVISIBILITY = 0.7


def config_dict(extra=None, precision="f32", keyframes="every20"):
    kf = ("keyframe every 20 frames" if keyframes == "every20" else
          f"new keyframe when the covisibility ratio with it falls below {KF_COVISIBILITY}")
    d = {"workload": "synthetic 640x480 room sequence, 300 frames at 30 Hz; frame-to-keyframe alignment on a "
                     f"4-level pyramid [10,5,5,5] iterations, fusion of every frame, {kf}",
         "width": W, "height": H, "levels": LEVELS, "iters_fine_to_coarse": list(ITERS),
         "frames": N_FRAMES, "keyframes": kf,
         "precision": ("plain FP32 planes" if precision == "f32" else
                       "bf16 intensity / fp16 inverse-depth planes, FP32 residuals, compensated FP32 sums, "
                       "FP32 Cholesky refined by one FP64 step, FP64 pose update"),
         "l2": "flushed between steps (512 MiB write), outside the timed intervals",
         "e2e": "each frame copied from pinned host memory into one of the tracker's two staging slots; frame k+1's "
                "copy runs on a copy stream during frame k, inside frame k's timed interval (gated on its start)"}
    if extra:
        d["note"] = extra
    return d


# ----------------------------------------------------------------------------- native arm
def native(args):
    import numpy as np
    import torch

    from paper_1807_08271_gb300 import rgbid as R
    from paper_1807_08271_gb300 import synth
    from paper_1807_08271_gb300.tracker import Tracker

    rank, world, local = ranks_from_env()
    torch.cuda.set_device(local)
    dist = init_ranks(world, "nccl", torch.device("cuda", local))

    seq = synth.render_sequence(seed=rank, n_frames=N_FRAMES)
    dev = torch.device("cuda", local)
    I_all = torch.from_numpy(seq["I"]).to(dev)
    W_all = torch.from_numpy(seq["W"]).to(dev)
    K = seq["K"]
    I_host = torch.from_numpy(seq["I"]).pin_memory()
    W_host = torch.from_numpy(seq["W"]).pin_memory()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    per_step_launches = sum(ITERS[:LEVELS])
    # the robust-scale kernel is timed live over the device-resident steps, the
    # sweep kernel over the end-to-end steps (one kernel per timed region)
    timer_robust = R.KernelTimer(R.KERNEL_ROBUST, (per_step_launches + 1) * max(1, min(args.steps, 60)) + 8)
    timer_sweep = R.KernelTimer(R.KERNEL_SWEEP, per_step_launches * max(1, min(args.steps, 60)) + 8)
    timer_level = R.KernelTimer(R.KERNEL_LEVEL, LEVELS * max(1, min(args.steps, 60)) + 8)
    timer_split = R.KernelTimer(R.KERNEL_SPLIT, LEVELS * max(1, min(args.steps, 60)) + 8)
    prec = R.PLANES_BF16_F16 if args.precision == "bf16" else R.PLANES_F32
    bytes_per_unit = BYTES_PER_UNIT[args.precision]
    covis = KF_COVISIBILITY if args.keyframes == "covisibility" else None
    trk = Tracker(W, H, K, levels=LEVELS, iters=ITERS, kf_every=KF_EVERY, max_frames=N_FRAMES + 1, device=dev,
                  precision=prec, kf_covisibility=covis, level_kernel=not args.no_level_kernel)
    align_launches = None      # known once the first frame has built the pyramids

    launches = {"n": 0}

    def kernels_in_step(k):
        # frame pyramid (one launch, every level) + predict + the alignment (init, two
        # per iteration or one level kernel per level, the closing reduction) + kf
        # pyramid, and then fuse, or switch (compose + init_kf), or with the
        # covisibility policy: covisibility + decision + fuse-or-switch
        n = 1 + 1 + align_launches + 1
        if covis is not None:
            return n + 3
        n += 2 if k % KF_EVERY == 0 else 1
        return n

    state = {"frame": 0}

    def next_frame():
        """Frame index for the next step; a new pass restarts tracking at frame 0."""
        if state["frame"] >= N_FRAMES:
            state["frame"] = 0
        if state["frame"] == 0:
            trk.k = 0
            with torch.cuda.stream(stream):
                trk.step(I_all[0], W_all[0], stream)
            state["frame"] = 1
        k = state["frame"]
        state["frame"] += 1
        return k

    def peek_next():
        """The frame index the next call of next_frame() returns."""
        f = state["frame"]
        if f >= N_FRAMES:
            f = 0
        return 1 if f == 0 else f

    # Every pass feeds the tracker through its two staging slots: frame k+1 is copied
    # on a copy stream into the slot it will read while frame k runs, gated on frame
    # k's start, so every copy lies inside a timed interval and none overlaps the L2
    # flush between steps; frame k+1 waits for its copy.  The device-resident pass
    # copies from the sequence held in HBM, the end-to-end pass from pinned host
    # memory (and reads each frame's result back to pinned host memory).
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    pipe = {"slot": 0, "ready": None}   # ready: (frame, slot, source) uploaded ahead

    def run_steps(n, timed, e2e=False, res_host=None):
        evs = []
        src_I, src_W = (I_host, W_host) if e2e else (I_all, W_all)
        for _ in range(n):
            k = next_frame()
            with torch.cuda.stream(stream):
                if timed:
                    flush.fill_(rank & 0xff)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                gate = torch.cuda.Event()
                gate.record(stream)          # the previous frame is done reading the other slot
                slot = pipe["slot"]
                SI, SW = trk.staging(slot)
                if pipe["ready"] == (k, slot, e2e):
                    stream.wait_event(copied[slot])
                else:
                    SI.copy_(src_I[k], non_blocking=True)
                    SW.copy_(src_W[k], non_blocking=True)
                trk.step(SI, SW, stream)
                nk, other = peek_next(), slot ^ 1
                copy_stream.wait_event(gate)
                with torch.cuda.stream(copy_stream):
                    OI, OW = trk.staging(other)
                    OI.copy_(src_I[nk], non_blocking=True)
                    OW.copy_(src_W[nk], non_blocking=True)
                    copied[other].record(copy_stream)
                pipe["slot"], pipe["ready"] = other, (nk, other, e2e)
                if e2e:
                    res_host.copy_(trk.res[0], non_blocking=True)
                if timed:
                    e1.record(stream)
                    evs.append((e0, e1))
                    launches["n"] += kernels_in_step(k)
        return evs

    # warm-up (also builds the library on first use and captures the frame graphs)
    run_steps(args.warmup, timed=False)
    torch.cuda.synchronize()
    align_launches = trk.align_launches()
    level_kernels = align_launches < 2 * per_step_launches + 2
    pipe["ready"] = None      # the first timed frame uploads inside its own interval

    # ---- device-resident timed region (no per-launch events: they would break the
    #      programmatic dependent launches between the kernels)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    evs = run_steps(args.steps, timed=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(sum(step_ms))
    gpu_launches = launches["n"]

    # ---- end-to-end through host buffers (no per-launch events either)
    res_host = torch.empty(R.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    run_steps(2, timed=False, e2e=True, res_host=res_host)
    pipe["ready"] = None      # the first timed frame uploads inside its own interval
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    evs2 = run_steps(args.steps, timed=True, e2e=True, res_host=res_host)
    torch.cuda.synchronize()
    e2e_ms = float(sum(a.elapsed_time(b) for a, b in evs2))

    # ---- the two alignment kernels timed live, each over its own pass of device-resident
    #      steps (CUDA events around every launch of that kernel on the tracker's stream)
    kern = {}
    n_kern = max(1, min(args.steps, 60))
    timed_kernels = [("robust_kernel", timer_robust), ("sweep_kernel", timer_sweep)]
    if level_kernels:
        timed_kernels += [("level_kernel", timer_level), ("split_kernel", timer_split)]
    for name, timer in timed_kernels:
        timer.reset()
        timer.attach(trk.params)
        evk = run_steps(n_kern, timed=True)
        torch.cuda.synchronize()
        trk.params.timing = None
        kern[name] = (timer.total_ms(), int(timer.t.units), int(timer.t.count),
                      float(sum(a.elapsed_time(b) for a, b in evk)))
    launches["n"] = gpu_launches

    # pose sanity: frames of the last pass vs ground truth
    traj = trk.trajectory()
    n_ok = trk.k
    rot = max((pose_err(seq["T_wc"][0] @ traj[i], seq["T_wc"][i])[0] for i in range(1, n_ok)), default=0.0)

    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], dist, dev)
    if rank != 0:
        dist.destroy_process_group()
        return
    value = whole_job_rate(world, args.steps, total_ms)
    e2e_val = whole_job_rate(world, args.steps, e2e_ms)
    peak, peak_kind = measured_peaks()
    rooflines = {}
    for name, (k_ms, k_units, k_count, region_ms) in kern.items():
        if k_count == 0:
            continue                                     # a kernel this configuration does not launch
        alg_bytes = bytes_per_unit * k_units             # 16 B (FP32 planes) or 8 B (bf16/fp16) per unit
        achieved = alg_bytes / (k_ms / 1000.0) / 1e9 if k_ms > 0 else 0.0
        rooflines[name] = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                           "unit": "GB/s", "frac": achieved / peak if peak else None,
                           "traffic": (TRAFFIC_PER_UNIT[name] * k_units / max(k_count, 1)
                                       if args.precision == "f32" and TRAFFIC_PER_UNIT.get(name) is not None
                                       else None),
                           "launches": k_count, "units_per_launch": k_units / max(k_count, 1),
                           "avg_launch_us": 1000.0 * k_ms / max(k_count, 1),
                           "share_of_step": k_ms / region_ms if region_ms else None}
    dominant = max(rooflines, key=lambda n: rooflines[n]["share_of_step"] or 0.0)
    # the kernel that evaluates every pixel of the finest level (the ALU roofline's)
    pixel_kernel = "sweep_kernel" if "sweep_kernel" in rooflines else "split_kernel"
    roofline = rooflines[dominant]
    others = {n: r for n, r in rooflines.items() if n != dominant}
    cpu = None
    if not args.no_cpu_baseline:
        n_cmp = 7
        r = run_oracle_sample(n_cmp, reduced=(args.precision == "bf16"))
        cpu = {"value": r["frames"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"frames 1..{r['frames']} of the sequence (align + fuse), one thread, numpy float64"
                         + (", bf16/fp16-rounded pyramids" if args.precision == "bf16" else ""),
               "host": host_info()}
    # every frame of a fresh GPU pass over the whole sequence against the FP64 oracle's
    # tracking of it (stored; seed 0): alignment poses kf_T_k and world poses
    pose_check = None
    gold = golden("seq640_oracle.json" if covis is None else "seq640_covis_oracle.json")
    if gold is not None and rank == 0:
        n_chk = N_FRAMES if covis is None else len(gold["fp32_planes"]["frames"]) + 1
        chk = Tracker(W, H, K, levels=LEVELS, iters=ITERS, kf_every=KF_EVERY, max_frames=n_chk, device=dev,
                      precision=prec, kf_covisibility=covis, level_kernel=not args.no_level_kernel)
        for k in range(n_chk):
            chk.step(I_all[k], W_all[k])
        torch.cuda.synchronize()
        gT, gr = chk.trajectory(), chk.frame_results()
        pose_check = {"frames": f"1..{n_chk - 1}",
                      "status": sorted(set(int(x["status"]) for x in gr)),
                      "max_rot_err_vs_truth_rad": max(pose_err(seq["T_wc"][0] @ gT[k], seq["T_wc"][k])[0]
                                                      for k in range(n_chk))}
        if covis is not None:
            fr = gold["fp32_planes"]["frames"]
            flags = chk.keyframe_flags()[1:]
            pose_check["keyframe_switches"] = [int(k) + 1 for k in np.argwhere(flags).ravel()]
            pose_check["switches_equal_oracle"] = bool(np.array_equal(flags, [f["switch"] for f in fr]))
            pose_check["max_covisibility_diff"] = float(np.max(np.abs(chk.covisibility_ratios()
                                                                      - [f["covisibility"] for f in fr])))
        planes = (("reduced_planes", "fp32_planes") if args.precision == "bf16" else ("fp32_planes",))
        if covis is not None:
            planes = ("fp32_planes",) if args.precision == "f32" else ()
        for name in planes:
            fr = gold[name]["frames"]
            pose_check[f"alignment_vs_oracle_{name}"] = err_stats(
                [pose_err(np.array(o["T"]).reshape(4, 4), x["T"]) for o, x in zip(fr, gr)])
            pose_check[f"world_vs_oracle_{name}"] = err_stats(
                [pose_err(np.array(o["T_world"]).reshape(4, 4), gT[o["k"]]) for o in fr])
        pose_check["oracle"] = ("stored FP64 oracle tracking of this sequence (tests/golden/"
                                + ("seq640_oracle.json)" if covis is None else "seq640_covis_oracle.json)"))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(precision=args.precision, keyframes=args.keyframes),
        "level_kernel": level_kernels, "align_launches_per_frame": align_launches,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * W * H * 4,
                "d2h_bytes_per_step": R.RESULT_BYTES},
        "roofline": roofline, "roofline_other_kernels": others,
        "alu_roofline": alu_roofline(pixel_kernel, rooflines[pixel_kernel]["units_per_launch"],
                                     rooflines[pixel_kernel]["avg_launch_us"] / 1000.0),
        "cpu_baseline": cpu, "clocks": clk, "gpu_launches": gpu_launches,
        "wall_s_timed": t_wall, "max_rot_err_vs_truth_rad": rot, "pose_check": pose_check,
    }
    if world == 1 and args.precision == "f32" and args.keyframes == "every20" and not args.no_extensions:
        line["extensions"] = run_extensions(args)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- extensions
EXTENSION_RUNS = {
    # name: (arguments, summary keys taken from the form's own line)
    "batched": (["--workload", "batch", "--steps", "120"], ("per_pair_form",)),
    "batched_bf16": (["--workload", "batch", "--precision", "bf16", "--steps", "120"], ("per_pair_form",)),
    "precision_bf16": (["--precision", "bf16", "--steps", "120"], ()),
    "keyframes_by_covisibility": (["--keyframes", "covisibility", "--steps", "120"], ()),
    "learned": (["--workload", "learned", "--steps", "256"], ("per_pair", "batched", "equal_accuracy")),
}


def run_extensions(args) -> dict:
    """The batched, reduced-precision and learned forms, each measured by its own
    run of this script on the same GPU (one line each, no CPU baseline, no nested
    extensions), summarised under the default line so that every form's throughput,
    roofline, pose check and clocks come from the same command."""
    out = {}
    for name, (extra, keys) in EXTENSION_RUNS.items():
        cmd = [sys.executable, os.path.abspath(__file__), "--no-cpu-baseline", "--no-extensions",
               "--warmup", str(max(3, args.warmup))] + extra
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            d = json.loads(r.stdout.strip().splitlines()[-1])
        except (subprocess.TimeoutExpired, ValueError, IndexError) as e:
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
            continue
        summ = {k: d.get(k) for k in ("metric", "value", "unit", "ms_per_step", "steps", "e2e", "roofline",
                                       "alu_roofline", "pose_check", "clocks", "gpu_launches")}
        summ["config"] = d.get("config")
        for k in keys:
            summ[k] = d.get(k)
        out[name] = summ
    return out


def host_info() -> dict:
    """Core count and CPU model of the host the CPU baseline ran on."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}

# ----------------------------------------------------------------------------- batched workload
BATCH_N = 64
BATCH_METRIC = "alignments/s of 64 uneven frame-keyframe pairs in one persistent launch (vs the per-pair form)"
BATCH_CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O
from paper_1807_08271_gb300 import synth
pairs = synth.make_batch(seed=0, n=4, sizes=synth.BATCH_SIZES)
t0 = time.perf_counter()
for p in pairs:
    A = O.build_pyramid{red}(p["I_A"], p["W_A"], p["K"], p["levels"])
    B = O.build_pyramid{red}(p["I_B"], p["W_B"], p["K"], p["levels"])
    O.align(A, B, p["T_init"], O.AlignParams(levels=p["levels"], iters=tuple(p["iters"])))
dt = time.perf_counter() - t0
print(json.dumps({{"alignments": len(pairs), "seconds": dt}}))
"""


BATCH_CPU_POOL_SNIPPET = r"""
import json, multiprocessing as mp, os, sys, time
sys.path.insert(0, {root!r})


def align(p):
    import oracle as O
    A = O.build_pyramid{red}(p["I_A"], p["W_A"], p["K"], p["levels"])
    B = O.build_pyramid{red}(p["I_B"], p["W_B"], p["K"], p["levels"])
    return O.align(A, B, p["T_init"], O.AlignParams(levels=p["levels"], iters=tuple(p["iters"])))["T"].tolist()


def ready(_):
    import oracle  # noqa: F401
    return os.getpid()


if __name__ == "__main__":
    from paper_1807_08271_gb300 import synth
    n = {n}
    pairs = synth.make_batch(seed=0, n=n, sizes=synth.BATCH_SIZES)
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map(ready, range(n))
        t0 = time.perf_counter()
        pool.map(align, pairs, chunksize=1)
        dt = time.perf_counter() - t0
    print(json.dumps({{"alignments": n, "seconds": dt, "processes": n}}))
"""


def run_oracle_batch_pool(reduced: bool = False) -> dict:
    """Time the FP64 oracle on all host cores: one spawned process per pair (one
    thread each; pairs are independent, so every pair's result is the one-thread
    oracle's), as many pairs as cores, an equal share of each resolution."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    n = max(4, 4 * ((os.cpu_count() or 4) // 4))
    code = BATCH_CPU_POOL_SNIPPET.format(root=ROOT, red="_reduced" if reduced else "", n=n)
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".py", prefix="rgbid_oracle_pool_")
    with os.fdopen(fd, "w") as f:
        f.write(code)
    try:
        out = subprocess.run([sys.executable, path], capture_output=True, text=True, env=env, check=True)
    finally:
        os.remove(path)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle_batch_sample(reduced: bool = False) -> dict:
    """Time the FP64 oracle (one thread) on one pair of each resolution of the batch."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    code = BATCH_CPU_SNIPPET.format(root=ROOT, red="_reduced" if reduced else "")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def batch_config_dict(precision="f32", shape=None):
    d = {"workload": "64 independent frame-keyframe pairs (loop-closure verification): 16 each at 320x240, "
                     "640x480, 960x720 and 1280x960, relative poses up to 10 deg / 20 cm, initial guess = truth "
                     "perturbed by up to 2 deg / 3 cm; levels 1 + floor(log2(w/80)), 10 iterations at the coarsest "
                     "level and 5 elsewhere; one persistent launch replayed from a CUDA graph",
         "pairs": BATCH_N,
         "precision": ("plain FP32 planes" if precision == "f32" else
                       "bf16 intensity / fp16 inverse-depth planes, FP32 residuals, compensated FP32 sums, "
                       "FP64 6x6 solve and update"),
         "l2": "flushed between steps (512 MiB write), outside the timed intervals"}
    if shape is not None:
        d["launch_shape"] = {"cluster": shape[0], "rows_per_warp": shape[1], "n_clusters": shape[2],
                             "chosen_by": "rgbid_batch_autotune"}
    return d


def reference_batch(args):
    if ranks_from_env()[0] != 0:      # rank 0 alone runs the reference arm
        return
    r = run_oracle_batch_pool(reduced=(args.precision == "bf16"))
    value = r["alignments"] / r["seconds"]
    sample = (f"{r['alignments']} pairs of the batch (an equal share of each resolution), one spawned process per "
              "pair on the host's cores, one thread each (numpy float64)")
    print(json.dumps({
        "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": 1000.0 * r["seconds"] / r["alignments"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": batch_config_dict(args.precision),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["processes"], "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def native_batch(args):
    import numpy as np
    import torch

    from paper_1807_08271_gb300 import rgbid as R
    from paper_1807_08271_gb300 import synth
    from paper_1807_08271_gb300.batch import BatchAligner

    rank, world, local = ranks_from_env()
    torch.cuda.set_device(local)
    dist = init_ranks(world, "nccl", torch.device("cuda", local))
    dev = torch.device("cuda", local)
    prec = R.PLANES_BF16_F16 if args.precision == "bf16" else R.PLANES_F32
    pairs = synth.make_batch(seed=rank, n=BATCH_N)

    # device-resident inputs (level-0 planes) and their pyramids; pinned host copies for e2e
    planes, host, pyr, items = [], [], [], []
    for p in pairs:
        w, h = p["width"], p["height"]
        ent = []
        for key in ("I_A", "W_A", "I_B", "W_B"):
            ent.append(torch.from_numpy(p[key]).to(dev))
            host.append(torch.from_numpy(p[key]).pin_memory())
        planes.append(ent)
        PA = R.DevicePyramid(w, h, p["levels"], prec, device=dev).build(ent[0], ent[1], p["K"])
        PB = R.DevicePyramid(w, h, p["levels"], prec, device=dev).build(ent[2], ent[3], p["K"])
        pyr.append((PA, PB))
        items.append(dict(ref=PA.desc, cur=PB.desc, T_init=p["T_init"], levels=p["levels"], iters=p["iters"]))
    B = BatchAligner(items, precision=prec, device=dev)
    B.tune(reps=3)
    shape = B.config.as_tuple()
    B.capture()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # pixel evaluations of one batch (the sweep's units): sum over pairs and levels of w_l h_l iters_l
    units = 0
    for p in pairs:
        for l in range(p["levels"]):
            units += (p["width"] >> l) * (p["height"] >> l) * p["iters"][l]
    bytes_per_unit = BYTES_PER_UNIT[args.precision]

    for _ in range(max(3, args.warmup)):
        B.replay()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(rank & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.replay()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    total_ms = float(sum(a.elapsed_time(b) for a, b in evs))

    # end to end: every step copies all 64 pairs' level-0 planes from pinned host memory,
    # rebuilds the 128 pyramids (same storage, so the item table stays valid), aligns the
    # batch and reads the 64 result records back
    res_host = torch.empty_like(B.results, device="cpu").pin_memory()

    def e2e_step():
        for i in range(len(pairs)):
            for j in range(4):
                planes[i][j].copy_(host[4 * i + j], non_blocking=True)
            p = pairs[i]
            pyr[i][0].build(planes[i][0], planes[i][1], p["K"])
            pyr[i][1].build(planes[i][2], planes[i][3], p["K"])
        B.replay()
        res_host.copy_(B.results, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    evs2 = []
    for _ in range(max(1, args.steps // 4)):
        flush.fill_(rank & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        evs2.append((e0, e1))
    torch.cuda.synchronize()
    e2e_ms = float(np.mean([a.elapsed_time(b) for a, b in evs2]))
    h2d = sum(int(t.numel()) * 4 for t in host)

    # the per-pair form on the same batch (one rgbid_align per pair), and pose agreement
    res_b = B.all_results()
    ps = [R.rgbid_default_params(levels=p["levels"], iters=p["iters"]) for p in pairs]
    wss = [R.new_workspace(pyr[i][0].desc, ps[i], device=dev) for i in range(len(pairs))]
    rs = [R.result_tensor(device=dev) for _ in pairs]

    def plain_pass():
        for i, p in enumerate(pairs):
            R.rgbid_align(pyr[i][0].desc, pyr[i][1].desc, p["T_init"], ps[i], wss[i], rs[i])

    plain_pass()
    torch.cuda.synchronize()
    plain_ms = []
    for _ in range(3):
        flush.fill_(rank & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain_pass()
        e1.record(stream)
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    res_p = [R.parse_result(r) for r in rs]

    d_plain = [pose_err(a["T"], b["T"]) for a, b in zip(res_b, res_p)]
    d_truth = [pose_err(a["T"], p["T_gt"])[0] for a, p in zip(res_b, pairs)]
    # against the FP64 oracle's alignment of every pair of this batch (seed 0 only)
    gold = golden("c3_oracle_poses_reduced.json" if args.precision == "bf16" else "c3_oracle_poses.json")
    d_oracle = None
    if gold is not None and rank == 0:
        d_oracle = [pose_err(np.array(gold["pairs"][str(i)]["T"]).reshape(4, 4), r["T"]) for i, r in enumerate(res_b)]
        d_oracle_pp = [pose_err(np.array(gold["pairs"][str(i)]["T"]).reshape(4, 4), r["T"]) for i, r in enumerate(res_p)]

    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], dist, dev)
    if rank != 0:
        dist.destroy_process_group()
        return
    step_ms = total_ms / args.steps
    value = whole_job_rate(world, BATCH_N * args.steps, total_ms)
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_unit * units / (step_ms / 1000.0) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        r = run_oracle_batch_sample(reduced=(args.precision == "bf16"))
        cpu = {"value": r["alignments"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one pair of each resolution (320x240, 640x480, 960x720, 1280x960), one thread, "
                         "numpy float64", "host": host_info()}
        rp = run_oracle_batch_pool(reduced=(args.precision == "bf16"))
        cpu["all_cores"] = {"value": rp["alignments"] / rp["seconds"], "unit": UNIT, "cores": rp["processes"],
                            "sample": f"{rp['alignments']} pairs, one spawned process per pair, one thread each"}
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": batch_config_dict(args.precision, shape),
        "e2e": {"value": whole_job_rate(world, BATCH_N, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(B.results.numel())},
        "roofline": {"bound": "hbm", "kernel": "batch_align_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "launches": args.steps, "units_per_launch": units,
                     "avg_launch_us": 1000.0 * step_ms},
        "alu_roofline": alu_roofline("batch_align_kernel", units, step_ms),
        "per_pair_form": {"value": BATCH_N / (float(np.median(plain_ms)) / 1000.0), "unit": UNIT,
                          "ms_per_batch": float(np.median(plain_ms))},
        "pose_check": {"max_vs_per_pair_form_rad": max(d[0] for d in d_plain),
                       "max_vs_per_pair_form_m": max(d[1] for d in d_plain),
                       "batched_vs_oracle": err_stats(d_oracle) if d_oracle else None,
                       "per_pair_form_vs_oracle": err_stats(d_oracle_pp) if d_oracle else None,
                       "oracle": ("stored FP64 oracle poses of every pair (tests/golden/"
                                  + ("c3_oracle_poses_reduced.json, reduced-precision pyramids)" if args.precision == "bf16"
                                     else "c3_oracle_poses.json)")) if d_oracle else None,
                       "median_vs_truth_rad": float(np.median(d_truth)), "max_vs_truth_rad": float(np.max(d_truth)),
                       "status": sorted(set(r["status"] for r in res_b))},
        "cpu_baseline": cpu, "clocks": clk, "gpu_launches": args.steps, "wall_s_timed": t_wall,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- learned-start workload
LEARNED_N = 512
LEARNED_METRIC = ("640x480 alignments/s with the learned start (per pair) at equal or better convergence than "
                  "the plain start")
LEARNED_CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O
from paper_1807_08271_gb300 import synth
pairs = [synth.make_pair(s, 640, 480, K=(525.0, 525.0, 319.5, 239.5), max_angle_deg=10.0, max_trans=0.15)
         for s in (11, 12)]
t0 = time.perf_counter()
for p in pairs:
    A = O.build_pyramid(p["I_A"], p["W_A"], p["K"], 4)
    B = O.build_pyramid(p["I_B"], p["W_B"], p["K"], 4)
    O.align(A, B, None, O.AlignParams(levels=4, iters=(5, 5, 5, 10)))
dt = time.perf_counter() - t0
print(json.dumps({{"alignments": len(pairs), "seconds": dt}}))
"""


def run_oracle_learned_sample() -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    out = subprocess.run([sys.executable, "-c", LEARNED_CPU_SNIPPET.format(root=ROOT)], capture_output=True,
                         text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def learned_config_dict(meta=None):
    d = {"workload": f"{LEARNED_N} held-out synthetic 640x480 pairs (object scenes, textures unseen in training), "
                     "relative poses up to 10 deg / 15 cm, no motion prior: the plain start is the identity with "
                     "the 4-level [10,5,5,5] schedule; the learned start is the network's proposal with the "
                     "coarsest level(s) skipped by confidence tier (plain otherwise)",
         "pairs": LEARNED_N, "converged": "final pose within 2 mrad / 5 mm of the plain method's pose started at "
                                          "the ground truth",
         "l2": "not flushed: each alignment's pyramids (3.3 MB) are read 15-25 times per alignment by design"}
    if meta:
        d["network"] = {k: meta.get(k) for k in ("train_pairs", "epochs", "thresholds")}
    return d


def reference_learned(args):
    if ranks_from_env()[0] != 0:      # rank 0 alone runs the reference arm
        return
    r = run_oracle_learned_sample()
    value = r["alignments"] / r["seconds"]
    print(json.dumps({
        "impl": "reference", "metric": LEARNED_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": 1000.0 * r["seconds"] / r["alignments"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": learned_config_dict(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "two 640x480 pairs aligned from the identity (plain schedule), one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def native_learned(args):
    import numpy as np
    import torch

    from paper_1807_08271_gb300 import rgbid as R
    from paper_1807_08271_gb300 import synth
    from paper_1807_08271_gb300 import learned as Lm
    from paper_1807_08271_gb300.learned_train import EvalSet, pose_diff, _sized
    from paper_1807_08271_gb300.synth import gpu as G

    rank, world, local = ranks_from_env()
    torch.cuda.set_device(local)
    dist = init_ranks(world, "nccl", torch.device("cuda", local))
    net = Lm.InitNet.load(Lm.WEIGHTS, max_batch=LEARNED_N)
    thr = net.meta["thresholds"]
    bank = G.TextureBank(4242 + rank, n=16)
    ev = EvalSet(9001 + rank, LEARNED_N, bank, 10.0, 0.15)
    n_steps = max(1, min(args.steps, LEARNED_N))

    # per-pair forms: one alignment per step, timed with CUDA events on the stream
    params = R.rgbid_default_params(levels=4, iters=[5, 5, 5, 10])
    ws = R.new_workspace(ev.pyr[0][0].desc, params)
    res = R.result_tensor(LEARNED_N)
    la = Lm.LearnedAligner(_sized(net, 1), thr, levels=4, iters=[5, 5, 5, 10])
    la.set_pairs([(a.desc, b.desc) for a, b in ev.pyr])
    # the kernel of the two finest levels (the split kernel; the per-iteration sweep where
    # the device cannot schedule it): most of a learned-start alignment's time
    timed_name = "split_kernel"
    timer = R.KernelTimer(R.KERNEL_SPLIT, 25 * n_steps + 8)
    stream = torch.cuda.current_stream()

    def run(kind, k, timed=False):
        if kind == "plain":
            R.rgbid_align(ev.pyr[k][0].desc, ev.pyr[k][1].desc, None, params, ws, res[k])
        else:
            la.align(k, ws, res[k])

    out = {}
    clk = None
    kept = {}
    for kind in ("plain", "learned"):
        for k in range(max(3, args.warmup)):
            run(kind, k)
        torch.cuda.synchronize()
        if kind == "learned":
            clocks = ClockSampler(local)
            clocks.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(n_steps):
            run(kind, k)
        e1.record(stream)
        torch.cuda.synchronize()
        if kind == "learned":
            clk = clocks.stop()
        rr = [R.parse_result(res[k]) for k in range(n_steps)]
        kept[kind] = rr
        ok = ev.converged(rr)
        out[kind] = dict(ms=e0.elapsed_time(e1), converged=float(np.mean(ok)),
                         iters=float(np.mean([r["iters_done"] for r in rr])),
                         median_err=float(np.median([pose_diff(r["T"], ev.T_gt[k])[0] for k, r in enumerate(rr)])))
    # that kernel timed live over a separate pass (events around each launch add their own
    # cost, so the timed value above runs without them)
    for _ in range(2):
        timer.attach(la.params)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(n_steps):
            run("learned", k)
        e1.record(stream)
        torch.cuda.synchronize()
        la.params.timing = None
        timer_region_ms = e0.elapsed_time(e1)
        if int(timer.t.count) > 0 or timed_name == "sweep_kernel":
            break
        timed_name, timer = "sweep_kernel", R.KernelTimer(R.KERNEL_SWEEP, 25 * n_steps + 8)

    # end to end (learned): each step copies the pair's four planes from pinned host memory,
    # rebuilds both pyramids in place and reads the result record back
    res_host = torch.empty(R.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    d = G.make_pairs_gpu(9001 + rank, n_steps, bank, 640, 480, 10.0, 0.15)
    I_h, W_h = d["I"].cpu().pin_memory(), d["W"].cpu().pin_memory()
    I_d, W_d = torch.empty_like(d["I"][0]), torch.empty_like(d["W"][0])
    PA = R.DevicePyramid(640, 480, 4).build(I_d[0], W_d[0], d["K"])
    PB = R.DevicePyramid(640, 480, 4).build(I_d[1], W_d[1], d["K"])
    la_e = Lm.LearnedAligner(_sized(net, 1), thr, levels=4, iters=[5, 5, 5, 10])
    la_e.set_pairs([(PA.desc, PB.desc)])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(n_steps):
        I_d.copy_(I_h[k], non_blocking=True)
        W_d.copy_(W_h[k], non_blocking=True)
        PA.build(I_d[0], W_d[0], d["K"])
        PB.build(I_d[1], W_d[1], d["K"])
        la_e.align(0, ws, res[0])
        res_host.copy_(res[0], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    # the metric's own criterion: the learned start's final pose within 1e-5 rad and
    # 1e-5 m of the plain form's (identity start, all levels), pair by pair
    def agreement(a, b):
        d = np.array([pose_err(x["T"], y["T"]) for x, y in zip(a, b)])
        return {"pairs": int(d.shape[0]), "within_1e-5_rad_and_m": float(np.mean((d[:, 0] <= 1e-5) & (d[:, 1] <= 1e-5))),
                "median_rad": float(np.median(d[:, 0])), "median_m": float(np.median(d[:, 1]))}

    agree_10deg = agreement(kept["learned"], kept["plain"])

    # held-out pairs shaped like the tracking workload: frames 20 j + d of another
    # seeded room sequence aligned to frame 20 j (d = 1..19), identity start
    seq1 = synth.render_sequence(seed=1 + rank, n_frames=81)
    c1_pairs = [(20 * j, 20 * j + d) for j in range(4) for d in range(1, 20)]
    pyr_c1 = {}
    for f in sorted({i for pr in c1_pairs for i in pr}):
        pyr_c1[f] = R.DevicePyramid(640, 480, 4).build(torch.from_numpy(seq1["I"][f]).cuda(),
                                                        torch.from_numpy(seq1["W"][f]).cuda(), seq1["K"])
    la_c1 = Lm.LearnedAligner(_sized(net, 1), thr, levels=4, iters=[5, 5, 5, 10])
    la_c1.set_pairs([(pyr_c1[a].desc, pyr_c1[b].desc) for a, b in c1_pairs])
    res_c1 = {k: R.result_tensor(len(c1_pairs)) for k in ("plain", "learned")}
    c1 = {}
    for kind in ("plain", "learned", "plain", "learned"):      # the second round is timed
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, (a_, b_) in enumerate(c1_pairs):
            if kind == "plain":
                R.rgbid_align(pyr_c1[a_].desc, pyr_c1[b_].desc, None, params, ws, res_c1[kind][i])
            else:
                la_c1.align(i, ws, res_c1[kind][i])
        e1.record(stream)
        torch.cuda.synchronize()
        rr = [R.parse_result(res_c1[kind][i]) for i in range(len(c1_pairs))]
        c1[kind] = {"alignments_per_s": len(c1_pairs) / (e0.elapsed_time(e1) / 1000.0),
                    "mean_iterations": float(np.mean([r["iters_done"] for r in rr])), "results": rr}
    gt = [np.linalg.inv(seq1["T_wc"][a_]) @ seq1["T_wc"][b_] for a_, b_ in c1_pairs]
    c1_summary = {kind: {"alignments_per_s": v["alignments_per_s"], "mean_iterations": v["mean_iterations"],
                         "median_rot_err_vs_truth_rad": float(np.median([pose_err(r["T"], g)[0]
                                                                         for r, g in zip(v["results"], gt)]))}
                  for kind, v in c1.items()}
    c1_summary["learned_vs_plain"] = agreement(c1["learned"]["results"], c1["plain"]["results"])
    c1_summary["pairs"] = ("frame 20 j + d of the seeded 640x480 room sequence (seed 1) aligned to frame 20 j, "
                           "j = 0..3, d = 1..19, identity start")

    # the batched forms on the whole held-out set (one persistent launch each)
    res_p, ms_p, _ = ev.run(None, reps=5)
    from paper_1807_08271_gb300.learned import LearnedPlanner
    res_l, ms_l, _ = ev.run(lambda m, prec: LearnedPlanner(_sized(net, m), m, prec, thr), reps=5)

    learned_ms, e2e_ms = max_over_ranks([out["learned"]["ms"], e2e_ms], dist, "cuda")
    if rank != 0:
        dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    k_ms, k_units, k_count = timer.total_ms(), int(timer.t.units), int(timer.t.count)
    achieved = BYTES_PER_UNIT["f32"] * k_units / (k_ms / 1000.0) / 1e9 if k_ms > 0 else 0.0
    cpu = None
    if not args.no_cpu_baseline:
        r = run_oracle_learned_sample()
        cpu = {"value": r["alignments"] / r["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "two 640x480 pairs aligned from the identity with the plain schedule, one thread, "
                         "numpy float64"}
    line = {
        "metric": LEARNED_METRIC, "value": whole_job_rate(world, n_steps, learned_ms), "unit": UNIT, "n_gpus": world,
        "steps": n_steps, "warmup": max(3, args.warmup), "ms_per_step": learned_ms / n_steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 alignment, bf16 network",
        "data": "synthetic", "config": learned_config_dict(net.meta),
        "e2e": {"value": whole_job_rate(world, n_steps, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": 4 * 640 * 480 * 4, "d2h_bytes_per_step": R.RESULT_BYTES},
        "roofline": {"bound": "hbm", "kernel": timed_name, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "traffic": None, "launches": k_count, "units_per_launch": k_units / max(k_count, 1),
                     "avg_launch_us": 1000.0 * k_ms / max(k_count, 1), "share_of_step": k_ms / timer_region_ms},
        "per_pair": {kind: {"alignments_per_s": n_steps / (v["ms"] / 1000.0), "converged_fraction": v["converged"],
                            "mean_iterations": v["iters"], "median_rot_err_vs_truth_rad": v["median_err"]}
                     for kind, v in out.items()},
        "equal_accuracy": {"criterion": "learned-start pose within 1e-5 rad and 1e-5 m of the plain form's",
                           "held_out_10deg": agree_10deg, "tracking_like_pairs": c1_summary},
        "batched": {"plain_alignments_per_s": LEARNED_N / (ms_p / 1000.0),
                    "learned_alignments_per_s": LEARNED_N / (ms_l / 1000.0),
                    "plain_converged": float(np.mean(ev.converged(res_p))),
                    "learned_converged": float(np.mean(ev.converged(res_l)))},
        # per learned alignment: input packing, bf16 weights, 6 GEMMs and the split-K reductions
        # of the five that split at batch 1, the plan, then the alignment's launches (a skipped
        # level's launch included)
        "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": n_steps * (14 + R.rgbid_align_launches(ev.pyr[0][0].desc, la.params)),
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.workload == "batch":
        (reference_batch if args.impl == "reference" else native_batch)(args)
    elif args.workload == "learned":
        (reference_learned if args.impl == "reference" else native_learned)(args)
    elif args.impl == "reference":
        reference(args)
    else:
        native(args)


if __name__ == "__main__":
    main()
