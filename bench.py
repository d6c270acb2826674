#!/usr/bin/env python
"""Benchmark of the forward delay-and-sum pass (paper Sec. 2, Eq. 2).

Workload (default): 128^3 voxels x 1024 elements x 16 diverging-wave
transmits, complex IQ channel data with 2048 samples, 20 frames per step
(seeded speckle + point phantom), float32 storage and sums.  A step is one
das_forward call on the 20 frames: relayout of the channel data plus the DAS
kernel.  The inputs (5.4 GB) are larger than L2, so no flush is needed.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead,
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "volumes/s, forward DAS at 128^3 voxels x 1024 elements x 16 transmits (IQ, float32)"


def metric_for(storage: str, tensor_cores: bool) -> str:
    """The metric text of a paper-workload line: the storage and path it ran."""
    if storage == "f32" and not tensor_cores:
        return METRIC
    path = ", tensor cores" if tensor_cores else ""
    return METRIC.replace("(IQ, float32)", f"(IQ, {storage} storage{path})")
FP32_LANES_PER_SM = 128


def sm_count(device=0) -> int:
    """Streaming multiprocessors of the device (cudaDevAttrMultiProcessorCount)."""
    import torch

    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def fp32_peak_tflops(sm_max_mhz: float, device=0) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flop x the maximum SM clock."""
    return sm_count(device) * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["paper", "batched", "table1", "diff"], default="paper",
                    help="paper: the 128^3 x 1024 x 16 forward; batched: three uneven plans, 64 frames, one "
                         "launch; table1: the paper's Table 1 configuration (B 128, Q 1, K 256)")
    ap.add_argument("--frames", type=int, default=20)
    ap.add_argument("--K", type=int, default=2048, help="samples per channel (all delays lie below 400)")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16", "e4m3", "e5m2"], default="f32")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--staging", action="store_true", help="stage sample windows in shared memory (bulk copies)")
    ap.add_argument("--load-width", type=int, default=0, choices=[0, 128, 256], help="bits per lane of each load")
    ap.add_argument("--fb", type=int, default=0, help="frames per thread (0: automatic)")
    ap.add_argument("--adj-rows", type=int, default=0, help="sample rows per adjoint CTA (0: automatic)")
    ap.add_argument("--vpt", type=int, default=0, choices=[0, 1, 2],
                    help="voxels per thread of the float32 IQ kernel (0: automatic = 1)")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="forward pass as the tcgen05 tile contraction (f16 / bf16 storage)")
    ap.add_argument("--ctas", type=int, default=0, help="CTAs per SM of the tensor-core kernel (0: automatic)")
    ap.add_argument("--tc-chain", type=int, default=0,
                    help="MMA sub-items per tensor-memory accumulation chain (0: automatic, -1: one per tile)")
    return ap.parse_args()


def huge_page_fraction(t) -> "float | None":
    """Share of a host tensor's resident pages that are transparent huge pages
    (from /proc/self/smaps), None where unreadable."""
    lo, hi = t.data_ptr(), t.data_ptr() + t.numel() * t.element_size()
    rss = huge = 0
    try:
        cur = False
        with open("/proc/self/smaps") as f:
            for line in f:
                head = line.split()
                if "-" in head[0] and len(head) >= 5:
                    a, b = (int(v, 16) for v in head[0].split("-"))
                    cur = a < hi and b > lo
                elif cur and head[0] == "Rss:":
                    rss += int(head[1])
                elif cur and head[0] == "AnonHugePages:":
                    huge += int(head[1])
    except (OSError, ValueError, IndexError):
        return None
    return huge / rss if rss else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def apply_tuning(plan, args) -> None:
    if args.tensor_cores:
        plan.set_tuning(tensor_cores=True, ctas_per_sm=args.ctas, tc_chain=args.tc_chain)
    elif args.staging or args.fb or args.load_width or args.vpt:
        plan.set_tuning(frames_per_thread=args.fb, staging=args.staging, load_width=args.load_width,
                        voxels_per_thread=args.vpt)


def tensor_roofline(plan, items0: int, launches: int, kern_ms: float, storage: str, profile: str,
                    useful_flops: float, work_text: str, items1: "int | None" = None) -> dict:
    """Tensor-pipe roofline of the tcgen05 kernel.  `frac` counts the method's
    work (contributing terms x frames x 16 flop, the complex two-tap
    interpolation and rotation of Eq. 2) over the kernel's event time against
    the measured sustained dense bf16 (= f16) rate.  The MMA flops the kernel
    issues (sub-items x 2 x 128 x N x 32, counted by the kernel between the
    counter readings items0 and items1, the timed launches) include the zero
    rows of each weight window and the padded columns of N; they are reported
    beside it as `mma_issue_frac`."""
    peaks, src = measured_peaks()
    info = plan.info()
    items = ((info["tc_mma_items"] if items1 is None else items1) - items0) / max(launches, 1)
    n = info["tc_mma_n"]
    issued = items * 2.0 * 128 * n * 32
    achieved = useful_flops / (kern_ms * 1e-3) / 1e12
    issued_t = issued / (kern_ms * 1e-3) / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": profiled_traffic(storage, profile, TC_SOURCES),
            "kernel": "tc_kernel (tcgen05 tile contraction)", "kernel_ms": kern_ms,
            "peak_source": f"{src} dense bf16 sustained (f16 runs at the same rate)",
            "work_per_launch": work_text,
            "mma_issue_tflops": issued_t, "mma_issue_frac": issued_t / peak,
            "mma_issued_per_launch": f"{items:.0f} MMA sub-items x 128 x {n} x 32 x 2 flop",
            "dense_to_useful": issued / useful_flops if useful_flops else None}


TILE_SOURCES = ("das_tile.cuh", "das_tile_tma.cuh", "das_tile_f32.cu", "das_internal.cuh")
PAIR_SOURCES = ("das_tile_pair.cuh", "das_tile_pair.cu", "das_tile.cuh", "das_internal.cuh")
TC_SOURCES = ("das_tc.cu", "das_tc.cuh", "das_async.cuh", "das_internal.cuh")


def kernel_source_hash(files=TILE_SOURCES) -> str:
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2606_13259_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(storage: str, name: str = "tile_kernel_paper_iq", files=TILE_SOURCES):
    """DRAM bytes per launch of a kernel from its committed ncu summary
    (profiles/<name>_<storage>.md), if that summary was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{name}_{storage}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha1:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_source_hash(files):
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_seed(rank: int) -> int:
    """Each rank beamforms its own independent frames (weak scaling)."""
    return 2 + 100000 * rank


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the step time)."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def make_inputs(frames: int, rank: int, device, K: int = 2048):
    from paper_2606_13259_gb300 import synth as S

    sc = S.scene_paper(K)
    y = S.frames(sc, frames, seed=rank_seed(rank), n_speckle=20000, points=S.paper_points(sc), device=device)
    return sc, y


def cpu_baseline(sc, y_cpu, frames: int, target_s: float):
    """The FP64 oracle, as it stands, on a bounded voxel sample of the workload."""
    import numpy as np

    from oracle import oracle as O

    O.build()
    rng = np.random.default_rng(123)
    probe = rng.choice(sc.N, 32, replace=False)
    t0 = time.perf_counter()
    O.forward(sc, y_cpu, voxels=probe)
    dt = time.perf_counter() - t0
    n = int(max(32, min(sc.N, 32 * target_s / max(dt, 1e-6))))
    vox = rng.choice(sc.N, n, replace=False)
    t0 = time.perf_counter()
    O.forward(sc, y_cpu, voxels=vox)
    dt = time.perf_counter() - t0
    volumes = frames * n / sc.N
    return {"value": volumes / dt, "unit": "volumes/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n} random voxels x {frames} frames of the workload ({n / sc.N:.2%} of each volume), "
                      f"{dt:.1f} s, float64, OpenMP over voxels"}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores."""
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    sc, y = make_inputs(args.frames, 0, dev, args.K)
    y_cpu = y.cpu().numpy()
    del y
    from oracle import oracle as O

    O.build()
    rng = np.random.default_rng(7)
    probe = rng.choice(sc.N, 16, replace=False)
    t0 = time.perf_counter()
    O.forward(sc, y_cpu, voxels=probe)
    per_voxel = (time.perf_counter() - t0) / 16
    budget = 150.0 / max(1, args.steps + args.warmup)
    n = int(max(16, min(sc.N, budget / max(per_voxel, 1e-9))))
    for _ in range(args.warmup):
        O.forward(sc, y_cpu, voxels=rng.choice(sc.N, n, replace=False))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.forward(sc, y_cpu, voxels=rng.choice(sc.N, n, replace=False))
    dt = (time.perf_counter() - t0) / args.steps
    value = args.frames * n / sc.N / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "volumes/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": sc.name, "frames_per_step": args.frames, "voxels": sc.N, "elements": sc.M,
                   "transmits": sc.Q, "samples": sc.K, "sample_per_step_voxels": n},
        "cpu_baseline": {"value": value, "unit": "volumes/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{n} random voxels x {args.frames} frames per step"},
        "e2e": {"value": value, "unit": "volumes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Batched form: 64 FP16 IQ frames drawn from three uneven plans (frame f
    belongs to plan f mod 3), all in one persistent launch replayed from a CUDA
    graph, launch shape from the autotuner."""
    import torch

    from paper_2606_13259_gb300 import Batch, Plan, autotune
    from paper_2606_13259_gb300 import build as B
    from paper_2606_13259_gb300 import synth as S

    torch.cuda.set_device(0)
    B.build()
    scenes = S.scenes_batched()
    total = 64
    frames = [len(range(i, total, 3)) for i in range(3)]
    ys = [S.frames(sc, f, seed=4 + 100000 * i, n_speckle=20000, points=S.paper_points(sc), device="cuda")
          for i, (sc, f) in enumerate(zip(scenes, frames))]
    plans = [Plan.from_scene(sc, storage=args.storage if args.storage != "f32" else "f16", max_batch=f)
             for sc, f in zip(scenes, frames)]
    batch = Batch(plans, frames)
    outs = [torch.empty((f,) + p.shape, dtype=torch.complex64, device="cuda") for p, f in zip(plans, frames)]
    tuned = autotune.tune_batch(batch, ys, outs, reps=2)
    for _ in range(args.warmup):
        batch.forward(ys, outs)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        batch.forward(ys, outs)
    e1.record(s)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    for p in plans:
        p.check()
    info = batch.info()
    # each plan alone, for reference (own launches, own tuned shape)
    alone = []
    for p, y, o in zip(plans, ys, outs):
        autotune.tune_plan(p, y, o, reps=2)
        t = autotune._time(lambda: p.forward(y, o), max(2, args.steps // 2), 1)
        alone.append(y.shape[0] / (t * 1e-3))
    actives = [p.count_active() for p in plans]
    flops = sum(a * f * 16.0 for a, f in zip(actives, frames))
    sm_max = float(measured_peaks()[0].get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_peak_tflops(sm_max)
    line = {
        "metric": "volumes/s, batched forward DAS over 3 uneven plans in one persistent launch (FP16 IQ storage)",
        "value": total / (ms * 1e-3), "unit": "volumes/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16 storage, f32 arithmetic", "data": "synthetic",
        "config": {"workload": "batched_3plans_64frames",
                   "plans": [dict(sc.describe(), frames=f) for sc, f in zip(scenes, frames)],
                   "tuning": {k: tuned.get(k) for k in ("frames_per_thread", "ctas_per_sm", "staging",
                                                         "plan_tensor_cores")},
                   "work_items": info["work_items"]},
        "per_plan_volumes_per_s_in_batch": [f / (ms * 1e-3) for f in frames],
        "per_plan_volumes_per_s_alone": alone,
        "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": flops / (ms * 1e-3) / 1e12 / fp32_peak, "traffic": None,
                     "note": "whole graph time (relayouts + persistent kernel)"},
        "gpu_launches": info["kernels_per_launch"] * args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()


def run_table1(args):
    """The paper's Table 1 configuration: 128 frames, 32x32 elements at pitch
    lambda, 128^3 voxels at lambda / 2, one observation, 256 IQ samples."""
    import torch

    from paper_2606_13259_gb300 import Plan
    from paper_2606_13259_gb300 import build as B
    from paper_2606_13259_gb300 import synth as S

    torch.cuda.set_device(0)
    B.build()
    sc = S.scene_table1()
    F = 128
    y = S.frames(sc, F, seed=6, n_speckle=4000, points=S.paper_points(sc), device="cuda")
    plan = Plan.from_scene(sc, storage=args.storage, max_batch=F)
    apply_tuning(plan, args)
    out = torch.empty((F,) + plan.shape, dtype=torch.complex64, device="cuda")
    active = plan.count_active()
    for _ in range(args.warmup):
        plan.forward(y, out)
    torch.cuda.synchronize()
    items0 = plan.info()["tc_mma_items"]
    plan.enable_timing(args.steps)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        plan.forward(y, out)
    e1.record(s)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    plan.check()
    ms = e0.elapsed_time(e1) / args.steps
    kms, kn = plan.timing()
    kern_ms = kms / max(kn, 1)
    sm_max = float(measured_peaks()[0].get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_peak_tflops(sm_max)
    flops = active * F * 16.0
    work = f"{active} contributing terms x {F} frames x 16 flop"
    line = {
        "metric": "volumes/s, forward DAS in the paper's Table 1 configuration (B 128, M 1024, Q 1, K 256, N 128^3)",
        "value": F / (ms * 1e-3), "unit": "volumes/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.storage + " storage, f32 arithmetic", "data": "synthetic",
        "config": {"workload": sc.name, "frames_per_step": F, "scene": sc.describe()},
        "roofline": tensor_roofline(plan, items0, kn, kern_ms, args.storage, "tc_kernel_table1", flops, work)
        if args.tensor_cores else
        {"bound": "alu", "achieved": flops / (kern_ms * 1e-3) / 1e12, "peak": fp32_peak,
         "unit": "TFLOP/s", "frac": flops / (kern_ms * 1e-3) / 1e12 / fp32_peak, "traffic": None,
         "kernel_ms": kern_ms},
        "tensor_cores": bool(args.tensor_cores),
        **({"tc_chain": args.tc_chain or "auto"} if args.tensor_cores else {}),
        "gpu_launches": None, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    plan.close()


def run_diff(args):
    """Differentiation form: 96^3 voxels x 1024 elements x 8 transmits, IQ,
    1536 samples, one frame.  A step is the forward pass, the adjoint of an
    image-space cotangent and the sound-speed derivative (what a gradient
    step of an autofocus loop costs)."""
    import torch

    from paper_2606_13259_gb300 import Plan
    from paper_2606_13259_gb300 import build as B
    from paper_2606_13259_gb300 import synth as S

    torch.cuda.set_device(0)
    B.build()
    sc = S.scene_diff(c=1500.0)
    y = S.frames(sc, 1, seed=5, n_speckle=20000, points=S.paper_points(sc), c=1540.0, device="cuda")
    g = S.random_image(sc, 1, seed=12).cuda().reshape((1, sc.nz, sc.ny, sc.nx))
    plan = Plan.from_scene(sc)
    if args.adj_rows:
        plan.set_tuning(adjoint_rows=args.adj_rows)
    x = torch.empty((1,) + plan.shape, dtype=torch.complex64, device="cuda")
    ya = torch.empty_like(y)
    dc = torch.empty((), dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(args.steps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    t_fwd = timed(lambda: plan.forward(y, x))
    t_adj = timed(lambda: plan.adjoint(g, ya))
    t_dc = timed(lambda: plan.grad_c(y, g, dc))
    clocks = sampler.stop()
    plan.check()
    active = plan.count_active()
    step = t_fwd + t_adj + t_dc
    line = {
        "metric": "differentiation steps/s (forward + adjoint + dL/dc) at 96^3 voxels x 1024 elements x 8 transmits",
        "value": 1e3 / step, "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": sc.name, "frames": 1, "scene": sc.describe(),
                                        "adjoint_rows": args.adj_rows or "auto"},
        "ms": {"forward": t_fwd, "adjoint": t_adj, "grad_c": t_dc},
        "terms_per_ms": {"forward": active / t_fwd, "adjoint": active / t_adj, "grad_c": active / t_dc},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    plan.close()


def main():
    args = parse_args()
    if args.workload == "diff":
        return run_diff(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "table1":
        return run_table1(args)
    import torch

    from paper_2606_13259_gb300 import Plan
    from paper_2606_13259_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())

    sc, y = make_inputs(args.frames, rank, dev, args.K)
    F = args.frames
    plan = Plan.from_scene(sc, storage=args.storage, max_batch=F)
    apply_tuning(plan, args)
    out = torch.empty((F,) + plan.shape, dtype=torch.complex64, device=dev)
    active = plan.count_active()

    for _ in range(args.warmup):
        plan.forward(y, out)
    torch.cuda.synchronize()
    items0 = plan.info()["tc_mma_items"]
    plan.enable_timing(args.steps)
    launches0 = plan.info()["kernel_launches"]
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        plan.forward(y, out)
    e1.record(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1) / args.steps
    plan.check()
    kern_ms_total, kern_n = plan.timing()
    kern_ms = kern_ms_total / max(kern_n, 1)
    info1 = plan.info()
    launches = info1["kernel_launches"] - launches0
    items1 = info1["tc_mma_items"]  # MMA sub-items of the timed launches (the e2e calls below add more)
    ms, kern_ms = max_over_ranks([ms, kern_ms], dist, dev)

    # end to end through the C-ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        from paper_2606_13259_gb300 import host_empty

        y_host = host_empty(y.shape, y.dtype)  # page-locked huge pages (das_host_alloc)
        y_host.copy_(y)
        # one output buffer per step: every step copies its input in and its image out
        n_e2e = max(5, min(args.steps, 10))
        x_hosts = [host_empty(out.shape, out.dtype) for _ in range(n_e2e)]
        x_host = x_hosts[0]
        plan.forward_host(y_host, x_host)
        plan.forward_host_many([y_host] * 2, x_hosts[:2])  # staging slots allocated outside the timing
        # single host call per step (copies, then the forward pass, then the image back)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            plan.forward_host(y_host, x_hosts[i])
        dt_serial = (time.perf_counter() - t0) / n_e2e
        # the steps as one sequence call: step i + 1's input copy and step i - 1's
        # image copy run during step i's forward pass
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        plan.forward_host_many([y_host] * n_e2e, x_hosts)
        dt = (time.perf_counter() - t0) / n_e2e
        # host_io = 2: the kernels read the channel data from, and write the
        # image to, the page-locked host buffers directly (no copy engines)
        plan.set_tuning(host_io=2, tensor_cores=args.tensor_cores, ctas_per_sm=args.ctas, tc_chain=args.tc_chain,
                        frames_per_thread=args.fb, staging=args.staging, load_width=args.load_width,
                        voxels_per_thread=args.vpt)
        plan.forward_host_many([y_host] * 2, x_hosts[:2])
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        plan.forward_host_many([y_host] * n_e2e, x_hosts)
        dt_direct = (time.perf_counter() - t0) / n_e2e
        plan.set_tuning(host_io=0, tensor_cores=args.tensor_cores, ctas_per_sm=args.ctas, tc_chain=args.tc_chain,
                        frames_per_thread=args.fb, staging=args.staging, load_width=args.load_width,
                        voxels_per_thread=args.vpt)
        dt, dt_serial, dt_direct = max_over_ranks([dt, dt_serial, dt_direct], dist, dev)
        # the copy legs alone, for the record
        t1 = time.perf_counter()
        y.copy_(y_host, non_blocking=True)
        torch.cuda.synchronize()
        h2d = time.perf_counter() - t1
        t1 = time.perf_counter()
        x_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        d2h = time.perf_counter() - t1
        direct_wins = dt_direct < dt
        e2e = {"value": world * F / min(dt, dt_direct), "unit": "volumes/s", "h2d_bytes_per_step": y_host.numel() * 8,
               "d2h_bytes_per_step": x_host.numel() * 8, "ms_per_step": min(dt, dt_direct) * 1e3,
               "api": (f"das_forward_host_many with host_io = 2, {n_e2e} steps in one call (the relayout kernel "
                       f"reads the page-locked host input, the DAS kernel writes the host image)") if direct_wins
               else f"das_forward_host_many, {n_e2e} steps in one call (copies overlapped with forward passes)",
               "copies_value": world * F / dt, "direct_value": world * F / dt_direct,
               "choice": "the faster of the two host transfers of das_forward_host_many, both measured here",
               "serial_value": world * F / dt_serial, "serial_api": "das_forward_host, one call per step",
               "h2d_ms_torch_copy": h2d * 1e3, "d2h_ms_torch_copy": d2h * 1e3,
               "input_huge_page_fraction": huge_page_fraction(y_host)}
        del y_host, x_host, x_hosts

    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = sm_count(dev)
    fp32_peak = fp32_peak_tflops(sm_max, dev)
    flops = active * F * 16.0          # 8 FMA per contributing (voxel, element, transmit, frame) term
    work = f"{active} contributing terms x {F} frames x 16 flop"
    achieved = flops / (kern_ms * 1e-3) / 1e12
    bytes_store = {"f32": 8, "f16": 4, "bf16": 4, "e4m3": 2, "e5m2": 2}[args.storage]
    alg_bytes = sc.Q * sc.M * sc.K * F * bytes_store + F * sc.N * 8
    if args.tensor_cores:
        roof = tensor_roofline(plan, items0, kern_n, kern_ms, args.storage, "tc_kernel_paper_iq", flops, work,
                               items1)
        roof.update({"hbm_algorithmic_gbs": alg_bytes / (kern_ms * 1e-3) / 1e9, "sm_count": sms})
    else:
        roof = None
    # --vpt 2 runs the two-voxels-per-thread kernel (das_tile_pair.cuh)
    pair = (args.storage == "f32" and not args.tensor_cores and args.vpt == 2 and not args.staging
            and not args.load_width)
    roof = roof or {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "traffic": profiled_traffic(args.storage, "pair_kernel_paper_iq", PAIR_SOURCES) if pair
            else profiled_traffic(args.storage),
            "kernel": "pair_kernel (forward DAS, two voxels per thread)" if pair else "tile_kernel (forward DAS)",
            "kernel_ms": kern_ms,
            "peak_source": f"{sms} SMs (device attribute) x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                           f"({peak_src} max SM clock)",
            "hbm_algorithmic_gbs": alg_bytes / (kern_ms * 1e-3) / 1e9,
            "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)),
            "work_per_launch": work}

    line = {
        "metric": metric_for(args.storage, args.tensor_cores), "value": world * F / (ms * 1e-3), "unit": "volumes/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else args.storage,
        "data": "synthetic (seeded speckle + 10 point targets, time-domain simulator)",
        "config": {"workload": sc.name, "frames_per_step": F, "voxels": sc.N, "elements": sc.M,
                   "transmits": sc.Q, "samples": sc.K, "storage": args.storage,
                   "l2": f"inputs {y.numel() * 8 / 1e9:.1f} GB > 129 MB L2, no flush", "per_rank_frames": F,
                   "staging": args.staging,
                   "row_loads": f"row order, {args.load_width}-bit" if args.load_width else "column order, 128-bit",
                   "frames_per_thread": args.fb or "auto", "tensor_cores": bool(args.tensor_cores),
                   "voxels_per_thread": args.vpt or "auto",
                   **({"tc_chain": args.tc_chain or "auto"} if args.tensor_cores else {})},
        "accumulations_per_s": world * F * sc.N * sc.M * sc.Q / (ms * 1e-3),
        "accumulations_note": "accumulations_per_s counts the dense N x M x Q terms per volume (the paper's "
                              "3.4e10); contributing_terms_per_s counts those inside the f-number aperture and "
                              "the sample range, the work the roofline uses",
        "contributing_terms_per_volume": active,
        "contributing_terms_per_s": world * F * active / (ms * 1e-3),
        "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, y.cpu().numpy(), F, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
