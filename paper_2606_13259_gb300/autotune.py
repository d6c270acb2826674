"""Autotuner for the launch shape of the forward kernels.

Times every candidate (frames per thread, persistent CTAs per SM, staged or
global sample windows) on the caller's own data with CUDA events, keeps the
fastest and caches the choice in a JSON file keyed by the GPU name and a
signature of the workload (grid, elements, transmits, samples, frames, data
and storage types).  The cache lives at $DAS_TUNING_CACHE, else
~/.cache/paper_2606_13259_gb300/tuning.json.
"""
from __future__ import annotations

import json
import os
from typing import Iterable, Optional

import torch

from . import _lib as L
from .plan import Batch, Plan

F32_FB = (2, 4, 8, 12, 16, 20)
F16_FB = (4, 8, 12, 16, 20, 24)


def cache_path() -> str:
    return os.environ.get("DAS_TUNING_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2606_13259_gb300", "tuning.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    data = _load()
    data[key] = value
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _plan_sig(p: Plan) -> str:
    return f"{p.shape[2]}x{p.shape[1]}x{p.shape[0]}/M{p.M}/Q{p.Q}/K{p.K}/{'iq' if p.iq else 'rf'}/{p.storage}"


def _time(fn, reps: int, warmup: int) -> float:
    for _ in range(warmup):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _set_plan_tc(batch: Batch, flags) -> None:
    """Each plan on or off the tensor cores, its other settings kept."""
    for p, on in zip(batch.plans, flags):
        p.set_tuning(**dict(p.tuning(), tensor_cores=bool(on)))


def tune_batch(batch: Batch, ys, outs, fbs: Optional[Iterable[int]] = None,
               ctas: Iterable[int] = (0, 1, 2, 3), staging=(False, True), reps: int = 3, warmup: int = 1,
               use_cache: bool = True, tensor_cores: bool = True) -> dict:
    """Pick (frames per thread, CTAs per SM, staged windows) for a batch, and
    for each plan that can take them whether it runs on the tensor cores
    (greedily, heaviest plan first, each kept only if the whole batch gets
    faster); applies and returns it."""
    key = "batch:" + torch.cuda.get_device_name() + ":" + ";".join(
        f"{_plan_sig(p)}/B{f}" for p, f in zip(batch.plans, batch.frames))
    if use_cache:
        hit = _load().get(key)
        if hit:
            _set_plan_tc(batch, hit.get("plan_tensor_cores", [False] * len(batch.plans)))
            batch.set_tuning(hit["frames_per_thread"], hit["ctas_per_sm"], hit.get("staging", False))
            return dict(hit, cached=True)
    tc_flags = [False] * len(batch.plans)
    _set_plan_tc(batch, tc_flags)
    p0 = batch.plans[0]
    if fbs is None:
        fbs = F32_FB if p0.storage == "f32" else F16_FB
    results = []
    for fb in fbs:
        for c in ctas:
            for st in staging:
                try:
                    batch.set_tuning(fb, c, st)
                except L.DASError:
                    continue
                ms = _time(lambda: batch.forward(ys, outs), reps, warmup)
                results.append({"frames_per_thread": fb, "ctas_per_sm": c, "staging": st, "ms": ms})
    best = min(results, key=lambda r: r["ms"])
    batch.set_tuning(best["frames_per_thread"], best["ctas_per_sm"], best["staging"])
    best_ms = best["ms"]
    if tensor_cores:
        order = sorted(range(len(batch.plans)), key=lambda i: -batch.plans[i].M * batch.plans[i].Q * batch.frames[i])
        for i in order:
            p = batch.plans[i]
            if not (p.iq and p.storage in ("f16", "bf16")):
                continue
            trial = list(tc_flags)
            trial[i] = True
            _set_plan_tc(batch, trial)
            batch.set_tuning(best["frames_per_thread"], best["ctas_per_sm"], best["staging"])
            ms = _time(lambda: batch.forward(ys, outs), reps, warmup)
            results.append({"frames_per_thread": best["frames_per_thread"], "ctas_per_sm": best["ctas_per_sm"],
                            "staging": best["staging"], "plan_tensor_cores": trial, "ms": ms})
            if ms < best_ms:
                tc_flags, best_ms = trial, ms
        _set_plan_tc(batch, tc_flags)
        batch.set_tuning(best["frames_per_thread"], best["ctas_per_sm"], best["staging"])
    out = {"frames_per_thread": best["frames_per_thread"], "ctas_per_sm": best["ctas_per_sm"],
           "staging": best["staging"], "plan_tensor_cores": tc_flags, "ms": best_ms, "candidates": results}
    if use_cache:
        _store(key, out)
    return dict(out, cached=False)


_SHAPE_KEYS = ("frames_per_thread", "ctas_per_sm", "staging", "load_width", "tensor_cores")


def _apply(plan: Plan, cfg: dict) -> None:
    """The forward-kernel shape of `cfg`; the plan's other settings kept."""
    plan.set_tuning(**dict(plan.tuning(), **{k: cfg.get(k, plan.tuning()[k]) for k in _SHAPE_KEYS}))


def tune_plan(plan: Plan, y, out, fbs: Optional[Iterable[int]] = None, staging=(False, True),
              load_widths=(0, 128, 256), tensor_cores=(False, True), reps: int = 3, warmup: int = 1,
              use_cache: bool = True) -> dict:
    """Pick the forward kernel of single-plan calls: CUDA-core tile kernel
    (frames per thread, staged windows, row load: 0 column order, 128 / 256
    row order with that load width) or the tensor-core tile
    contraction (CTAs per SM), the latter for IQ plans with 16-bit storage."""
    B = y.shape[0]
    key = "plan:" + torch.cuda.get_device_name() + ":" + _plan_sig(plan) + f"/B{B}"
    if use_cache:
        hit = _load().get(key)
        if hit:
            _apply(plan, hit)
            return dict(hit, cached=True)
    if fbs is None:
        fbs = [f for f in ((1,) + (F32_FB if plan.storage == "f32" else F16_FB)) if f <= max(B, 1) * 2]
    results = []
    for fb in fbs:
        for st in staging:
            for lw in (load_widths if not st else (128,)):
                cfg = {"tensor_cores": False, "frames_per_thread": fb, "staging": st, "load_width": lw,
                       "ctas_per_sm": 0}
                try:
                    _apply(plan, cfg)
                except L.DASError:
                    continue
                results.append(dict(cfg, ms=_time(lambda: plan.forward(y, out), reps, warmup)))
    if True in tuple(tensor_cores) and plan.iq and plan.storage in ("f16", "bf16"):
        for ctas in (1, 2, 3, 4):
            cfg = {"tensor_cores": True, "frames_per_thread": 0, "staging": False, "load_width": 0,
                   "ctas_per_sm": ctas}
            try:
                _apply(plan, cfg)
            except L.DASError:
                continue
            results.append(dict(cfg, ms=_time(lambda: plan.forward(y, out), reps, warmup)))
    best = min(results, key=lambda r: r["ms"])
    _apply(plan, best)
    res = dict(best, candidates=results)
    if use_cache:
        _store(key, res)
    return dict(res, cached=False)
