"""Autotuner for the launch shapes of libsvlf (svlf_set_tuning).

It times a caller-supplied step function on the caller's own workload for a
set of candidate shapes, with CUDA events on the current stream, keeps the
fastest, and remembers it in a JSON cache keyed by the GPU and workload, so a
later run applies it without searching again. Shapes never change results.

The search is coordinate-wise: traversal shape first (steps between lane
refills, block size), then the tensor-core forward (tiles in flight per CTA,
form of the hidden-layer epilogue).
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional

import torch

from . import svlf

TRACE_CANDIDATES = [dict(trace_budget=b, trace_block=t) for b in (16, 32, 64, 128) for t in (128, 256)]
MLP_CANDIDATES = [dict(mlp_warpgroups=w, mlp_epilogue_batch=e) for w in (2, 3, 4) for e in (1, 2, 3)
                  if not (e == 2 and w > 3)]

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "svlf_autotune.json")


def _time(fn: Callable[[], None], repeats: int) -> float:
    fn()  # warm-up (also compiles nothing: all kernels are prebuilt)
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def device_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.major}{p.minor}|{p.multi_processor_count}"


def autotune(step: Callable[[], None], workload_key: str, repeats: int = 5,
             cache_path: Optional[str] = DEFAULT_CACHE, search: bool = True) -> Dict:
    """Pick launch shapes for `step` (a callable that runs the workload once).
    Returns {"tuning": {...}, "ms": best time, "searched": bool}."""
    key = f"{device_key()}|{workload_key}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if key in cache and not search:
        svlf.svlf_set_tuning(**cache[key]["tuning"])
        return dict(cache[key], searched=False)
    best = dict(svlf.svlf_get_tuning())
    best_ms = _time(step, repeats)
    for group in (TRACE_CANDIDATES, MLP_CANDIDATES):
        for cand in group:
            trial = dict(best, **cand)
            svlf.svlf_set_tuning(**trial)
            ms = _time(step, repeats)
            if ms < best_ms:
                best, best_ms = trial, ms
    svlf.svlf_set_tuning(**best)
    entry = {"tuning": best, "ms": best_ms}
    if cache_path:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache[key] = entry
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return dict(entry, searched=True)
