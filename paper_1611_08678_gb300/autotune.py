"""Autotuner of the batched path's launch shapes.

The kernels expose two shape knobs (include/abm.h, abm_plan_opts):
  near_warps : warps per state component in the near kernel, the chain warp
               plus helpers summing slices of the next step's window while the
               chain runs: 1 (chain only), 2 or 3 - FP64 latency per step
               against instruction count when many column tiles share an SM
  far_split  : how far the tensor-core far kernel may split each column
               tile's history across CTAs: at most far_split times the waves
               of the unsplit launch (the parts are added on the device)
The tuner times a full batched solve (CUDA events, after one warm-up) for
each candidate and keeps the fastest.  Results are cached in a JSON file
keyed by GPU, system, precision and the workload's shape buckets, so a later
plan for the same shape starts from the tuned values without re-timing.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Dict, Iterable, List, Optional, Tuple

import numpy as np

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = tuple(
    (nw, fs) for nw in (1, 2, 3) for fs in (1, 2, 4))
_lock = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("ABM_GB300_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache")), "abm_gb300")
    return os.path.join(base, "autotune.json")


def shape_key(gpu: str, system: str, prec: str, M: int, N, alpha) -> str:
    """Bucketed description of a batched workload (powers of two)."""
    N = np.asarray(N)
    b = lambda x: int(2 ** math.ceil(math.log2(max(int(x), 1))))
    return "|".join([gpu, system, prec, f"M{b(M)}", f"Nmax{b(N.max())}", f"Nmin{b(N.min())}",
                     f"groups{len(np.unique(np.asarray(alpha)))}"])


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def store_cache(key: str, entry: dict, path: Optional[str] = None) -> None:
    path = path or cache_path()
    with _lock:
        data = load_cache(path)
        data[key] = entry
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def select(timings: Iterable[Tuple[Tuple[int, int], float]]) -> Tuple[int, int]:
    """Fastest candidate; ties go to the earlier candidate."""
    best, best_ms = None, float("inf")
    for cand, ms in timings:
        if ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        raise ValueError("no timings")
    return best


def tune(time_fn: Callable[[int, int], float], candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES):
    """Times every candidate with time_fn(near_warps, far_split) -> ms and
    returns (best, [(candidate, ms), ...])."""
    results: List[Tuple[Tuple[int, int], float]] = []
    for cand in candidates:
        results.append((cand, float(time_fn(*cand))))
    return select(results), results


def tune_batched(batch, prec: str, candidates=DEFAULT_CANDIDATES, use_cache: bool = True,
                 cache: Optional[str] = None) -> dict:
    """Tunes (near_warps, far_split) for one batched workload on the current GPU.
    Returns {"near_warps", "far_split", "ms", "results", "key", "cached"}."""
    import torch

    from . import abm
    gpu = torch.cuda.get_device_name()
    key = shape_key(gpu, batch.system, prec, batch.M, batch.N, batch.alpha)
    if use_cache:
        hit = load_cache(cache).get(key)
        if hit:
            return dict(hit, key=key, cached=True)
    params = torch.as_tensor(batch.params, device="cuda")
    y0 = torch.as_tensor(batch.y0, device="cuda")
    ldY = int(batch.N.max()) + 1
    Y = torch.empty(batch.M, ldY, batch.d, dtype=torch.float64, device="cuda")

    def time_fn(nw: int, fs: int) -> float:
        plan = abm.Plan(batch.system, n_max=int(batch.N.max()), max_batch=batch.M, prec=prec,
                        near_warps=nw, far_split=fs)
        try:
            plan.solve_batched(batch.alpha, batch.h, batch.N, params, y0, Y=Y, ldY=ldY)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.solve_batched(batch.alpha, batch.h, batch.N, params, y0, Y=Y, ldY=ldY, sync=False)
            e1.record()
            plan.sync()
            return e0.elapsed_time(e1)
        finally:
            plan.close()

    (nw, fs), results = tune(time_fn, candidates)
    entry = {"near_warps": nw, "far_split": fs, "ms": dict(results)[(nw, fs)],
             "results": [[list(c), ms] for c, ms in results]}
    if use_cache:
        store_cache(key, entry, cache)
    return dict(entry, key=key, cached=False)
