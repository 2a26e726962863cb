"""Autotuner of the batched path's launch shapes.

The kernels expose three shape knobs (include/abm.h, abm_plan_opts):
  far_split  : how far the tensor-core far kernel may split each column
               tile's history (its K range) across CTAs: at most far_split
               times the waves of the unsplit launch (the parts are added on
               the device)
  near_warps : warps per state component in the near kernel, the chain warp
               plus helpers summing slices of the next step's lag window while
               the chain runs: 1 (chain only), 2 or 3 - FP64 latency per step
               against instruction count when many column tiles share an SM
  near_split : the near kernel's batch-tile width: a column tile's 32
               trajectories run in 1, 2, 4 or 8 CTAs (32, 16, 8 or 4
               trajectories per CTA), or 0 = chosen per time tile from the
               number of active tiles (8 or 4 CTAs when they fit on the SMs)
The time-tile length (64 steps) is fixed by the tensor-core operand layout
(one 64-row K block per time tile).  The tuner times a full batched solve
(CUDA events, after one warm-up, best of two) per candidate and keeps the
fastest.  With the default search it walks the knobs one at a time
(coordinate descent: far_split with the library's near defaults, then
near_warps, then near_split, each step keeping the best value so far),
which times 9 candidates instead of the 48 of the full grid; each knob is
judged by the summed launch times of the kernel it shapes (far_split by the
far kernel, the near knobs by the near kernel), which a full-solve time
would blur with the other kernel's run-to-run spread.  Results are cached in a JSON
file keyed by GPU, system, precision and the workload's shape buckets, so a
later plan for the same shape starts from the tuned values without
re-timing.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

KNOBS: Tuple[str, ...] = ("far_split", "near_warps", "near_split")
# values searched per knob, in the order the coordinate descent visits them;
# the first value of each is the starting point (the library's default rule)
SPACE: Dict[str, Tuple[int, ...]] = {
    "far_split": (2, 1, 4),
    "near_warps": (0, 1, 2, 3),
    "near_split": (0, 1, 4, 8),
}
# the full grid, for exhaustive tuning of small workloads
DEFAULT_CANDIDATES: Tuple[Tuple[int, int, int], ...] = tuple(
    (fs, nw, ns) for fs in SPACE["far_split"] for nw in SPACE["near_warps"] for ns in SPACE["near_split"])
_lock = threading.Lock()

Candidate = Tuple[int, int, int]  # (far_split, near_warps, near_split)


def cache_path() -> str:
    base = os.environ.get("ABM_GB300_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache")), "abm_gb300")
    return os.path.join(base, "autotune.json")


def shape_key(gpu: str, system: str, prec: str, M: int, N, alpha) -> str:
    """Bucketed description of a batched workload (powers of two)."""
    N = np.asarray(N)
    b = lambda x: int(2 ** math.ceil(math.log2(max(int(x), 1))))
    groups = len({tuple(np.atleast_1d(a)) for a in np.asarray(alpha).reshape(len(N), -1)})
    return "|".join([gpu, system, prec, f"M{b(M)}", f"Nmax{b(N.max())}", f"Nmin{b(N.min())}", f"groups{groups}",
                     "knobs3"])


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


def select(timings: Iterable[Tuple[Candidate, float]]) -> Candidate:
    """Fastest candidate; ties go to the earlier candidate."""
    best, best_ms = None, float("inf")
    for cand, ms in timings:
        if ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        raise ValueError("no timings")
    return best


def tune(time_fn: Callable[..., float], candidates: Iterable[Candidate] = DEFAULT_CANDIDATES):
    """Times every candidate with time_fn(far_split, near_warps, near_split) -> ms
    and returns (best, [(candidate, ms), ...])."""
    results: List[Tuple[Candidate, float]] = []
    for cand in candidates:
        results.append((tuple(cand), float(time_fn(*cand))))
    return select(results), results


def tune_descent(time_fn: Callable[..., object], space: Dict[str, Sequence[int]] = SPACE,
                 objective: Optional[Dict[str, str]] = None):
    """Coordinate descent over the knobs in KNOBS order: each knob's values are
    timed with the other knobs at their best values so far (a candidate timed
    before is not timed again).  time_fn returns the ms of a solve, or a dict
    of ms per part ({"total", "far", "near"}); objective[knob] names the part
    that decides that knob (default "total"), so a knob is judged by the
    kernel it shapes and not by the noise of the other.  Returns (best,
    [(candidate, ms of the total), ...])."""
    objective = objective or {}
    cur = {k: space[k][0] for k in KNOBS}
    seen: Dict[Candidate, dict] = {}
    order: List[Tuple[Candidate, float]] = []
    for knob in KNOBS:
        part = objective.get(knob, "total")
        trial = []
        for v in space[knob]:
            c = dict(cur, **{knob: v})
            cand = tuple(c[k] for k in KNOBS)
            if cand not in seen:
                r = time_fn(*cand)
                seen[cand] = r if isinstance(r, dict) else {"total": float(r)}
                order.append((cand, float(seen[cand]["total"])))
            trial.append((cand, float(seen[cand].get(part, seen[cand]["total"]))))
        best = select(trial)
        cur = dict(zip(KNOBS, best))
    return tuple(cur[k] for k in KNOBS), order


# the kernel each knob shapes: its summed launch times decide the knob
OBJECTIVE = {"far_split": "far", "near_warps": "near", "near_split": "near"}


def tune_batched(batch, prec: str, candidates=None, use_cache: bool = True, cache: Optional[str] = None) -> dict:
    """Tunes (far_split, near_warps, near_split) for one batched workload on the
    current GPU: coordinate descent by default, the given candidate list when
    one is passed.  Returns {"far_split", "near_warps", "near_split", "ms",
    "results", "key", "cached"}."""
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

    def time_parts(fs: int, nw: int, ns: int) -> dict:
        """Best of two timed solves after a warm-up: the whole solve and the
        summed far and near kernel times (CUDA events around every launch)."""
        plan = abm.Plan(batch.system, n_max=int(batch.N.max()), max_batch=batch.M, prec=prec,
                        near_warps=nw, far_split=fs, near_split=ns, profile=True)
        try:
            plan.solve_batched(batch.alpha, batch.h, batch.N, params, y0, Y=Y, ldY=ldY)  # warm-up
            best = None
            for _ in range(2):
                for k in abm.KERNEL_KINDS:
                    plan.kernel_times(k, reset=True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.solve_batched(batch.alpha, batch.h, batch.N, params, y0, Y=Y, ldY=ldY, sync=False)
                e1.record()
                plan.sync()
                r = {"total": e0.elapsed_time(e1), "far": plan.kernel_times("far")[1],
                     "near": plan.kernel_times("near")[1]}
                best = r if best is None else {k: min(best[k], r[k]) for k in r}
            return best
        finally:
            plan.close()

    if candidates is None:
        best, results = tune_descent(time_parts, objective=OBJECTIVE)
    else:
        best, results = tune(lambda *c: time_parts(*c)["total"], candidates)
    entry = dict(zip(KNOBS, best))
    entry.update({"ms": dict(results)[best], "results": [[list(c), ms] for c, ms in results]})
    if use_cache:
        store_cache(key, entry, cache)
    return dict(entry, key=key, cached=False)
