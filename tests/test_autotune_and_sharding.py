"""CPU tests of the host logic: autotuner selection and cache, benchmark
sharding of trajectories across ranks and the max-over-ranks timing
reduction (two gloo processes on the CPU)."""
import os
import tempfile

import numpy as np
import pytest

from paper_1611_08678_gb300 import autotune, workloads


def test_select_picks_fastest_and_breaks_ties_in_order():
    assert autotune.select([((1, 1, 0), 5.0), ((2, 1, 0), 3.0), ((4, 2, 0), 3.0)]) == (2, 1, 0)
    with pytest.raises(ValueError):
        autotune.select([])


def test_search_space_spans_tile_shapes():
    """The candidates cover the history split, the warps per component and
    the near kernel's batch-tile width (32, 16, 8 or 4 trajectories per CTA,
    or the per-time-tile rule)."""
    assert autotune.KNOBS == ("far_split", "near_warps", "near_split")
    assert set(autotune.SPACE["near_split"]) == {0, 1, 4, 8}
    assert set(autotune.SPACE["near_warps"]) >= {1, 2, 3}
    assert len(autotune.DEFAULT_CANDIDATES) == 3 * 4 * 4
    assert {c[2] for c in autotune.DEFAULT_CANDIDATES} == {0, 1, 4, 8}


def test_tune_times_every_candidate():
    seen = []

    def fake(fs, nw, ns):
        seen.append((fs, nw, ns))
        return 10.0 / max(nw, 1) + fs + (0 if ns == 8 else 1)  # fastest: most near warps, fs = 1, ns = 8

    best, results = autotune.tune(fake)
    assert best == (1, 3, 8)
    assert sorted(seen) == sorted(autotune.DEFAULT_CANDIDATES)
    assert len(results) == len(autotune.DEFAULT_CANDIDATES)


def test_descent_walks_one_knob_at_a_time():
    """Separable costs: coordinate descent finds the grid optimum with one
    timing per distinct candidate (3 + 4 + 4 values, two shared) and keeps
    each knob's best value while it varies the next."""
    seen = []
    cost = {"far_split": {2: 1.0, 1: 0.5, 4: 2.0}, "near_warps": {0: 3.0, 1: 2.0, 2: 1.0, 3: 1.5},
            "near_split": {0: 1.0, 1: 2.0, 4: 0.2, 8: 0.7}}

    def fake(fs, nw, ns):
        seen.append((fs, nw, ns))
        return cost["far_split"][fs] + cost["near_warps"][nw] + cost["near_split"][ns]

    best, results = autotune.tune_descent(fake)
    descent = list(seen)
    assert best == (1, 2, 4)
    full_best, _ = autotune.tune(fake)
    assert full_best == best
    seen = descent
    assert len(seen) == len(set(seen)) == len(results) == 3 + 3 + 3
    assert seen[:3] == [(2, 0, 0), (1, 0, 0), (4, 0, 0)]  # far split first, near knobs at the library rule
    assert all(c[0] == 1 for c in seen[3:]) and all(c[1] == 2 for c in seen[6:])


def test_descent_judges_each_knob_by_its_kernel():
    """With per-part timings, far_split follows the far kernel's time and the
    near knobs the near kernel's, even when the total says otherwise (noise
    in the other part)."""
    def fake(fs, nw, ns):
        far = {2: 10.0, 1: 9.0, 4: 11.0}[fs]
        near = {0: 5.0, 1: 4.0, 2: 4.5, 3: 6.0}[nw] + {0: 0.0, 1: 0.0, 4: 1.0, 8: 2.0}[ns]
        noise = 3.0 if (fs, nw, ns) == (1, 0, 0) else 0.0  # the total of the best far split is noisy
        return {"total": far + near + noise, "far": far, "near": near}

    best, results = autotune.tune_descent(fake, objective=autotune.OBJECTIVE)
    assert best == (1, 1, 0)
    assert all(isinstance(ms, float) for _, ms in results)


def test_cache_roundtrip_and_shape_key_buckets():
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sub", "tune.json")
        b = workloads.rossler_batched(M=300, n_lo=1000, n_hi=5000)
        k = autotune.shape_key("GB300", b.system, "bf16x6", b.M, b.N, b.alpha)
        assert "M512" in k and "Nmax8192" in k and "groups8" in k and "knobs3" in k
        # per-component orders count distinct tuples
        al = np.tile([[0.9, 1.1, 0.9]], (b.M, 1))
        al[::2] = 0.95
        assert "groups2" in autotune.shape_key("GB300", b.system, "fp64", b.M, b.N, al)
        autotune.store_cache(k, {"near_warps": 2, "far_split": 4, "near_split": 8, "ms": 1.5}, path)
        autotune.store_cache("other", {"near_warps": 1, "far_split": 1, "near_split": 0, "ms": 2.0}, path)
        c = autotune.load_cache(path)
        assert c[k]["near_warps"] == 2 and c[k]["far_split"] == 4 and c[k]["near_split"] == 8 and "other" in c


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = workloads.rossler_batched(M=100, n_lo=64, n_hi=256)
    idx = bench.shard_indices(w.M, rank, world)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    gathered = [None] * world
    dist.all_gather_object(gathered, idx.tolist())
    if rank == 0:
        out.put((t.item(), gathered))
    dist.destroy_process_group()


def test_batched_sharding_two_gloo_ranks():
    """Trajectories are split across ranks with no overlap and nothing left
    out; the timed region is the max over ranks."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tmax, shards = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 2.0
    allidx = sorted(shards[0] + shards[1])
    assert allidx == list(range(100)) and not set(shards[0]) & set(shards[1])
