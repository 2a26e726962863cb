"""CPU tests of the host logic: autotuner selection and cache, benchmark
sharding of trajectories across ranks and the max-over-ranks timing
reduction (two gloo processes on the CPU)."""
import os
import tempfile

import numpy as np
import pytest

from paper_1611_08678_gb300 import autotune, workloads


def test_select_picks_fastest_and_breaks_ties_in_order():
    assert autotune.select([((1, 1), 5.0), ((2, 1), 3.0), ((4, 2), 3.0)]) == (2, 1)
    with pytest.raises(ValueError):
        autotune.select([])


def test_tune_times_every_candidate():
    seen = []

    def fake(nw, fs):
        seen.append((nw, fs))
        return 10.0 / nw + fs  # fastest: the most near warps, fs = 1

    best, results = autotune.tune(fake)
    assert best == (max(c[0] for c in autotune.DEFAULT_CANDIDATES), 1)
    assert sorted(seen) == sorted(autotune.DEFAULT_CANDIDATES)
    assert len(results) == len(autotune.DEFAULT_CANDIDATES)


def test_cache_roundtrip_and_shape_key_buckets():
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sub", "tune.json")
        b = workloads.rossler_batched(M=300, n_lo=1000, n_hi=5000)
        k = autotune.shape_key("GB300", b.system, "bf16x6", b.M, b.N, b.alpha)
        assert "M512" in k and "Nmax8192" in k and "groups8" in k
        autotune.store_cache(k, {"near_warps": 2, "far_split": 4, "ms": 1.5}, path)
        autotune.store_cache("other", {"near_warps": 1, "far_split": 1, "ms": 2.0}, path)
        c = autotune.load_cache(path)
        assert c[k]["near_warps"] == 2 and c[k]["far_split"] == 4 and "other" in c


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
