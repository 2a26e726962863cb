"""The benchmark's roofline accounting (no GPU): the algorithmic far-history
work and operand bytes bench.py divides by the measured kernel time are
checked against brute-force counts written independently here."""
import importlib.util
import os

import numpy as np

from paper_1611_08678_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_for_accounting", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_far_flops_match_a_step_by_step_count():
    """Every target step n of trajectory i (0 <= n < N_i) lies in time tile
    s = 64 floor(n / 64); its predictor and corrector far sums cover history
    rows 1 <= k < s (row 0 stays FP64 in the near step): 2 sums x d columns x
    (s - 1) multiply-adds of 2 flops."""
    bench = _bench()
    w = workloads.random_batch("rossler", 40, 100, 900, [0.85, 0.9, 1.0])
    alg, _, _ = bench.far_work(w, 6, 3)
    want = 0.0
    for i in range(w.M):
        for n in range(int(w.N[i])):
            s = (n // 64) * 64
            want += 2.0 * 2 * w.d * max(s - 1, 0)
    assert alg == want


def test_far_bytes_of_one_launch_match_the_profile_count():
    """The 512-trajectory Rossler case at time tile s = 38464: 8 active column
    tiles (one per alpha group) stream 38464 rows x 96 columns x 3 BF16 pieces,
    and each group's Toeplitz block 128 rows x 38464 x 3 pieces."""
    bench = _bench()
    w = workloads.rossler_batched().subset(np.arange(512))
    tiles = bench.tile_schedule(w)
    s = 38464
    act = [t for t in tiles if t[0] > s]
    assert len(act) == 8 and len({t[1] for t in act}) == 8
    one_launch = len(act) * s * 96 * 2 * 3 + len({t[1] for t in act}) * 128 * s * 2 * 3
    assert one_launch == 413564928  # the algorithmic bytes the far_tc profile divides by
    # and the whole-solve total is the sum of such launches
    _, _, byts = bench.far_work(w, 6, 3)
    total = 0
    for j in range(1, (max(t[0] for t in tiles) + 63) // 64):
        s = j * 64
        a = [t for t in tiles if t[0] > s]
        total += len(a) * s * 96 * 6 + len({t[1] for t in a}) * 128 * s * 6
    assert byts == total


def test_tile_schedule_groups_alpha_and_sorts_by_length():
    bench = _bench()
    w = workloads.random_batch("rossler", 100, 50, 5000, [0.85, 0.95])
    tiles = bench.tile_schedule(w)
    assert sum(len(t[2]) for t in tiles) == w.M
    for n_tile, g, Ns in tiles:
        assert n_tile == Ns.max() and np.all(np.diff(Ns) <= 0) and len(Ns) <= 32
