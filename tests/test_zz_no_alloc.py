"""abm_solve_noalloc, the single-trajectory solve for callers that may not
allocate device memory (its scratch is a static device array inside the
library), checked against abm_solve, the allocating entry point, through the
C ABI.  Kept in a file of its own that collects last."""
import numpy as np
import pytest

import oracle
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    ("lorenz", 0.98, 0.01, 8192, [10.0, 28.0, 8.0 / 3.0], [0.1, 0.1, 0.1]),
    ("chen", 0.9, 0.001, 5000, [35.0, 3.0, 28.0], [-9.0, -5.0, 14.0]),
    ("linear", 0.6, 0.01, 777, [-1.5, 0.3, 0.2], [1.0]),
]


def _reference(abm, system, alpha, h, N, p, y0):
    plan = abm.Plan(system, n_max=N)
    Y, YP = plan.solve(alpha, h, N, p, y0, want_yp=True)
    return Y.cpu().numpy(), YP.cpu().numpy()


def _free_unchanged(call):
    """Runs call() and tells whether the device's free memory stayed the
    same.  Free memory counts every context on the GPU, so another process
    may move it: a difference is retried twice before it counts."""
    for _ in range(3):
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        call()
        torch.cuda.synchronize()
        if torch.cuda.mem_get_info()[0] == before:
            return True
    return False


def test_noalloc_matches_abm_solve_on_consecutive_calls():
    from paper_1611_08678_gb300 import abm
    refs = [_reference(abm, *c) for c in CASES]
    order = [0, 1, 2, 0]  # consecutive calls share the scratch array
    for step, i in enumerate(order):
        system, alpha, h, N, p, y0 = CASES[i]
        d = len(y0)
        Y = torch.full((N + 1, d), float("nan"), dtype=torch.float64, device="cuda")
        YP = torch.full((N + 1, d), float("nan"), dtype=torch.float64, device="cuda")
        reserved = torch.cuda.memory_reserved()
        call = lambda: abm.solve_noalloc(system, alpha, h, N, p, y0, Y, YP)
        if step == 0:  # the first call may load the module that holds the array
            call()
        else:
            assert _free_unchanged(call), "abm_solve_noalloc allocated device memory"
        assert torch.cuda.memory_reserved() == reserved
        Yr, YPr = refs[i]
        assert rel_err(Y.cpu().numpy(), Yr) <= 1e-11, (step, system)
        assert rel_err(YP.cpu().numpy()[1:], YPr[1:]) <= 1e-11, (step, system)


def test_noalloc_matches_the_oracle():
    """The same entry point against the CPU oracle directly (pointwise window
    t <= 5, t <= 3 for Chen, whose conditioning limits FP64 agreement)."""
    from paper_1611_08678_gb300 import abm
    for system, alpha, h, N, p, y0 in CASES:
        d = len(y0)
        Y = torch.empty((N + 1, d), dtype=torch.float64, device="cuda")
        abm.solve_noalloc(system, alpha, h, N, p, y0, Y)
        n = min(N, int(round((3.0 if system == "chen" else 5.0) / h)))
        Yo, _ = oracle.solve(system, alpha, h, n, p, y0)
        assert rel_err(Y.cpu().numpy()[: n + 1], Yo) <= 1e-11, system


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1611_08678_gb300 import abm
    Y = torch.empty(40000, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(abm.AbmError) as ei:
        abm.solve_noalloc("lorenz", 0.9, 0.01, 32769, [10.0, 28.0, 8 / 3], [0.1, 0.1, 0.1], Y)
    assert ei.value.status == 1 and "32768" in str(ei.value)
