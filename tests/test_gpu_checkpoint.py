"""Checkpoint and resume through the C ABI (abm_history, abm_solve_resume,
abm_history_batched, abm_solve_batched_resume): a solve split at step n0 -
the first part, its f history exported, then resumed from that history -
equals the uninterrupted solve bit for bit with FP64 arithmetic, and both
match the oracle (Sec. 2: the state at step n is y(0), y'(0) and f_0..f_n)."""
import numpy as np
import pytest

import oracle
from paper_1611_08678_gb300 import workloads
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LORENZ = [10.0, 28.0, 8.0 / 3.0]


@pytest.fixture(scope="module")
def abm():
    from paper_1611_08678_gb300 import abm as m
    m.load()
    return m


@pytest.mark.parametrize("n0", [0, 17, 32, 1237, 2048])
def test_single_split_and_resumed_equals_one_solve(abm, n0):
    N, h, y0 = 3000, 0.01, [0.1, 0.1, 0.1]
    plan = abm.Plan("lorenz", n_max=N)
    Yf, YPf = plan.solve(0.98, h, N, LORENZ, y0, want_yp=True)
    Ffull = plan.history(N + 1).cpu().numpy()
    Yf, YPf = Yf.cpu().numpy(), YPf.cpu().numpy()
    Y = torch.full((N + 1, 3), float("nan"), dtype=torch.float64, device="cuda")
    YP = torch.full((N + 1, 3), float("nan"), dtype=torch.float64, device="cuda")
    if n0 > 0:
        part = plan.solve(0.98, h, n0, LORENZ, y0, Y=Y[: n0 + 1], YP=YP[: n0 + 1])
        assert part is not None
    hist = plan.history(n0 + 1) if n0 > 0 else torch.zeros(1, 3, dtype=torch.float64, device="cuda")
    if n0 > 0:
        assert np.array_equal(hist.cpu().numpy(), Ffull[: n0 + 1])
    plan.solve_resume(0.98, h, n0, N, LORENZ, y0, hist, Y=Y, YP=YP)
    assert np.array_equal(Y.cpu().numpy(), Yf)
    assert np.array_equal(YP.cpu().numpy()[1:], YPf[1:])
    Yo, _, Fo = oracle.solve("lorenz", 0.98, h, 500, LORENZ, y0, return_f=True)
    assert rel_err(Y.cpu().numpy()[:501], Yo) <= 1e-11
    assert rel_err(Ffull[:501], Fo) <= 1e-11


def test_single_resume_from_host_history_general_order(abm):
    """Orders above one and per component, P(EC)^2 E, history kept in
    page-locked host memory between the two parts."""
    N, n0, h = 1500, 700, 0.01
    al, p, y0, y0d = [0.9, 1.3, 1.1], [0.2, 0.2, 5.7], [0.5, -0.3, 0.1], [0.1, 0.2, 0.3]
    plan = abm.Plan("rossler", n_max=N, corrector_passes=2)
    Yf = plan.solve_ext(al, h, N, p, y0, y0d=y0d).cpu().numpy()
    Y = torch.empty(N + 1, 3, dtype=torch.float64, device="cuda")
    plan.solve_ext(al, h, n0, p, y0, y0d=y0d, Y=Y[: n0 + 1])
    hist = plan.history(n0 + 1, F=torch.empty(n0 + 1, 3, dtype=torch.float64, pin_memory=True))
    plan.solve_resume(al, h, n0, N, p, y0, hist, y0d=y0d, Y=Y)
    assert np.array_equal(Y.cpu().numpy(), Yf)
    Yo, _ = oracle.solve_ext("rossler", al, h, 500, p, y0, y0d=y0d, passes=2)
    assert rel_err(Yf[:501], Yo) <= 1e-11


def test_single_resume_rejects_bad_arguments(abm):
    plan = abm.Plan("lorenz", n_max=200)
    plan.solve(0.9, 0.01, 200, LORENZ, [0.1, 0.1, 0.1])
    F = plan.history(201)
    for n0, N in ((-1, 100), (150, 100), (50, 201)):
        with pytest.raises(abm.AbmError) as ei:
            plan.solve_resume(0.9, 0.01, n0, N, LORENZ, [0.1, 0.1, 0.1], F,
                              Y=torch.empty(202, 3, dtype=torch.float64, device="cuda"))
        assert ei.value.status == 1
    with pytest.raises(abm.AbmError) as ei:
        plan.history(202)
    assert ei.value.status == 1


def _split_batched(abm, b, prec, n0, al, y0d):
    """(uninterrupted Y, split-and-resumed Y) of one batch."""
    M, ldY = b.M, int(b.N.max()) + 1
    plan = abm.Plan(b.system, n_max=int(b.N.max()), max_batch=M, prec=prec)
    Yf = plan.solve_batched_ext(al, b.h, b.N, b.params, b.y0, y0d=y0d, ldY=ldY).cpu().numpy()
    Ffull = plan.history_batched(al, b.h, b.N, ldY)
    N0 = np.full(M, n0)
    Y = torch.zeros(M, ldY, 3, dtype=torch.float64, device="cuda")
    plan.solve_batched_ext(al, b.h, N0, b.params, b.y0, y0d=y0d, Y=Y, ldY=ldY)
    hist = plan.history_batched(al, b.h, N0, n0 + 1)
    plan.solve_batched_resume(al, b.h, b.N, n0, b.params, b.y0, hist, y0d=y0d, Y=Y, ldY=ldY)
    return Yf, Y.cpu().numpy(), Ffull.cpu().numpy(), hist.cpu().numpy()


@pytest.mark.parametrize("n0", [64, 333])
def test_batched_fp64_split_and_resumed_equals_one_solve(abm, n0):
    b = workloads.random_batch("rossler", 70, 400, 900, [0.9])
    rng = np.random.default_rng(1611)
    tuples = np.array([(0.9, 0.9, 0.9), (1.1, 1.1, 1.1), (1.2, 0.8, 1.0)])
    al = tuples[rng.integers(0, 3, b.M)]
    y0d = rng.uniform(-0.2, 0.2, (b.M, 3))
    Yf, Yr, Ffull, hist = _split_batched(abm, b, "fp64", n0, al, y0d)
    assert np.array_equal(Yr, Yf)
    assert np.array_equal(hist[:, : n0 + 1], Ffull[:, : n0 + 1])
    worst = 0.0
    for i in range(0, b.M, 9):
        n = min(int(b.N[i]), 500)
        Yo, _ = oracle.solve_ext("rossler", al[i], b.h[i], n, b.params[i], b.y0[i], y0d=y0d[i])
        worst = max(worst, rel_err(Yr[i, : n + 1], Yo))
    assert worst <= 1e-11


def test_batched_tensor_core_resume(abm):
    """BF16x6: the resumed solve rebuilds the split history pieces of the
    imported rows; it matches the uninterrupted solve and the oracle."""
    b = workloads.random_batch("rossler", 64, 900, 1400, [0.9, 1.0])
    al = np.repeat(b.alpha[:, None], 3, axis=1)
    Yf, Yr, _, _ = _split_batched(abm, b, "bf16x6", 640, al, None)
    assert rel_err(Yr[0], Yf[0]) <= 1e-9
    worst = 0.0
    for i in range(0, b.M, 7):
        Yo, _ = oracle.solve("rossler", b.alpha[i], b.h[i], 500, b.params[i], b.y0[i])
        worst = max(worst, rel_err(Yr[i, :501], Yo), rel_err(Yf[i, :501], Yo))
    assert worst <= 1e-6
    for i in range(b.M):
        assert np.all(np.isfinite(Yr[i, : int(b.N[i]) + 1]))
