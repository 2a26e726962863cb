"""GPU parity of P(EC)^m E (Plan(corrector_passes=m)): the corrector applied m
times per step, each pass evaluating f at the previous pass's state, against
the oracle's P(EC)^m E, through the C ABI.  Single trajectory (persistent
kernel), batched with the one-CTA and the split near kernels, FP64 and BF16x6
far history."""
import numpy as np
import pytest

import oracle
from paper_1611_08678_gb300 import workloads
from tests._metrics import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abm():
    from paper_1611_08678_gb300 import abm as m
    m.load()
    return m


@pytest.mark.parametrize("m", [2, 3])
def test_single_pecm_matches_oracle(abm, m):
    p, y0 = [10.0, 28.0, 8.0 / 3.0], [0.1, 0.1, 0.1]
    plan = abm.Plan("lorenz", n_max=1000, corrector_passes=m)
    Y, YP = plan.solve(0.98, 0.01, 1000, p, y0, want_yp=True)
    Yo, YPo = oracle.solve("lorenz", 0.98, 0.01, 1000, p, y0, passes=m)
    assert rel_err(Y.cpu().numpy()[:501], Yo[:501]) <= 1e-11
    assert rel_err(YP.cpu().numpy()[1:501], YPo[1:501]) <= 1e-11
    # the passes change the trajectory: PECE differs
    Y1, _ = oracle.solve("lorenz", 0.98, 0.01, 1000, p, y0)
    assert rel_err(Y1[:501], Yo[:501]) > 1e-8


def test_single_pecm_linear_whole_range(abm):
    plan = abm.Plan("linear", n_max=700, corrector_passes=4)
    Y = plan.solve(0.6, 0.02, 700, [-2.0, 0.3, 0.0], [1.0]).cpu().numpy()
    Yo, _ = oracle.solve("linear", 0.6, 0.02, 700, [-2.0, 0.3, 0.0], [1.0], passes=4)
    assert float(np.abs(Y - Yo).max() / np.abs(Yo).max()) <= 1e-11


@pytest.mark.parametrize("near_split", [1, 8])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("bf16x6", 1e-6)])
def test_batched_pecm_matches_oracle(abm, near_split, prec, tol):
    batch = workloads.random_batch("rossler", 70, 64, 700, [0.9, 1.0])
    plan = abm.Plan("rossler", n_max=int(batch.N.max()), max_batch=batch.M, prec=prec, near_split=near_split,
                    corrector_passes=2)
    Y = plan.solve_batched(batch.alpha, batch.h, batch.N, batch.params, batch.y0).cpu().numpy()
    worst = 0.0
    for i in range(batch.M):
        N = int(batch.N[i])
        n = min(N, int(round(5.0 / batch.h[i])))
        Yo, _ = oracle.solve("rossler", batch.alpha[i], batch.h[i], n, batch.params[i], batch.y0[i], passes=2)
        worst = max(worst, rel_err(Y[i, : n + 1], Yo))
        assert np.all(Y[i, N + 1:] == 0.0)
    assert worst <= tol, (near_split, prec, worst)


def test_pecm_top_of_range_ragged_tiles(abm):
    """m = 8, the largest accepted pass count, with N = 777 (not a multiple of
    the 32-step or 64-step time tiles), so the ysh/ysh2 exchange alternates
    through every parity across tile boundaries: persistent single-trajectory
    kernel and the batched split near kernel (8 CTAs per tile)."""
    p, y0 = [10.0, 28.0, 8.0 / 3.0], [0.1, 0.1, 0.1]
    Yo, YPo = oracle.solve("lorenz", 0.98, 0.01, 777, p, y0, passes=8)
    plan = abm.Plan("lorenz", n_max=777, corrector_passes=8)
    Y, YP = plan.solve(0.98, 0.01, 777, p, y0, want_yp=True)
    assert rel_err(Y.cpu().numpy()[:501], Yo[:501]) <= 1e-11
    assert rel_err(YP.cpu().numpy()[1:501], YPo[1:501]) <= 1e-11
    M = 40
    bplan = abm.Plan("lorenz", n_max=777, max_batch=M, near_split=8, corrector_passes=8)
    al, hh, NN = np.full(M, 0.98), np.full(M, 0.01), np.full(M, 777)
    rng = np.random.default_rng(1611)
    P = np.tile(p, (M, 1)) + rng.normal(0.0, 0.05, (M, 3))
    Y0 = np.tile(y0, (M, 1))
    Yb = bplan.solve_batched(al, hh, NN, P, Y0).cpu().numpy()
    for i in (0, 17, M - 1):
        Yi, _ = oracle.solve("lorenz", 0.98, 0.01, 500, P[i], Y0[i], passes=8)
        assert rel_err(Yb[i, :501], Yi) <= 1e-11, i


def test_adjoint_rejects_pecm_plans(abm):
    batch = workloads.random_batch("lorenz", 4, 50, 80, [0.9])
    plan = abm.Plan("lorenz", n_max=80, max_batch=4, corrector_passes=2)
    Y, YP = plan.solve_batched(batch.alpha, batch.h, batch.N, batch.params, batch.y0, want_yp=True)
    params = torch.as_tensor(batch.params, device="cuda")
    y0 = torch.as_tensor(batch.y0, device="cuda")
    with pytest.raises(abm.AbmError) as ei:
        plan.adjoint(batch.alpha, batch.h, batch.N, params, y0, Y, YP, torch.zeros_like(Y))
    assert ei.value.status == 6
