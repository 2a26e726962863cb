"""GPU parity of the batched path (ragged N, several alpha groups, column
tiles, K-split far history) against the FP64 CPU oracle, trajectory by
trajectory, through the C ABI."""
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


def _run(abm, batch, prec, want_yp=False):
    plan = abm.Plan(batch.system, n_max=int(batch.N.max()), max_batch=batch.M, prec=prec)
    out = plan.solve_batched(batch.alpha, batch.h, batch.N, batch.params, batch.y0, want_yp=want_yp)
    return out


def _errors(batch, Y, t_max=None, YP=None):
    errs = []
    for i in range(batch.M):
        N = int(batch.N[i])
        Yo, YPo = oracle.solve(batch.system, batch.alpha[i], batch.h[i], N, batch.params[i], batch.y0[i])
        n = N if t_max is None else min(N, int(round(t_max / batch.h[i])))
        e = rel_err(Y[i, : n + 1], Yo[: n + 1])
        if YP is not None:
            e = max(e, rel_err(YP[i, 1: n + 1], YPo[1: n + 1]))
        errs.append(e)
    return np.array(errs)


@pytest.mark.parametrize("system,alphas,n_lo,n_hi,M", [
    ("linear", [0.4, 0.8, 1.0], 1, 700, 70),
    ("lorenz", [0.9, 0.98], 100, 1300, 45),
    ("rossler", list(np.linspace(0.85, 1.0, 8)), 64, 1100, 80),
    ("financial", [0.95], 500, 900, 33),
])
def test_batched_fp64_matches_oracle(abm, system, alphas, n_lo, n_hi, M):
    batch = workloads.random_batch(system, M, n_lo, n_hi, alphas)
    Y, YP = _run(abm, batch, "fp64", want_yp=True)
    Y, YP = Y.cpu().numpy(), YP.cpu().numpy()
    errs = _errors(batch, Y, t_max=5.0, YP=YP)
    assert errs.max() <= 1e-11, (int(errs.argmax()), errs.max())
    # rows beyond each trajectory's N stay untouched (zero-initialised)
    for i in range(batch.M):
        assert np.all(Y[i, int(batch.N[i]) + 1:] == 0.0)


@pytest.mark.parametrize("system,alphas", [("lorenz", [0.98]), ("rossler", [0.85, 0.9, 1.0]),
                                           ("financial", [0.95])])
def test_batched_fp32_far_error_reported(abm, system, alphas):
    """FP32 far history: no exact pin; the max relative error against the
    FP64 oracle up to t = 5 must stay within 1e-6."""
    batch = workloads.random_batch(system, 40, 300, 1100, alphas)
    Y = _run(abm, batch, "fp32").cpu().numpy()
    errs = _errors(batch, Y, t_max=5.0)
    print(f"{system} fp32-far max rel err (t<=5): {errs.max():.3e}")
    assert errs.max() <= 1e-6


def test_batched_single_equivalence(abm):
    """A batch of one equals the single-trajectory path to rounding order."""
    batch = workloads.random_batch("lorenz", 1, 900, 900, [0.98])
    Yb = _run(abm, batch, "fp64").cpu().numpy()[0]
    plan = abm.Plan("lorenz", n_max=900)
    Ys = plan.solve(batch.alpha[0], batch.h[0], 900, batch.params[0], batch.y0[0]).cpu().numpy()
    assert rel_err(Yb[:501], Ys[:501]) <= 1e-12


def test_batched_rejects_bad_arguments(abm):
    batch = workloads.random_batch("lorenz", 4, 10, 20, [0.9])
    plan = abm.Plan("lorenz", n_max=20, max_batch=4)
    bad = batch.N.copy(); bad[2] = 0
    with pytest.raises(abm.AbmError):
        plan.solve_batched(batch.alpha, batch.h, bad, batch.params, batch.y0)
    bad = batch.alpha.copy(); bad[1] = 1.2
    with pytest.raises(abm.AbmError):
        plan.solve_batched(bad, batch.h, batch.N, batch.params, batch.y0)
    big = workloads.random_batch("lorenz", 5, 10, 20, [0.9])
    with pytest.raises(abm.AbmError):
        plan.solve_batched(big.alpha, big.h, big.N, big.params, big.y0)
