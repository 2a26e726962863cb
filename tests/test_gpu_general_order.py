"""GPU parity of the general problem of eq. (1) through the C ABI
(abm_solve_ext, abm_solve_batched_ext): orders in (0, 2] with the initial
derivative y'(0) in the Taylor sum of eq. (2) and the corrector, and one order
per state component (non-commensurate systems), against the oracle's
oracle_solve_ext.  FP64 paths within 1e-11 (pointwise, t <= 5); FP32 and the
tensor-core BF16x6 far history within 1e-6 (equal orders per trajectory on the
tensor cores)."""
import math

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


def test_single_ext_equal_orders_is_abm_solve(abm):
    """Equal orders at most one: abm_solve_ext runs the commensurate kernel and
    returns abm_solve's values bit for bit (y'(0) is not used)."""
    plan = abm.Plan("lorenz", n_max=2000)
    Y = plan.solve(0.9, 0.01, 2000, LORENZ, [0.1, 0.1, 0.1]).cpu().numpy()
    Ye = plan.solve_ext([0.9, 0.9, 0.9], 0.01, 2000, LORENZ, [0.1, 0.1, 0.1], y0d=[3.0, 1.0, 2.0]).cpu().numpy()
    assert np.array_equal(Y, Ye)


@pytest.mark.parametrize("alpha", [1.3, 1.8, 2.0])
def test_single_ext_linear_forcing_above_one(abm, alpha):
    """D^a y = q0 + q1 t, y(0) = y0, y'(0) = y1: the oracle and the closed form
    y0 + y1 t + q0 t^a/Gamma(a+1) + q1 t^(a+1)/Gamma(a+2)."""
    N, h, q0, q1, y0, y1 = 1500, 0.01, 1.3, -0.7, 0.25, -0.6
    plan = abm.Plan("linear", n_max=N)
    Y = plan.solve_ext(alpha, h, N, [0.0, q0, q1], [y0], y0d=[y1]).cpu().numpy()[:, 0]
    Yo, _ = oracle.solve_ext("linear", alpha, h, N, [0.0, q0, q1], [y0], y0d=[y1])
    t = np.arange(N + 1) * h
    ex = y0 + y1 * t + q0 * t ** alpha / math.gamma(alpha + 1) + q1 * t ** (alpha + 1) / math.gamma(alpha + 2)
    assert float(np.abs(Y - Yo[:, 0]).max() / np.abs(Yo).max()) <= 1e-11
    assert float(np.abs(Y - ex).max() / np.abs(ex).max()) <= 1e-11


@pytest.mark.parametrize("system,alpha,h,N,p,y0,y0d", [
    ("lorenz", [0.95, 1.2, 0.8], 0.005, 1000, LORENZ, [0.1, 0.1, 0.1], [0.0, 0.5, 0.0]),
    ("rossler", [1.5, 1.5, 1.5], 0.01, 1000, [0.2, 0.2, 5.7], [0.5, -0.3, 0.1], [0.1, 0.2, 0.0]),
    ("rossler", [0.9, 1.3, 1.1], 0.01, 1000, [0.2, 0.2, 5.7], [0.5, -0.3, 0.1], [0.1, 0.2, 0.3]),
    ("financial", [1.2, 0.9, 1.05], 0.01, 1000, [3.0, 0.1, 1.0], [2.0, 3.0, 2.0], [0.1, -0.1, 0.2]),
    ("hindmarsh_rose", [0.98, 1.4, 0.9], 0.01, 1000, workloads.HR_PARAMS, [0.1, 0.2, 0.3], [0.0, 0.1, 0.0]),
])
def test_single_ext_matches_oracle(abm, system, alpha, h, N, p, y0, y0d):
    plan = abm.Plan(system, n_max=N)
    Y, YP = plan.solve_ext(alpha, h, N, p, y0, y0d=y0d, want_yp=True)
    Yo, YPo = oracle.solve_ext(system, alpha, h, N, p, y0, y0d=y0d)
    assert rel_err(Y.cpu().numpy(), Yo) <= 1e-11
    assert rel_err(YP.cpu().numpy()[1:], YPo[1:]) <= 1e-11


def test_single_ext_decoupled_components(abm):
    """Lorenz with sigma = 0 and x(0) = 0: y and z obey D^a y = -y and
    D^c z = -beta z at their own orders, so each equals the oracle's scalar
    solve at that order."""
    beta = 8.0 / 3.0
    al, y0, y0d = [0.8, 1.4, 0.6], [0.0, 0.7, -0.4], [0.0, 0.3, 0.0]
    plan = abm.Plan("lorenz", n_max=1200)
    Y = plan.solve_ext(al, 0.01, 1200, [0.0, 28.0, beta], y0, y0d=y0d).cpu().numpy()
    assert np.all(Y[:, 0] == 0.0)
    Yy, _ = oracle.solve_ext("linear", al[1], 0.01, 1200, [-1.0, 0.0, 0.0], [y0[1]], y0d=[y0d[1]])
    Yz, _ = oracle.solve_ext("linear", al[2], 0.01, 1200, [-beta, 0.0, 0.0], [y0[2]])
    assert rel_err(Y[:, 1:2], Yy) <= 1e-11 and rel_err(Y[:, 2:3], Yz) <= 1e-11


def test_single_ext_rejects_orders_outside_range(abm):
    plan = abm.Plan("lorenz", n_max=100)
    for al in ([0.9, 2.5, 0.9], [0.0, 0.9, 0.9], [0.9, float("nan"), 0.9]):
        with pytest.raises(abm.AbmError) as ei:
            plan.solve_ext(al, 0.01, 50, LORENZ, [0.1, 0.1, 0.1])
        assert ei.value.status == 1
    with pytest.raises(abm.AbmError) as ei:
        plan.solve_ext(1.5, 0.01, 50, LORENZ, [0.1, 0.1, 0.1], y0d=[0.0, float("inf"), 0.0])
    assert ei.value.status == 1


# Order tuples of the batched tests: commensurate at, below and above one, and
# non-commensurate with components on both sides of one.
# (Commensurate Roessler flows above about 1.1 leave every bound within these
# runs' lengths for some of the drawn parameters.)
TUPLES = [(0.95, 0.95, 0.95), (1.1, 1.1, 1.1), (0.9, 1.3, 1.1), (1.2, 0.8, 1.0)]


def _ext_batch(M, n_lo, n_hi, tuples, seed=1611):
    b = workloads.random_batch("rossler", M, n_lo, n_hi, [0.9])
    rng = np.random.default_rng(seed)
    al = np.array(tuples, float)[rng.integers(0, len(tuples), M)]
    y0d = rng.uniform(-0.2, 0.2, (M, 3))
    return b, al, y0d


def _worst(b, al, y0d, Y, passes=1, idx=None):
    worst = 0.0
    for i in (range(b.M) if idx is None else idx):
        n = min(int(b.N[i]), int(round(5.0 / b.h[i])))
        Yo, _ = oracle.solve_ext("rossler", al[i], b.h[i], n, b.params[i], b.y0[i], y0d=y0d[i], passes=passes)
        worst = max(worst, rel_err(Y[i, : n + 1], Yo))
    return worst


@pytest.mark.parametrize("near_split", [1, 8])
def test_batched_ext_fp64_matches_oracle(abm, near_split):
    b, al, y0d = _ext_batch(72, 64, 700, TUPLES)
    plan = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, near_split=near_split)
    Y = plan.solve_batched_ext(al, b.h, b.N, b.params, b.y0, y0d=y0d).cpu().numpy()
    assert _worst(b, al, y0d, Y) <= 1e-11
    for i in range(b.M):
        assert np.all(Y[i, int(b.N[i]) + 1:] == 0.0)


def test_batched_ext_fp32_far_matches_oracle(abm):
    b, al, y0d = _ext_batch(72, 600, 1400, TUPLES)
    plan = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, prec="fp32")
    Y = plan.solve_batched_ext(al, b.h, b.N, b.params, b.y0, y0d=y0d).cpu().numpy()
    worst = _worst(b, al, y0d, Y)
    print(f"fp32 far, general orders: {worst:.2e}")
    assert worst <= 1e-6


def test_batched_ext_tensor_core_equal_orders(abm):
    """BF16x6 far history with equal orders per trajectory above and below one."""
    b, al, y0d = _ext_batch(80, 600, 1400, [(0.95, 0.95, 0.95), (1.1, 1.1, 1.1), (1.05, 1.05, 1.05)])
    plan = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, prec="bf16x6")
    Y = plan.solve_batched_ext(al, b.h, b.N, b.params, b.y0, y0d=y0d).cpu().numpy()
    worst = _worst(b, al, y0d, Y)
    print(f"bf16x6 far, orders above one: {worst:.2e}")
    assert worst <= 1e-6


def test_batched_ext_tensor_core_rejects_per_component_orders(abm):
    b, al, y0d = _ext_batch(8, 64, 200, TUPLES)
    plan = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, prec="bf16x6")
    with pytest.raises(abm.AbmError) as ei:
        plan.solve_batched_ext(al, b.h, b.N, b.params, b.y0, y0d=y0d)
    assert ei.value.status == 6


def test_batched_ext_pecm_and_graph(abm):
    """P(EC)^2 E with general orders, replayed from a captured CUDA graph."""
    b, al, y0d = _ext_batch(40, 64, 500, TUPLES)
    plan = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, corrector_passes=2, use_graph=True)
    ldY = int(b.N.max()) + 1
    params = torch.as_tensor(b.params, device="cuda")
    y0 = torch.as_tensor(b.y0, device="cuda")
    yd = torch.as_tensor(y0d, device="cuda")
    Y = torch.zeros(b.M, ldY, 3, dtype=torch.float64, device="cuda")
    plan.solve_batched_ext(al, b.h, b.N, params, y0, y0d=yd, Y=Y)  # capture
    first = Y.cpu().numpy()
    Y.zero_()
    plan.solve_batched_ext(al, b.h, b.N, params, y0, y0d=yd, Y=Y)  # replay
    again = Y.cpu().numpy()
    assert np.array_equal(first, again)
    assert _worst(b, al, y0d, again, passes=2) <= 1e-11
