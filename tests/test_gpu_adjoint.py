"""GPU adjoint (abm_adjoint, A6) against the oracle's tangent-linear gradient
and against central finite differences of the GPU forward solve."""
import numpy as np
import pytest

import oracle
from paper_1611_08678_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abm():
    from paper_1611_08678_gb300 import abm as m
    m.load()
    return m


def _loss_partials(batch, Y, target):
    """loss = sum_i mean over rows 0..N_i and components of (y - target)^2."""
    G = np.zeros_like(Y)
    for i in range(batch.M):
        n = int(batch.N[i])
        G[i, : n + 1] = 2.0 * (Y[i, : n + 1] - target[i, : n + 1]) / ((n + 1) * batch.d)
    return G


def _case(abm, system, M, n_lo, n_hi, alphas, prec, seed=workloads.SEED_PERTURB, near_split=0):
    batch = workloads.random_batch(system, M, n_lo, n_hi, alphas)
    plan = abm.Plan(system, n_max=int(batch.N.max()), max_batch=M, prec=prec, near_split=near_split)
    Y, YP = plan.solve_batched(batch.alpha, batch.h, batch.N, batch.params, batch.y0, want_yp=True)
    Yn = Y.cpu().numpy()
    rng = np.random.default_rng(seed)
    target = Yn + 0.05 * rng.standard_normal(Yn.shape)
    G = _loss_partials(batch, Yn, target)
    params = torch.as_tensor(batch.params, device="cuda")
    y0 = torch.as_tensor(batch.y0, device="cuda")
    dp, dy0 = plan.adjoint(batch.alpha, batch.h, batch.N, params, y0, Y, YP, torch.as_tensor(G, device="cuda"))
    return batch, plan, Y, YP, target, G, dp.cpu().numpy(), dy0.cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("system,M,n_lo,n_hi,alphas", [
    ("lorenz", 5, 40, 300, [0.9, 0.98]),
    ("financial", 40, 60, 200, [0.95]),
    ("rossler", 36, 100, 260, [0.85, 1.0]),
    ("hindmarsh_rose", 20, 60, 200, [0.95]),
])
def test_adjoint_fp64_matches_tangent_linear_oracle(abm, system, M, n_lo, n_hi, alphas):
    batch, plan, Y, YP, target, G, dp, dy0 = _case(abm, system, M, n_lo, n_hi, alphas, "fp64")
    worst = 0.0
    for i in range(batch.M):
        n = int(batch.N[i])
        op, oy = oracle.tangent(system, batch.alpha[i], batch.h[i], n, batch.params[i], batch.y0[i], G[i, : n + 1])
        worst = max(worst, _rel(dp[i], op), _rel(dy0[i], oy))
    print(f"{system} fp64 adjoint vs tangent-linear: max rel {worst:.2e}")
    assert worst <= 1e-9


@pytest.mark.parametrize("near_split", [1, 4, 8])
@pytest.mark.parametrize("system,M,n_lo,n_hi,alphas", [
    ("lorenz", 40, 60, 300, [0.9, 0.98]),
    ("hindmarsh_rose", 12, 64, 200, [0.95]),
])
def test_adjoint_near_split_matches_tangent_linear_oracle(abm, near_split, system, M, n_lo, n_hi, alphas):
    """The adjoint near kernel with each forward tile spread over 4 or 8 CTAs
    (lanes of a trajectory summing interleaved lag slices of both windows)
    gives the tangent-linear oracle's gradients like the one-CTA kernel."""
    batch, plan, Y, YP, target, G, dp, dy0 = _case(abm, system, M, n_lo, n_hi, alphas, "fp64",
                                                   near_split=near_split)
    worst = 0.0
    for i in range(batch.M):
        n = int(batch.N[i])
        op, oy = oracle.tangent(system, batch.alpha[i], batch.h[i], n, batch.params[i], batch.y0[i], G[i, : n + 1])
        worst = max(worst, _rel(dp[i], op), _rel(dy0[i], oy))
    assert worst <= 1e-9, (near_split, system, worst)


def test_adjoint_matches_central_differences_of_gpu_solve(abm):
    """Window t <= 2 (200 steps at h = 0.01): dL/dtheta by the adjoint against
    central differences (step 1e-6) of the FP64 GPU solve, within 1e-6."""
    batch, plan, Y, YP, target, G, dp, dy0 = _case(abm, "lorenz", 3, 200, 200, [0.98], "fp64")

    def loss(params, y0):
        Yv = plan.solve_batched(batch.alpha, batch.h, batch.N, params, y0).cpu().numpy()
        return sum(np.mean((Yv[i, : int(batch.N[i]) + 1] - target[i, : int(batch.N[i]) + 1]) ** 2)
                   for i in range(batch.M))

    worst = 0.0
    for i in range(batch.M):
        for j in range(3):
            for which in ("p", "y0"):
                P, Y0 = batch.params.copy(), batch.y0.copy()
                arr = P if which == "p" else Y0
                delta = 1e-6 * max(1.0, abs(arr[i, j]))
                arr[i, j] += delta
                lp = loss(P, Y0)
                arr[i, j] -= 2 * delta
                lm = loss(P, Y0)
                fd = (lp - lm) / (2 * delta)
                an = dp[i, j] if which == "p" else dy0[i, j]
                worst = max(worst, abs(an - fd) / max(abs(fd), 1e-3))
    print(f"adjoint vs central differences: max rel {worst:.2e}")
    assert worst <= 1e-6


@pytest.mark.parametrize("prec,tol", [("bf16x6", 1e-5), ("bf16x3", 1e-3)])
def test_adjoint_tensor_core_error_reported(abm, prec, tol):
    batch, plan, Y, YP, target, G, dp, dy0 = _case(abm, "lorenz", 40, 100, 400, [0.98], prec)
    worst = 0.0
    for i in range(0, batch.M, 7):
        n = int(batch.N[i])
        op, oy = oracle.tangent("lorenz", batch.alpha[i], batch.h[i], n, batch.params[i], batch.y0[i], G[i, : n + 1])
        worst = max(worst, _rel(dp[i], op), _rel(dy0[i], oy))
    print(f"{prec} adjoint vs tangent-linear: max rel {worst:.2e}")
    assert worst <= tol


def test_autograd_function_backward(abm):
    from paper_1611_08678_gb300.autograd import abm_solve
    batch = workloads.random_batch("lorenz", 4, 120, 150, [0.98])
    plan = abm.Plan("lorenz", n_max=int(batch.N.max()), max_batch=4, prec="fp64")
    params = torch.as_tensor(batch.params, device="cuda").requires_grad_(True)
    y0 = torch.as_tensor(batch.y0, device="cuda").requires_grad_(True)
    Y = abm_solve(plan, batch.alpha, batch.h, batch.N, params, y0)
    loss = (Y ** 2).sum() * 1e-3
    loss.backward()
    Yn = Y.detach().cpu().numpy()
    for i in range(batch.M):
        n = int(batch.N[i])
        G = 2e-3 * Yn[i, : n + 1]
        op, oy = oracle.tangent("lorenz", batch.alpha[i], batch.h[i], n, batch.params[i], batch.y0[i], G)
        assert _rel(params.grad[i].cpu().numpy(), op) <= 1e-9
        assert _rel(y0.grad[i].cpu().numpy(), oy) <= 1e-9
