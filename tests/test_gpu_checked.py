"""The checked build (libabm_gb300_checked.so, compiled with ABM_CHECKED):
every kernel compares the indices it derives from the host's layout with the
extents of the buffers they address.  On the hot paths it must find nothing
and compute what the plain library computes; a testing option that moves one
output row past the end of Y must come back as ABM_ERR_BOUNDS, with the store
skipped and the plan still usable."""
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
    m.load(m.CHECKED_LIB_PATH)
    return m


def test_checked_single_and_resume(abm):
    N = 3000
    plain = abm.Plan("lorenz", n_max=N)
    chk = abm.Plan("lorenz", n_max=N, checked=True)
    Yp = plain.solve(0.98, 0.01, N, LORENZ, [0.1, 0.1, 0.1]).cpu().numpy()
    Yc = chk.solve(0.98, 0.01, N, LORENZ, [0.1, 0.1, 0.1]).cpu().numpy()
    assert rel_err(Yc, Yp) <= 1e-13
    hist = chk.history(1500)
    Yr = torch.empty(N + 1, 3, dtype=torch.float64, device="cuda")
    Yr[:1500] = torch.as_tensor(Yc[:1500], device="cuda")
    chk.solve_resume(0.98, 0.01, 1499, N, LORENZ, [0.1, 0.1, 0.1], hist, Y=Yr)
    assert rel_err(Yr.cpu().numpy(), Yc) <= 1e-13
    Yo, _ = oracle.solve("lorenz", 0.98, 0.01, 500, LORENZ, [0.1, 0.1, 0.1])
    assert rel_err(Yc[:501], Yo) <= 1e-11


@pytest.mark.parametrize("prec,near_split,tol", [("fp64", 0, 1e-11), ("fp64", 8, 1e-11), ("fp32", 0, 1e-6),
                                                 ("bf16x6", 0, 1e-6), ("bf16x3", 1, 1e-5)])
def test_checked_batched_paths(abm, prec, near_split, tol):
    b = workloads.random_batch("rossler", 70, 200, 1400, [0.9, 1.0])
    kw = dict(n_max=int(b.N.max()), max_batch=b.M, prec=prec, near_split=near_split)
    Yp = abm.Plan("rossler", **kw).solve_batched(b.alpha, b.h, b.N, b.params, b.y0).cpu().numpy()
    chk = abm.Plan("rossler", checked=True, **kw)
    Yc = chk.solve_batched(b.alpha, b.h, b.N, b.params, b.y0).cpu().numpy()
    assert rel_err(Yc.reshape(-1, 3), Yp.reshape(-1, 3)) <= (1e-13 if prec == "fp64" else 10 * tol)
    worst = 0.0
    for i in range(0, b.M, 11):
        n = min(int(b.N[i]), 1000)
        Yo, _ = oracle.solve("rossler", b.alpha[i], b.h[i], n, b.params[i], b.y0[i])
        worst = max(worst, rel_err(Yc[i, : n + 1], Yo))
    assert worst <= tol, worst
    # the general problem and checkpoint/resume on the checked build
    al = np.repeat(b.alpha[:, None], 3, axis=1)
    Y2 = torch.zeros(b.M, int(b.N.max()) + 1, 3, dtype=torch.float64, device="cuda")
    chk.solve_batched_ext(al, b.h, np.full(b.M, 200), b.params, b.y0, Y=Y2, ldY=Y2.shape[1])
    hist = chk.history_batched(al, b.h, np.full(b.M, 200), 201)
    chk.solve_batched_resume(al, b.h, b.N, 200, b.params, b.y0, hist, Y=Y2)
    assert rel_err(Y2.cpu().numpy()[0], Yc[0]) <= (0.0 if prec == "fp64" else 1e-9)


def test_checked_adjoint_and_host_buffers(abm):
    b = workloads.random_batch("lorenz", 40, 100, 300, [0.95])
    chk = abm.Plan("lorenz", n_max=int(b.N.max()), max_batch=b.M, prec="bf16x6", checked=True)
    Y, YP = chk.solve_batched(b.alpha, b.h, b.N, b.params, b.y0, want_yp=True)
    dp, dy0 = chk.adjoint(b.alpha, b.h, b.N, b.params, b.y0, Y, YP, torch.ones_like(Y) * 1e-3)
    assert torch.isfinite(dp).all() and torch.isfinite(dy0).all()
    Yh = chk.solve_batched_host(b.alpha, b.h, b.N, b.params, b.y0)
    for i in range(b.M):
        n = int(b.N[i])
        assert rel_err(Yh.numpy()[i, : n + 1], Y.cpu().numpy()[i, : n + 1]) <= 1e-12


@pytest.mark.parametrize("near_split", [1, 8])
def test_checked_build_reports_an_index_outside_its_buffer(abm, near_split):
    """Trajectory 4's output row is moved past the end of Y (testing option):
    the checked near kernel skips that store and the call reports
    ABM_ERR_BOUNDS naming the kernel; the other trajectories are complete and
    the plan stays usable."""
    b = workloads.random_batch("rossler", 40, 100, 300, [0.9])
    chk = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, checked=True, test_bad_index=5,
                   near_split=near_split)
    Y = torch.zeros(b.M, int(b.N.max()) + 1, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(abm.AbmError) as ei:
        chk.solve_batched(b.alpha, b.h, b.N, b.params, b.y0, Y=Y)
    assert ei.value.status == 7
    assert "near kernel" in str(ei.value), str(ei.value)
    Yc = Y.cpu().numpy()
    assert np.all(Yc[4, 1:] == 0.0)  # the store was skipped
    ok = abm.Plan("rossler", n_max=int(b.N.max()), max_batch=b.M, checked=True)
    Yok = ok.solve_batched(b.alpha, b.h, b.N, b.params, b.y0).cpu().numpy()
    for i in (0, 3, 5, 39):
        n = int(b.N[i])
        assert rel_err(Yc[i, : n + 1], Yok[i, : n + 1]) <= 1e-13
