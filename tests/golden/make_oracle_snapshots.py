"""Writes ``oracle_snapshots.txt``: sampled outputs of the FP64 CPU oracle.

Calls nothing but the oracle.  The snapshot is a regression fixture, not a pin:
``tests/test_golden.py`` recomputes every value and fails when the oracle's
arithmetic changes, so a change to the oracle is always a deliberate one.
Regenerate with ``python tests/golden/make_oracle_snapshots.py``.

Cases: the fractional ABM PECE scheme of Section 2 (eq. (2) predictor, product
trapezoid corrector) on every built-in right-hand side, three P(EC)^m E solves
(the corrector repeated m times per step), and the weights b_m, a_m, c_m, g of
Section 2 at lags on both sides of the kernels' series switch.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

# (system, alpha, h, N, params, y0): small solves, a few time units at most
SOLVES = [
    ("linear", 0.6, 0.05, 64, [-1.5, 0.4, 0.2], [1.0]),
    ("manufactured", 0.7, 1.0 / 64, 64, [1.0, -0.5, 0.3, -1.0, -0.5, 0.2, 1.0, -0.5, 0.3], [0.2]),
    ("lorenz", 0.98, 0.01, 64, [10.0, 28.0, 8.0 / 3.0], [0.1, 0.1, 0.1]),
    ("chen", 0.9, 0.001, 64, [35.0, 3.0, 28.0], [-9.0, -5.0, 14.0]),
    ("rossler", 0.9, 0.005, 64, [0.2, 0.2, 5.7], [0.5, 1.0, 1.5]),
    ("financial", 0.95, 0.01, 64, [1.0, 0.1, 1.0], [2.0, 3.0, 2.0]),
    ("hindmarsh_rose", 0.98, 0.01, 64, [1.0, 3.0, 1.0, 5.0, 0.006, 4.0, -1.6, 3.25], [0.1, 0.2, 0.3]),
]
SOLVE_ROWS = [1, 2, 3, 17, 33, 63, 64]
# (case index into SOLVES, corrector passes m > 1): P(EC)^m E solves
PECM = [(2, 2), (4, 3), (6, 2)]
WEIGHT_ALPHAS = [0.3, 0.5, 0.9, 0.98, 1.0]
WEIGHT_LAGS = [0, 1, 2, 15, 16, 17, 31, 32, 33, 1000, 65536, 262144]


def lines():
    out = ["# kind case index component value  (regenerate: python tests/golden/make_oracle_snapshots.py)"]
    for i, (system, alpha, h, N, p, y0) in enumerate(SOLVES):
        Y, YP = oracle.solve(system, alpha, h, N, p, y0)
        for n in SOLVE_ROWS:
            for j in range(Y.shape[1]):
                out.append(f"Y {i} {n} {j} {float(Y[n, j])!r}")
                out.append(f"YP {i} {n} {j} {float(YP[n, j])!r}")
    for q, (i, m) in enumerate(PECM):
        system, alpha, h, N, p, y0 = SOLVES[i]
        Y, _ = oracle.solve(system, alpha, h, N, p, y0, passes=m)
        for n in SOLVE_ROWS:
            for j in range(Y.shape[1]):
                out.append(f"YM {q} {n} {j} {float(Y[n, j])!r}")
    for i, alpha in enumerate(WEIGHT_ALPHAS):
        b, a, c, g = oracle.weights(alpha, WEIGHT_LAGS[-1])
        for m in WEIGHT_LAGS:
            out.append(f"b {i} {m} 0 {float(b[m])!r}")
            out.append(f"a {i} {m} 0 {float(a[m])!r}")
            if m >= 1:
                out.append(f"c {i} {m} 0 {float(c[m])!r}")
        out.append(f"g {i} 0 0 {float(g)!r}")
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_snapshots.txt"), "w") as fh:
        fh.write("\n".join(lines()) + "\n")
