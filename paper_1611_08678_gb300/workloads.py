"""Seeded synthetic inputs for the fractional ABM workloads.

This module holds no arithmetic of the method: it only draws parameters,
orders and initial values.  Both the test suite (oracle side and GPU side) and
the benchmark take their inputs from here, so the two sides see identical
inputs.  Seeds: 1611 for inputs, 8678 for perturbations and targets.

Workloads (the paper gives no dataset; its Hindmarsh-Rose run lacks parameters,
so these synthetic systems stand in, with the shapes named below):
  lorenz_single     fractional Lorenz, sigma=10, rho=28, beta=8/3, alpha=0.98,
                    y0=(0.1,0.1,0.1), h=0.01, N=8192, d=3
  chen_single       fractional Chen, a=35, b=3, c=28, alpha=0.9,
                    y0=(-9,-5,14), h=0.001, N=2^18, d=3
  rossler_batched   4096 fractional Roessler trajectories, a=b=0.2,
                    c ~ U[4,12], alpha from linspace(0.85, 1.0, 8),
                    y0 ~ U[-1,1]^3, h=0.005, N_i = floor(exp(U[ln 2^12, ln 2^16]))
  financial_batched 16384 fractional financial-system trajectories, a=3,
                    b=0.1, c=1, alpha=0.95, y0=(2,3,2)+N(0,0.01^2), h=0.01, N=2^16
  lorenz_adjoint    1024 fractional Lorenz trajectories, alpha=0.98, h=0.01,
                    N=2^14, (sigma,rho,beta) ~ N((10,28,8/3), 0.1^2),
                    y0 ~ (0.1,0.1,0.1)+N(0,0.01^2); target trajectories from
                    parameters perturbed by N(0, 0.1^2)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_INPUTS = 1611
SEED_PERTURB = 8678

DIMS = {"linear": 1, "manufactured": 1, "lorenz": 3, "chen": 3, "rossler": 3, "financial": 3,
        "hindmarsh_rose": 3}
NPARAMS = {"linear": 3, "manufactured": 9, "lorenz": 3, "chen": 3, "rossler": 3, "financial": 3,
           "hindmarsh_rose": 8}

# The 3-D Hindmarsh-Rose model in its chaotic-bursting regime: (a, b, c, d, r,
# s, xR, I).  The paper simulates this model (Sec. 4) without stating its
# parameters, alpha, h or y0; these are this project's choices.
HR_PARAMS = [1.0, 3.0, 1.0, 5.0, 0.006, 4.0, -1.6, 3.25]


@dataclass
class Batch:
    """M independent trajectories of one system (host arrays, FP64 / int64)."""
    system: str
    alpha: np.ndarray   # (M,)
    h: np.ndarray       # (M,)
    N: np.ndarray       # (M,) int64
    params: np.ndarray  # (M, n_params)
    y0: np.ndarray      # (M, d)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.alpha.shape[0])

    @property
    def d(self) -> int:
        return DIMS[self.system]

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx)
        return Batch(self.system, self.alpha[idx].copy(), self.h[idx].copy(), self.N[idx].copy(),
                     self.params[idx].copy(), self.y0[idx].copy(), self.name, dict(self.meta))

    def history_macs(self) -> float:
        """Predictor + corrector history multiply-adds: sum_i N_i (N_i + 1) d."""
        n = self.N.astype(np.float64)
        return float(np.sum(n * (n + 1.0)) * self.d)


def _single(system, alpha, h, N, params, y0, name):
    return Batch(system, np.array([alpha], float), np.array([h], float), np.array([N], np.int64),
                 np.array([params], float), np.array([y0], float), name)


def lorenz_single(N: int = 8192) -> Batch:
    return _single("lorenz", 0.98, 0.01, N, [10.0, 28.0, 8.0 / 3.0], [0.1, 0.1, 0.1], "lorenz_single")


def chen_single(N: int = 1 << 18) -> Batch:
    return _single("chen", 0.9, 0.001, N, [35.0, 3.0, 28.0], [-9.0, -5.0, 14.0], "chen_single")


def hindmarsh_rose_single(N: int = 100000) -> Batch:
    """The paper's workload at its own sizes (N = 1e5 .. 3e6 in Table 2)."""
    return _single("hindmarsh_rose", 0.98, 0.01, N, HR_PARAMS, [0.1, 0.2, 0.3], "hindmarsh_rose_single")


def rossler_batched(M: int = 4096, n_lo: int = 1 << 12, n_hi: int = 1 << 16, n_alpha: int = 8,
                    seed: int = SEED_INPUTS, alpha_grid: str = "linspace8") -> Batch:
    rng = np.random.default_rng(seed)
    c = rng.uniform(4.0, 12.0, M)
    if alpha_grid == "linspace8":
        grid = np.linspace(0.85, 1.0, n_alpha)
    else:  # the 7-point step-0.025 grid variant
        grid = np.arange(0.85, 1.0 + 1e-9, 0.025)
    alpha = grid[rng.integers(0, len(grid), M)]
    y0 = rng.uniform(-1.0, 1.0, (M, 3))
    N = np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), M))).astype(np.int64)
    N = np.clip(N, n_lo, n_hi)
    params = np.stack([np.full(M, 0.2), np.full(M, 0.2), c], axis=1)
    return Batch("rossler", alpha, np.full(M, 0.005), N, params, y0, "rossler_batched",
                 {"alpha_grid": alpha_grid})


def financial_batched(M: int = 16384, N: int = 1 << 16, seed: int = SEED_INPUTS) -> Batch:
    rng = np.random.default_rng(seed)
    y0 = np.array([2.0, 3.0, 2.0]) + rng.normal(0.0, 0.01, (M, 3))
    params = np.tile(np.array([3.0, 0.1, 1.0]), (M, 1))
    return Batch("financial", np.full(M, 0.95), np.full(M, 0.01), np.full(M, N, np.int64),
                 params, y0, "financial_batched")


def lorenz_adjoint(M: int = 1024, N: int = 1 << 14, seed: int = SEED_INPUTS):
    """Returns (batch, target_params): the loss is the mean squared distance of
    each trajectory to the trajectory of its perturbed parameters."""
    rng = np.random.default_rng(seed)
    params = np.array([10.0, 28.0, 8.0 / 3.0]) + rng.normal(0.0, 0.1, (M, 3))
    y0 = np.array([0.1, 0.1, 0.1]) + rng.normal(0.0, 0.01, (M, 3))
    prng = np.random.default_rng(SEED_PERTURB)
    target_params = params + prng.normal(0.0, 0.1, (M, 3))
    b = Batch("lorenz", np.full(M, 0.98), np.full(M, 0.01), np.full(M, N, np.int64), params, y0,
              "lorenz_adjoint")
    return b, target_params


def random_batch(system: str, M: int, n_lo: int, n_hi: int, alphas, h: float = 0.01,
                 seed: int = SEED_INPUTS) -> Batch:
    """Small mixed batches for parity tests: ragged N, several alpha values."""
    rng = np.random.default_rng(seed)
    d = DIMS[system]
    N = rng.integers(n_lo, n_hi + 1, M).astype(np.int64)
    alpha = np.asarray(alphas, float)[rng.integers(0, len(alphas), M)]
    if system == "lorenz":
        params = np.array([10.0, 28.0, 8.0 / 3.0]) + rng.normal(0.0, 0.1, (M, 3))
        y0 = np.array([0.1, 0.1, 0.1]) + rng.normal(0.0, 0.01, (M, 3))
    elif system == "rossler":
        params = np.stack([np.full(M, 0.2), np.full(M, 0.2), rng.uniform(4, 12, M)], axis=1)
        y0 = rng.uniform(-1, 1, (M, 3))
    elif system == "financial":
        params = np.tile(np.array([3.0, 0.1, 1.0]), (M, 1))
        y0 = np.array([2.0, 3.0, 2.0]) + rng.normal(0.0, 0.01, (M, 3))
    elif system == "chen":
        params = np.tile(np.array([35.0, 3.0, 28.0]), (M, 1))
        y0 = np.array([-9.0, -5.0, 14.0]) + rng.normal(0.0, 0.1, (M, 3))
    elif system == "hindmarsh_rose":
        params = np.tile(np.array(HR_PARAMS), (M, 1))
        params[:, 7] = rng.uniform(2.9, 3.3, M)  # the input current I
        y0 = rng.uniform(-1, 1, (M, 3))
    elif system == "linear":
        params = np.stack([rng.uniform(-2, 0.5, M), rng.uniform(-1, 1, M), rng.uniform(-1, 1, M)], axis=1)
        y0 = rng.uniform(-1, 1, (M, 1))
    else:
        raise ValueError(system)
    return Batch(system, alpha, np.full(M, h), N, params, y0, f"random_{system}")
