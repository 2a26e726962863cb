"""Python wrapper of the plain FP64 CPU oracle (``abm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` are the only callers.  The
product path (the CUDA library and ``paper_1611_08678_gb300``) never imports
this package and shares no code with it.

What the oracle computes is the fractional Adams-Bashforth-Moulton PECE scheme
of Section 2 (eq. (2) predictor, the corrector after it, and the weights
b_m, a_m, c_m), with weights evaluated in binary128 and everything else in
FP64 with sums in index order.  See the header of ``abm_oracle.c``.

Parity status per function (each pin lives in ``tests/test_oracle.py``):
  weights      pinned: mpmath 50-digit definitions, brute-force quadrature of
               the product-integration kernels, alpha = 1 closed values.
  solve        pinned: exact for y-independent linear forcing (corrector) and
               constant forcing (predictor), Mittag-Leffler convergence,
               alpha = 1 integral-form trapezoid identity, observed order.
  solve, passes > 1 (P(EC)^m E)
               pinned: on D^a y = lam y many passes reach the implicit
               corrector's solution, solved in closed form step by step;
               y-independent forcing gives the same result for every m.
  solve_ext    (orders in (0, 2], one per component, y'(0) in the Taylor sum)
               pinned: equal to ``solve`` operation for operation when the
               orders agree and are at most one; exact for y-independent
               linear forcing at orders above one; the alpha = 2 weights in
               closed form and order 2 on y'' = -y; Mittag-Leffler
               y0 E_a(lam t^a) + y1 t E_{a,2}(lam t^a); a decoupled Lorenz
               case whose components equal scalar solves at their own orders.
  tangent      pinned: central finite differences of ``solve``.
  history      pinned through the pinned solve: its predictor sum gives every
               y^P_{n+1} and its corrector sum (c_n at row 0, a_{n-k} beyond)
               every y_{n+1} of a solve; row ranges split and add up; three
               compiled mutants of it are rejected.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libabm_oracle.so")
_lock = threading.Lock()
_lib = None

SYSTEMS = {"linear": 0, "manufactured": 1, "lorenz": 2, "chen": 3, "rossler": 4, "financial": 5,
           "hindmarsh_rose": 6}

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no FMA contraction, IEEE semantics)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    import platform
    libs = ["-lquadmath"] if platform.machine() in ("x86_64", "AMD64", "i686") else []
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"] + libs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
    lib.oracle_dim.argtypes = [I]
    lib.oracle_nparams.argtypes = [I]
    lib.oracle_weights.argtypes = [D, L, _dp, _dp, _dp, _dp]
    lib.oracle_weights.restype = I
    lib.oracle_rhs.argtypes = [I, D, _dp, D, _dp, _dp]
    lib.oracle_rhs.restype = None
    lib.oracle_jac.argtypes = [I, D, _dp, D, _dp, _dp, _dp]
    lib.oracle_jac.restype = None
    lib.oracle_history.argtypes = [_dp, _dp, _dp, L, _dp, L, L, L, _dp, _dp]
    lib.oracle_history.restype = None
    lib.oracle_solve.argtypes = [I, D, D, L, _dp, _dp, _dp, _dp, _dp]
    lib.oracle_solve.restype = I
    lib.oracle_tangent.argtypes = [I, D, D, L, _dp, _dp, _dp, _dp, _dp]
    lib.oracle_tangent.restype = I
    lib.oracle_solve_pecm.argtypes = [I, D, D, L, _dp, _dp, I, _dp, _dp, _dp]
    lib.oracle_solve_pecm.restype = I
    lib.oracle_solve_ext.argtypes = [I, _dp, _dp, D, L, _dp, _dp, I, _dp, _dp, _dp]
    lib.oracle_solve_ext.restype = I
    return lib


def _load():
    global _lib
    if _current_override is not None:
        return _current_override
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


_current_override = None


class use_library:
    """Context manager: route this module's functions to another compiled copy
    of the oracle (used by the mutation tests, which compile deliberately
    broken copies of abm_oracle.c and check that the pins reject them)."""

    def __init__(self, path: str):
        self.lib = _bind(ctypes.CDLL(path))

    def __enter__(self):
        global _current_override
        self._prev = _current_override
        _current_override = self.lib
        return self

    def __exit__(self, *exc):
        global _current_override
        _current_override = self._prev
        return False


def compile_source(src_text: str, out_path: str) -> str:
    """Compile a (possibly modified) copy of the oracle source into out_path."""
    import platform
    c_path = out_path + ".c"
    with open(c_path, "w") as fh:
        fh.write(src_text)
    libs = ["-lquadmath"] if platform.machine() in ("x86_64", "AMD64", "i686") else []
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", c_path, "-o", out_path, "-lm"] + libs, check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _ptr(x: np.ndarray):
    assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data_as(_dp)


def _sys_id(system: str) -> int:
    if system not in SYSTEMS:
        raise ValueError(f"unknown system {system!r}")
    return SYSTEMS[system]


def dim(system: str) -> int:
    return _load().oracle_dim(_sys_id(system))


def nparams(system: str) -> int:
    return _load().oracle_nparams(_sys_id(system))


def weights(alpha: float, M: int):
    """(b, a, c, g): FP64 weights for lags m = 0..M (Sec. 2), from binary128."""
    b = np.empty(M + 1); a = np.empty(M + 1); c = np.empty(M + 1); g = np.empty(1)
    rc = _load().oracle_weights(float(alpha), int(M), _ptr(b), _ptr(a), _ptr(c), _ptr(g))
    if rc:
        raise ValueError("oracle_weights: bad arguments")
    return b, a, c, float(g[0])


def rhs(system: str, alpha: float, params, t: float, y) -> np.ndarray:
    d = dim(system)
    p = np.ascontiguousarray(params, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    f = np.empty(d)
    _load().oracle_rhs(_sys_id(system), float(alpha), _ptr(p), float(t), _ptr(yy), _ptr(f))
    return f


def jac(system: str, alpha: float, params, t: float, y):
    d, n_p = dim(system), nparams(system)
    p = np.ascontiguousarray(params, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    J = np.empty((d, d)); Q = np.empty((d, n_p))
    _load().oracle_jac(_sys_id(system), float(alpha), _ptr(p), float(t), _ptr(yy), _ptr(J), _ptr(Q))
    return J, Q


def history(b, a, c, F, n: int, k_lo: int, k_hi: int):
    """History sums of target step n over rows [k_lo, k_hi) (see abm_oracle.c)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    if F.ndim == 1:
        F = F[:, None]
    cols = F.shape[1]
    P = np.empty(cols); C = np.empty(cols)
    b = np.ascontiguousarray(b, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    assert len(b) > n and len(a) > n and len(c) > n and 0 <= k_lo <= k_hi <= n + 1
    _load().oracle_history(_ptr(b), _ptr(a), _ptr(c), cols, _ptr(F), int(n), int(k_lo), int(k_hi),
                           _ptr(P), _ptr(C))
    return P, C


def solve(system: str, alpha: float, h: float, N: int, params, y0, return_f: bool = False, passes: int = 1):
    """ABM PECE solve (passes = 1), or P(EC)^m E with m = passes corrector
    passes per step (oracle_solve_pecm).  Returns (Y, YP[, F]) with shape
    (N+1, d); Y[0] = YP[0] = y0."""
    d = dim(system)
    p = np.ascontiguousarray(params, dtype=np.float64)
    y0a = np.ascontiguousarray(y0, dtype=np.float64).reshape(d)
    Y = np.empty((N + 1, d)); YP = np.empty((N + 1, d))
    F = np.empty((N + 1, d)) if return_f else None
    if passes == 1:
        rc = _load().oracle_solve(_sys_id(system), float(alpha), float(h), int(N), _ptr(p), _ptr(y0a),
                                  _ptr(Y), _ptr(YP), _ptr(F) if return_f else None)
    else:
        rc = _load().oracle_solve_pecm(_sys_id(system), float(alpha), float(h), int(N), _ptr(p), _ptr(y0a),
                                       int(passes), _ptr(Y), _ptr(YP), _ptr(F) if return_f else None)
    if rc:
        raise ValueError(f"oracle_solve failed (rc={rc})")
    return (Y, YP, F) if return_f else (Y, YP)


def solve_ext(system: str, alpha, h: float, N: int, params, y0, y0d=None, passes: int = 1,
              return_f: bool = False):
    """The general problem of eq. (1) (oracle_solve_ext): alpha a scalar or
    one order per component, each in (0, 2]; y0d the initial derivatives
    y'(0) (used where alpha > 1; None = zero).  Returns (Y, YP[, F])."""
    d = dim(system)
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (d,)))
    p = np.ascontiguousarray(params, dtype=np.float64)
    y0a = np.ascontiguousarray(y0, dtype=np.float64).reshape(d)
    yd = None if y0d is None else np.ascontiguousarray(y0d, dtype=np.float64).reshape(d)
    Y = np.empty((N + 1, d)); YP = np.empty((N + 1, d))
    F = np.empty((N + 1, d)) if return_f else None
    rc = _load().oracle_solve_ext(_sys_id(system), _ptr(al), _ptr(yd) if yd is not None else None, float(h),
                                  int(N), _ptr(p), _ptr(y0a), int(passes), _ptr(Y), _ptr(YP),
                                  _ptr(F) if return_f else None)
    if rc:
        raise ValueError(f"oracle_solve_ext failed (rc={rc})")
    return (Y, YP, F) if return_f else (Y, YP)


def tangent(system: str, alpha: float, h: float, N: int, params, y0, dLdY):
    """Tangent-linear gradient: (dL/dparams, dL/dy0) for partials dLdY of shape (N+1, d)."""
    d, n_p = dim(system), nparams(system)
    p = np.ascontiguousarray(params, dtype=np.float64)
    y0a = np.ascontiguousarray(y0, dtype=np.float64).reshape(d)
    g = np.ascontiguousarray(dLdY, dtype=np.float64).reshape(N + 1, d)
    dp = np.empty(n_p); dy0 = np.empty(d)
    rc = _load().oracle_tangent(_sys_id(system), float(alpha), float(h), int(N), _ptr(p), _ptr(y0a),
                                _ptr(g), _ptr(dp), _ptr(dy0))
    if rc:
        raise ValueError(f"oracle_tangent failed (rc={rc})")
    return dp, dy0
