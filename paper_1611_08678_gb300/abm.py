"""ctypes binding of libabm_gb300.so (include/abm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory and streams.  There is no CPU path:
if the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libabm_gb300.so")
# the same library compiled with ABM_CHECKED: every layout-derived index is
# checked against its buffer (ABM_ERR_BOUNDS instead of an access outside it)
CHECKED_LIB_PATH = os.path.join(_HERE, "libabm_gb300_checked.so")

SYSTEMS = {"linear": 0, "manufactured": 1, "lorenz": 2, "chen": 3, "rossler": 4, "financial": 5,
           "hindmarsh_rose": 6}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16x3": 2, "bf16x6": 3}
STATUS = {0: "ABM_OK", 1: "ABM_ERR_INVALID_ARG", 2: "ABM_ERR_CUDA", 3: "ABM_ERR_OOM",
          4: "ABM_ERR_TIMEOUT", 5: "ABM_ERR_NONFINITE", 6: "ABM_ERR_UNSUPPORTED", 7: "ABM_ERR_BOUNDS"}

# Every symbol include/abm.h declares (checked by the CPU test suite).
EXPORTS = ["abm_plan_opts_default", "abm_system_dim", "abm_system_nparams", "abm_plan_create",
           "abm_plan_destroy", "abm_plan_sync", "abm_last_error", "abm_weights", "abm_solve",
           "abm_solve_batched", "abm_solve_batched_host", "abm_adjoint", "abm_far_history", "abm_solve_noalloc",
           "abm_plan_kernel_times", "abm_solve_ext", "abm_solve_batched_ext", "abm_history", "abm_solve_resume",
           "abm_history_batched", "abm_solve_batched_resume", "abm_solve_host"]
KERNEL_KINDS = {"weights": 0, "far": 1, "near": 2, "single": 3, "adjoint": 4}


class AbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanOpts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("n_max", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("tile_B", ctypes.c_int), ("far_ctas", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("spin_timeout_cycles", ctypes.c_longlong), ("test_withhold_tile", ctypes.c_int),
                ("profile", ctypes.c_int), ("near_warps", ctypes.c_int), ("far_split", ctypes.c_int),
                ("near_split", ctypes.c_int), ("corrector_passes", ctypes.c_int),
                ("test_bad_index", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


_libs = {}
_lock = threading.Lock()
_vp, _dp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)


def load(path: str = LIB_PATH):
    """Loads the library (builds it first when sources are newer).  Raises if
    it cannot be built or loaded; there is no fallback.  path: LIB_PATH, or
    CHECKED_LIB_PATH for the bounds-checked build."""
    with _lock:
        if path in _libs:
            return _libs[path]
        from . import build as _build
        if not _build.up_to_date(path):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing")
        lib = ctypes.CDLL(path)
        I, LL, D = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        lib.abm_plan_opts_default.argtypes = [ctypes.POINTER(PlanOpts)]
        lib.abm_plan_opts_default.restype = None
        lib.abm_system_dim.argtypes = [I]
        lib.abm_system_nparams.argtypes = [I]
        lib.abm_plan_create.argtypes = [ctypes.POINTER(_vp), I, ctypes.POINTER(PlanOpts)]
        lib.abm_plan_destroy.argtypes = [_vp]
        lib.abm_plan_sync.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int64)]
        lib.abm_last_error.argtypes = [_vp]
        lib.abm_last_error.restype = ctypes.c_char_p
        lib.abm_weights.argtypes = [_vp, D, I, _vp, _vp, _vp, _vp]
        lib.abm_solve.argtypes = [_vp, D, D, I, _dp, _dp, _vp, _vp, _vp]
        lib.abm_solve_batched.argtypes = [_vp, I, _dp, _dp, _ip, _vp, _vp, _vp, LL, _vp, _vp]
        lib.abm_solve_ext.argtypes = [_vp, _dp, D, I, _dp, _dp, _dp, _vp, _vp, _vp]
        lib.abm_solve_host.argtypes = [_vp, D, D, I, _dp, _dp, _vp, _vp, _vp]
        lib.abm_solve_batched_ext.argtypes = [_vp, I, _dp, _dp, _ip, _vp, _vp, _vp, _vp, LL, _vp, _vp]
        lib.abm_solve_batched_host.argtypes = [_vp, I, _dp, _dp, _ip, _vp, _vp, _vp, LL, _vp, _vp]
        lib.abm_history.argtypes = [_vp, I, _vp, _vp]
        lib.abm_solve_resume.argtypes = [_vp, _dp, D, I, I, _dp, _dp, _dp, _vp, _vp, _vp, _vp]
        lib.abm_history_batched.argtypes = [_vp, I, _dp, _dp, _ip, I, _vp, LL, _vp]
        lib.abm_solve_batched_resume.argtypes = [_vp, I, _dp, _dp, _ip, I, _vp, _vp, _vp, _vp, LL, _vp, LL, _vp, _vp]
        lib.abm_adjoint.argtypes = [_vp, I, _dp, _dp, _ip, _vp, _vp, _vp, _vp, LL, _vp, _vp, _vp, _vp]
        lib.abm_far_history.argtypes = [_vp, D, _vp, LL, LL, LL, I, LL, LL, _vp, _vp, _vp]
        lib.abm_plan_kernel_times.argtypes = [_vp, I, _vp, I, ctypes.POINTER(LL), ctypes.POINTER(D)]
        lib.abm_solve_noalloc.argtypes = [I, D, D, I, _dp, _dp, _vp, _vp, _vp, ctypes.c_char_p, ctypes.c_size_t]
        for name in EXPORTS:
            if name not in ("abm_plan_opts_default", "abm_last_error", "abm_system_dim", "abm_system_nparams"):
                getattr(lib, name).restype = I
        _libs[path] = lib
        return lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the ABM library has no CPU path")
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev_f64(x, numel, name):
    """A contiguous float64 CUDA tensor of x (copied when x is a host array, a
    host tensor or another dtype) holding exactly numel values."""
    torch = _torch()
    t = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
    if t.numel() != numel:
        raise ValueError(f"{name} holds {t.numel()} values, expected {numel}")
    return t


def _check_out(t, shape, name, cuda=True, more_rows=False):
    """Output buffers are written in place: they must already have the layout
    the library writes (float64, contiguous, on the right side of the bus).
    more_rows: the first dimension may be longer than the rows written."""
    torch = _torch()
    if t is None:
        return
    ok = (torch.is_tensor(t) and t.dtype == torch.float64 and t.is_contiguous() and t.is_cuda == cuda
          and t.dim() == len(shape))
    if ok:
        ok = (t.shape[0] >= shape[0] if more_rows else t.shape[0] == shape[0]) and \
            tuple(t.shape[1:]) == tuple(shape[1:])
    if not ok:
        where = "CUDA" if cuda else "host"
        want = f"{tuple(shape)}{' (or more rows)' if more_rows else ''}"
        got = (tuple(t.shape), t.dtype, t.device) if torch.is_tensor(t) else type(t)
        raise ValueError(f"{name} must be a contiguous float64 {where} tensor of shape {want}, got {got}")


class Plan:
    """One plan = one system, workspace for n_max steps and max_batch trajectories."""

    def __init__(self, system: str, n_max: int, max_batch: int = 0, prec: str = "fp64", tile_B: int = 0,
                 far_ctas: int = 0, use_graph: bool = False, spin_timeout_cycles: int = 0,
                 test_withhold_tile: int = 0, profile: bool = False, near_warps: int = 0,
                 far_split: int = 0, near_split: int = 0, corrector_passes: int = 1, checked: bool = False,
                 test_bad_index: int = 0):
        self.lib = load(CHECKED_LIB_PATH if checked else LIB_PATH)
        self.system = system
        self.d = self.lib.abm_system_dim(SYSTEMS[system])
        self.np = self.lib.abm_system_nparams(SYSTEMS[system])
        self.prec = prec
        o = PlanOpts()
        self.lib.abm_plan_opts_default(ctypes.byref(o))
        o.prec = PRECISIONS[prec]
        o.n_max = int(n_max)
        o.max_batch = int(max_batch)
        o.tile_B = int(tile_B)
        o.far_ctas = int(far_ctas)
        o.use_graph = int(bool(use_graph))
        o.spin_timeout_cycles = int(spin_timeout_cycles)
        o.test_withhold_tile = int(test_withhold_tile)
        o.profile = int(bool(profile))
        o.near_warps = int(near_warps)
        o.far_split = int(far_split)
        o.near_split = int(near_split)
        o.corrector_passes = int(corrector_passes)
        o.test_bad_index = int(test_bad_index)
        h = _vp()
        st = self.lib.abm_plan_create(ctypes.byref(h), SYSTEMS[system], ctypes.byref(o))
        if st != 0:
            raise AbmError(st, "abm_plan_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.abm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != 0:
            raise AbmError(st, f"{what}: {self.lib.abm_last_error(self.h).decode()}")

    def sync(self, stream=None):
        where = ctypes.c_int64(0)
        st = self.lib.abm_plan_sync(self.h, _stream_ptr(stream), ctypes.byref(where))
        self._check(st, "device status")
        return where.value

    def kernel_times(self, kind: str, reset: bool = True, stream=None):
        """(launches, total device ms) of one kernel kind since the last reset."""
        n = ctypes.c_longlong(0)
        ms = ctypes.c_double(0.0)
        self._check(self.lib.abm_plan_kernel_times(self.h, KERNEL_KINDS[kind], _stream_ptr(stream), int(reset),
                                                   ctypes.byref(n), ctypes.byref(ms)), "abm_plan_kernel_times")
        return n.value, ms.value

    # -- A1 --
    def weights(self, alpha: float, M: int, stream=None):
        torch = _torch()
        b, a, c = (torch.empty(M + 1, dtype=torch.float64, device="cuda") for _ in range(3))
        self._check(self.lib.abm_weights(self.h, float(alpha), int(M), _dptr(b), _dptr(a), _dptr(c),
                                         _stream_ptr(stream)), "abm_weights")
        return b, a, c

    # -- A2 alone (FP64 plans) --
    def far_history(self, alpha, F, s, B, k_lo, k_hi, stream=None):
        torch = _torch()
        rows, cols = F.shape
        _check_out(F, (rows, cols), "F")
        P = torch.empty(B, cols, dtype=torch.float64, device="cuda")
        C = torch.empty(B, cols, dtype=torch.float64, device="cuda")
        self._check(self.lib.abm_far_history(self.h, float(alpha), _dptr(F), rows, cols, int(s), int(B),
                                             int(k_lo), int(k_hi), _dptr(P), _dptr(C), _stream_ptr(stream)),
                    "abm_far_history")
        return P, C

    # -- single trajectory --
    def solve(self, alpha, h, N, params, y0, Y=None, YP=None, want_yp=False, stream=None, sync=True):
        torch = _torch()
        p = np.ascontiguousarray(params, dtype=np.float64)
        y = np.ascontiguousarray(y0, dtype=np.float64)
        if p.size != self.np or y.size != self.d:
            raise ValueError("params / y0 have the wrong size for this system")
        if Y is None:
            Y = torch.empty(N + 1, self.d, dtype=torch.float64, device="cuda")
        if YP is None and want_yp:
            YP = torch.empty(N + 1, self.d, dtype=torch.float64, device="cuda")
        _check_out(Y, (N + 1, self.d), "Y", more_rows=True)
        _check_out(YP, (N + 1, self.d), "YP", more_rows=True)
        st = self.lib.abm_solve(self.h, float(alpha), float(h), int(N), p.ctypes.data_as(_dp),
                                y.ctypes.data_as(_dp), _dptr(Y), _dptr(YP), _stream_ptr(stream))
        self._check(st, "abm_solve")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    def solve_host(self, alpha, h, N, params, y0, Y=None, YP=None, want_yp=False, stream=None, sync=True):
        """abm_solve_host: the single-trajectory solve with the result in host
        memory (torch CPU tensors of shape (N+1, d), page-locked when
        allocated here)."""
        torch = _torch()
        p = np.ascontiguousarray(params, dtype=np.float64)
        y = np.ascontiguousarray(y0, dtype=np.float64)
        if p.size != self.np or y.size != self.d:
            raise ValueError("params / y0 have the wrong size for this system")
        if Y is None:
            Y = torch.empty(N + 1, self.d, dtype=torch.float64, pin_memory=True)
        if YP is None and want_yp:
            YP = torch.empty(N + 1, self.d, dtype=torch.float64, pin_memory=True)
        _check_out(Y, (N + 1, self.d), "Y", cuda=False, more_rows=True)
        _check_out(YP, (N + 1, self.d), "YP", cuda=False, more_rows=True)
        st = self.lib.abm_solve_host(self.h, float(alpha), float(h), int(N), p.ctypes.data_as(_dp),
                                     y.ctypes.data_as(_dp), ctypes.c_void_p(Y.data_ptr()),
                                     ctypes.c_void_p(YP.data_ptr()) if YP is not None else None,
                                     _stream_ptr(stream))
        self._check(st, "abm_solve_host")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    def solve_ext(self, alpha, h, N, params, y0, y0d=None, Y=None, YP=None, want_yp=False, stream=None,
                  sync=True):
        """abm_solve_ext: the general problem of eq. (1) - alpha a scalar or one
        order per component, each in (0, 2]; y0d the initial derivatives y'(0)
        (None: zero), used by components of order above one."""
        torch = _torch()
        al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (self.d,)))
        p = np.ascontiguousarray(params, dtype=np.float64)
        y = np.ascontiguousarray(y0, dtype=np.float64)
        yd = None if y0d is None else np.ascontiguousarray(y0d, dtype=np.float64)
        if p.size != self.np or y.size != self.d or (yd is not None and yd.size != self.d):
            raise ValueError("params / y0 / y0d have the wrong size for this system")
        if Y is None:
            Y = torch.empty(N + 1, self.d, dtype=torch.float64, device="cuda")
        if YP is None and want_yp:
            YP = torch.empty(N + 1, self.d, dtype=torch.float64, device="cuda")
        _check_out(Y, (N + 1, self.d), "Y", more_rows=True)
        _check_out(YP, (N + 1, self.d), "YP", more_rows=True)
        st = self.lib.abm_solve_ext(self.h, al.ctypes.data_as(_dp), float(h), int(N), p.ctypes.data_as(_dp),
                                    y.ctypes.data_as(_dp), yd.ctypes.data_as(_dp) if yd is not None else None,
                                    _dptr(Y), _dptr(YP), _stream_ptr(stream))
        self._check(st, "abm_solve_ext")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    # -- checkpoint / resume --
    def history(self, rows, F=None, stream=None, sync=True):
        """abm_history: f_0..f_{rows-1} of the last single-trajectory solve
        (a CUDA tensor (rows, d), or F given: CUDA or host float64 tensor)."""
        torch = _torch()
        if F is None:
            F = torch.empty(rows, self.d, dtype=torch.float64, device="cuda")
        _check_out(F, (rows, self.d), "F", cuda=F.is_cuda)
        self._check(self.lib.abm_history(self.h, int(rows), _dptr(F), _stream_ptr(stream)), "abm_history")
        if sync:
            self.sync(stream)
        return F

    def solve_resume(self, alpha, h, n0, N, params, y0, F, y0d=None, Y=None, YP=None, want_yp=False,
                     stream=None, sync=True):
        """abm_solve_resume: continue from step n0 to N with F = f_0..f_n0."""
        torch = _torch()
        al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (self.d,)))
        p = np.ascontiguousarray(params, dtype=np.float64)
        y = np.ascontiguousarray(y0, dtype=np.float64)
        yd = None if y0d is None else np.ascontiguousarray(y0d, dtype=np.float64)
        if p.size != self.np or y.size != self.d or (yd is not None and yd.size != self.d):
            raise ValueError("params / y0 / y0d have the wrong size for this system")
        if not (torch.is_tensor(F) and F.dtype == torch.float64 and F.is_contiguous() and F.numel() >= (n0 + 1) * self.d):
            raise ValueError("F must be a contiguous float64 tensor holding rows 0..n0")
        if Y is None:
            Y = torch.empty(N + 1, self.d, dtype=torch.float64, device="cuda")
        if YP is None and want_yp:
            YP = torch.empty(N + 1, self.d, dtype=torch.float64, device="cuda")
        _check_out(Y, (N + 1, self.d), "Y", more_rows=True)
        _check_out(YP, (N + 1, self.d), "YP", more_rows=True)
        st = self.lib.abm_solve_resume(self.h, al.ctypes.data_as(_dp), float(h), int(n0), int(N),
                                       p.ctypes.data_as(_dp), y.ctypes.data_as(_dp),
                                       yd.ctypes.data_as(_dp) if yd is not None else None, _dptr(F), _dptr(Y),
                                       _dptr(YP), _stream_ptr(stream))
        self._check(st, "abm_solve_resume")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    def _orders(self, alpha, M):
        al = np.asarray(alpha, dtype=np.float64)
        return np.ascontiguousarray(np.broadcast_to(al.reshape(M, -1), (M, self.d)))

    def history_batched(self, alpha, h, N, rows, F=None, ldF=None, stream=None, sync=True):
        """abm_history_batched: (M, ldF, d) CUDA tensor with f_0..f_min(rows, N_i+1)-1
        of every trajectory of the last batched solve (same alpha, h, N)."""
        torch = _torch()
        hh = np.ascontiguousarray(h, dtype=np.float64)
        NN = np.ascontiguousarray(N, dtype=np.int32)
        M = NN.size
        al = self._orders(alpha, M)
        ldF = int(ldF or rows)
        if F is None:
            F = torch.zeros(M, ldF, self.d, dtype=torch.float64, device="cuda")
        _check_out(F, (M, ldF, self.d), "F")
        st = self.lib.abm_history_batched(self.h, M, al.ctypes.data_as(_dp), hh.ctypes.data_as(_dp),
                                          NN.ctypes.data_as(_ip), int(rows), _dptr(F), ldF, _stream_ptr(stream))
        self._check(st, "abm_history_batched")
        if sync:
            self.sync(stream)
        return F

    def solve_batched_resume(self, alpha, h, N, n0, params, y0, F, y0d=None, Y=None, YP=None, ldY=None,
                             stream=None, sync=True):
        """abm_solve_batched_resume: continue every trajectory from step n0
        (F: (M, ldF, d) CUDA tensor of f_0..f_n0)."""
        torch = _torch()
        hh = np.ascontiguousarray(h, dtype=np.float64)
        NN = np.ascontiguousarray(N, dtype=np.int32)
        M = NN.size
        al = self._orders(alpha, M)
        params = _dev_f64(params, M * self.np, "params")
        y0 = _dev_f64(y0, M * self.d, "y0")
        yd = None if y0d is None else _dev_f64(y0d, M * self.d, "y0d")
        if not (torch.is_tensor(F) and F.is_cuda and F.dtype == torch.float64 and F.is_contiguous() and F.dim() == 3
                and F.shape[0] == M and F.shape[2] == self.d):
            raise ValueError("F must be a contiguous float64 CUDA tensor of shape (M, ldF, d)")
        if ldY is None:
            ldY = int(NN.max()) + 1
        if Y is None:
            Y = torch.zeros(M, ldY, self.d, dtype=torch.float64, device="cuda")
        _check_out(Y, (M, ldY, self.d), "Y")
        _check_out(YP, (M, ldY, self.d), "YP")
        self._ext_inputs = yd
        st = self.lib.abm_solve_batched_resume(self.h, M, al.ctypes.data_as(_dp), hh.ctypes.data_as(_dp),
                                               NN.ctypes.data_as(_ip), int(n0), _dptr(params), _dptr(y0), _dptr(yd),
                                               _dptr(F), int(F.shape[1]), _dptr(Y), int(ldY), _dptr(YP),
                                               _stream_ptr(stream))
        self._check(st, "abm_solve_batched_resume")
        if sync:
            self.sync(stream)
        return Y

    # -- batched --
    def solve_batched_ext(self, alpha, h, N, params, y0, y0d=None, Y=None, YP=None, want_yp=False, ldY=None,
                          stream=None, sync=True):
        """abm_solve_batched_ext: alpha (M,) or (M, d) orders in (0, 2] (host);
        y0d (M, d) initial derivatives (copied to the device) or None."""
        torch = _torch()
        hh = np.ascontiguousarray(h, dtype=np.float64)
        NN = np.ascontiguousarray(N, dtype=np.int32)
        M = NN.size
        al = np.asarray(alpha, dtype=np.float64)
        al = np.ascontiguousarray(np.broadcast_to(al.reshape(M, -1), (M, self.d)))
        if hh.size != M:
            raise ValueError("alpha, h and N need one entry per trajectory")
        params = _dev_f64(params, M * self.np, "params")
        y0 = _dev_f64(y0, M * self.d, "y0")
        yd = None if y0d is None else _dev_f64(y0d, M * self.d, "y0d")
        if ldY is None:
            ldY = int(NN.max()) + 1 if NN.size else 1
        if Y is None:
            Y = torch.zeros(M, ldY, self.d, dtype=torch.float64, device="cuda")
        if YP is None and want_yp:
            YP = torch.zeros(M, ldY, self.d, dtype=torch.float64, device="cuda")
        _check_out(Y, (M, ldY, self.d), "Y")
        _check_out(YP, (M, ldY, self.d), "YP")
        self._ext_inputs = yd  # kept alive until the asynchronous solve has read it
        st = self.lib.abm_solve_batched_ext(self.h, M, al.ctypes.data_as(_dp), hh.ctypes.data_as(_dp),
                                            NN.ctypes.data_as(_ip), _dptr(params), _dptr(y0), _dptr(yd), _dptr(Y),
                                            int(ldY), _dptr(YP), _stream_ptr(stream))
        self._check(st, "abm_solve_batched_ext")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    def solve_batched(self, alpha, h, N, params, y0, Y=None, YP=None, want_yp=False, ldY=None, stream=None,
                      sync=True):
        """alpha, h, N: host sequences (scheduling); params (M, np), y0 (M, d):
        torch CUDA tensors or host arrays (copied).  Returns Y (M, ldY, d)."""
        torch = _torch()
        al = np.ascontiguousarray(alpha, dtype=np.float64)
        hh = np.ascontiguousarray(h, dtype=np.float64)
        NN = np.ascontiguousarray(N, dtype=np.int32)
        M = al.size
        if hh.size != M or NN.size != M:
            raise ValueError("alpha, h and N need one entry per trajectory")
        params = _dev_f64(params, M * self.np, "params")
        y0 = _dev_f64(y0, M * self.d, "y0")
        if ldY is None:
            ldY = int(NN.max()) + 1 if NN.size else 1  # an empty batch reaches the library's M check
        if Y is None:
            Y = torch.zeros(M, ldY, self.d, dtype=torch.float64, device="cuda")
        if YP is None and want_yp:
            YP = torch.zeros(M, ldY, self.d, dtype=torch.float64, device="cuda")
        _check_out(Y, (M, ldY, self.d), "Y")
        _check_out(YP, (M, ldY, self.d), "YP")
        st = self.lib.abm_solve_batched(self.h, M, al.ctypes.data_as(_dp), hh.ctypes.data_as(_dp),
                                        NN.ctypes.data_as(_ip), _dptr(params), _dptr(y0), _dptr(Y), int(ldY),
                                        _dptr(YP), _stream_ptr(stream))
        self._check(st, "abm_solve_batched")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    def solve_batched_host(self, alpha, h, N, params, y0, Y=None, YP=None, want_yp=False, ldY=None,
                           stream=None, sync=True):
        """abm_solve_batched_host: params (M, np), y0 (M, d) and the results Y
        (M, ldY, d) [and YP] in host memory (torch CPU tensors, page-locked
        when allocated here); the library copies inputs up and each finished
        trajectory down while later time tiles run."""
        torch = _torch()
        al = np.ascontiguousarray(alpha, dtype=np.float64)
        hh = np.ascontiguousarray(h, dtype=np.float64)
        NN = np.ascontiguousarray(N, dtype=np.int32)
        M = al.size
        if hh.size != M or NN.size != M:
            raise ValueError("alpha, h and N need one entry per trajectory")
        params = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float64)) if not torch.is_tensor(params) \
            else params
        y0 = torch.as_tensor(np.ascontiguousarray(y0, dtype=np.float64)) if not torch.is_tensor(y0) else y0
        if params.is_cuda or y0.is_cuda:
            raise ValueError("solve_batched_host takes host tensors; use solve_batched for device tensors")
        params = params.to(torch.float64).contiguous()
        y0 = y0.to(torch.float64).contiguous()
        if params.numel() != M * self.np or y0.numel() != M * self.d:
            raise ValueError("params / y0 need n_params / d values per trajectory")
        if ldY is None:
            ldY = int(NN.max()) + 1 if NN.size else 1  # an empty batch reaches the library's M check
        if Y is None:
            Y = torch.zeros(M, ldY, self.d, dtype=torch.float64, pin_memory=True)
        if YP is None and want_yp:
            YP = torch.zeros(M, ldY, self.d, dtype=torch.float64, pin_memory=True)
        _check_out(Y, (M, ldY, self.d), "Y", cuda=False)
        _check_out(YP, (M, ldY, self.d), "YP", cuda=False)
        self._host_inputs = (params, y0)  # read by the asynchronous upload
        st = self.lib.abm_solve_batched_host(self.h, M, al.ctypes.data_as(_dp), hh.ctypes.data_as(_dp),
                                             NN.ctypes.data_as(_ip), ctypes.c_void_p(params.data_ptr()),
                                             ctypes.c_void_p(y0.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                             int(ldY), ctypes.c_void_p(YP.data_ptr()) if YP is not None else None,
                                             _stream_ptr(stream))
        self._check(st, "abm_solve_batched_host")
        if sync:
            self.sync(stream)
        return (Y, YP) if want_yp or YP is not None else Y

    def adjoint(self, alpha, h, N, params, y0, Y, YP, dLdY, stream=None, sync=True):
        torch = _torch()
        al = np.ascontiguousarray(alpha, dtype=np.float64)
        hh = np.ascontiguousarray(h, dtype=np.float64)
        NN = np.ascontiguousarray(N, dtype=np.int32)
        M = al.size
        if hh.size != M or NN.size != M:
            raise ValueError("alpha, h and N need one entry per trajectory")
        params = _dev_f64(params, M * self.np, "params")
        y0 = _dev_f64(y0, M * self.d, "y0")
        ldY = int(Y.shape[1]) if torch.is_tensor(Y) and Y.dim() == 3 else -1
        _check_out(Y, (M, ldY, self.d), "Y")
        _check_out(YP, (M, ldY, self.d), "YP")
        dLdY = _dev_f64(dLdY, M * ldY * self.d, "dLdY")
        dp = torch.empty(M, self.np, dtype=torch.float64, device="cuda")
        dy0 = torch.empty(M, self.d, dtype=torch.float64, device="cuda")
        st = self.lib.abm_adjoint(self.h, M, al.ctypes.data_as(_dp), hh.ctypes.data_as(_dp),
                                  NN.ctypes.data_as(_ip), _dptr(params), _dptr(y0),
                                  _dptr(Y), _dptr(YP), ldY, _dptr(dLdY), _dptr(dp),
                                  _dptr(dy0), _stream_ptr(stream))
        self._check(st, "abm_adjoint")
        if sync:
            self.sync(stream)
        return dp, dy0


def solve_noalloc(system: str, alpha, h, N, params, y0, Y, YP=None, stream=None):
    """abm_solve_noalloc: single-trajectory solve whose scratch is the
    library's static device array (no allocation).  Y (and YP) are
    caller-provided CUDA tensors of shape (N+1, d).  Synchronous."""
    lib = load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    y = np.ascontiguousarray(y0, dtype=np.float64)
    d = lib.abm_system_dim(SYSTEMS[system])
    if p.size != lib.abm_system_nparams(SYSTEMS[system]) or y.size != d:
        raise ValueError("params / y0 have the wrong size for this system")
    _check_out(Y, (N + 1, d), "Y", more_rows=True)
    _check_out(YP, (N + 1, d), "YP", more_rows=True)
    buf = ctypes.create_string_buffer(256)
    st = lib.abm_solve_noalloc(SYSTEMS[system], float(alpha), float(h), int(N), p.ctypes.data_as(_dp),
                               y.ctypes.data_as(_dp), _dptr(Y), _dptr(YP), _stream_ptr(stream), buf, 256)
    if st != 0:
        raise AbmError(st, buf.value.decode())
    return Y
