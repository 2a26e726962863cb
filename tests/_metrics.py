"""Error measures shared by the parity tests.

rel_err: max over steps of |y_gpu - y_ref|_inf / max(|y_ref_n|_inf, 1e-3 max_m |y_ref_m|_inf)
(the floor keeps zero crossings from dominating).
stats_close: per component min, max, mean and variance over a window, each
compared relatively (attractor bounds and time-averaged moments).
"""
import numpy as np


def rel_err(y, ref):
    y = np.asarray(y, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    nrm = np.abs(ref).max(axis=1)
    floor = 1e-3 * nrm.max() if nrm.size else 0.0
    den = np.maximum(nrm, max(floor, 1e-300))
    return float(np.max(np.abs(y - ref).max(axis=1) / den)) if len(ref) else 0.0


def stats(y):
    y = np.asarray(y, dtype=np.float64)
    return np.stack([y.min(axis=0), y.max(axis=0), y.mean(axis=0), y.var(axis=0)])


def stats_rel_diff(y, ref):
    a, b = stats(y), stats(ref)
    scale = np.maximum(np.abs(b), 1e-12)
    return float(np.max(np.abs(a - b) / scale))
