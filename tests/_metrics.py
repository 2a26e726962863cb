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


def chaos_stats_ratio(y, ref, refs_perturbed):
    """Statistics beyond the pointwise window of a chaotic run.

    Per component, min, max, mean and variance of y are compared with the
    reference run's.  The allowed difference is twice the largest difference
    between the reference and its own re-runs from initial values perturbed at
    the rounding level (the spread the flow itself creates), and at least 1e-3
    of the component's scale (range for min/max, standard deviation for the
    mean, variance for the variance).  Returns max(diff / allowed): <= 1 passes.
    """
    s_ref = stats(ref)
    spread = np.zeros_like(s_ref)
    for rp in refs_perturbed:
        spread = np.maximum(spread, np.abs(stats(rp) - s_ref))
    ref = np.asarray(ref, dtype=np.float64)
    rng = ref.max(axis=0) - ref.min(axis=0)
    sd = ref.std(axis=0)
    scale = np.stack([rng, rng, sd, ref.var(axis=0)])
    allowed = np.maximum(2.0 * spread, 1e-3 * scale)
    return float(np.max(np.abs(stats(y) - s_ref) / allowed))
