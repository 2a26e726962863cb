#!/usr/bin/env python
"""Benchmark of the fractional ABM history convolution on GB300.

Default workload: 16384 fractional financial-system trajectories
(a=3, b=0.1, c=1, alpha=0.95, y0=(2,3,2)+N(0,0.01^2), h=0.01, N=2^16, d=3),
the batched path with FP64 state and the far history on the tensor cores
(BF16x6 split).  One "step" = one whole batched solve.  Metric:
trajectory-steps/s and history MAC/s, measured beside the plain FP64 GPU path
(the same library with the far history in FP64) at the error each reaches
against the FP64 CPU oracle.  The plain FP64 path is timed on a seeded subset
of the trajectories and extrapolated by far-history multiply-adds (a full
FP64 solve of this workload runs for minutes); the line says so.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload financial_batched|rossler_batched|lorenz_adjoint|
                              chen_single|lorenz_single|hindmarsh_rose_single]
                  [--prec bf16x6|bf16x3|fp32|fp64] [--arms bf16x3,fp32,...]

Multi-GPU (torchrun, one rank per GPU): single-trajectory workloads run one
replica per rank (the path does not shard); batched workloads shard the
trajectories across ranks.  Both are weak scaling with no data-path
collective; the timing is the max over ranks.

The oracle (plain FP64 CPU implementation under oracle/) is executed here only
for the cpu_baseline leg, the error statements and --impl reference.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# GB300's nominal dense FP64 rate (NVIDIA's published figure, 1.25 TFLOP/s)
# is the peak of the FP64-ALU-bound kernels; a DFMA throughput test on the
# same GPUs reads 0.97 TFLOP/s and the single-trajectory solve reaches 1.2, so
# the nominal figure is the one quoted.  The HBM and BF16 tensor peaks are the
# measured ones in MEASURED_PEAKS.json.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flop x max clock


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0  # an earlier GB300 measurement, used when the file is absent


HBM_PEAK_GBS, BF16_PEAK_TFLOPS = _measured_peaks()

# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture of the current kernel; None when the kernel changed since the
# counters were taken.
NCU_TRAFFIC = {
    "chen_single": 6780160 + 96000,  # the 2^18-step Chen solve
}
# Batched far kernel: DRAM bytes of one captured launch over the algorithmic
# operand bytes of that launch, per workload and precision (ncu captures of
# the current kernel on a 512-trajectory Rossler and a 1024-trajectory
# financial case, time tile 38464); the bench line scales it to its own
# average launch, since DRAM bytes grow with the operand bytes.
NCU_TRAFFIC_RATIO = {
    "rossler_batched_bf16x6": (414429952 + 3411456) / 413564928,
    "financial_batched_bf16x6": (741771776 + 3026176) / 738508800,
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="financial_batched",
                    choices=["chen_single", "lorenz_single", "hindmarsh_rose_single", "rossler_batched",
                             "financial_batched", "lorenz_adjoint"])
    ap.add_argument("--n", type=int, default=0, help="single-trajectory workloads: number of steps N")
    ap.add_argument("--prec", default=None, help="far-history precision of batched workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mib", type=int, default=256)
    ap.add_argument("--no-tune", action="store_true", help="batched: skip the autotuner (library defaults)")
    ap.add_argument("--knobs", default="",
                    help="batched: far_split,near_warps,near_split to use instead of tuning (e.g. the "
                         "values a full-size run tuned, for a small profiling case)")
    ap.add_argument("--corrector-passes", type=int, default=1,
                    help="batched: corrector passes per step (1 = PECE, m > 1 = P(EC)^m E)")
    ap.add_argument("--trajectories", type=int, default=0,
                    help="batched workloads: first M trajectories only (small cases for profiling)")
    ap.add_argument("--arms", default="bf16x3,fp32",
                    help="batched: further far-history precisions run on the full workload beside the "
                         "headline one (comma list of bf16x3, bf16x6, fp32, fp64; empty for none)")
    ap.add_argument("--no-comparator", action="store_true",
                    help="batched: skip the plain FP64 GPU path")
    ap.add_argument("--comparator-trajectories", type=int, default=512,
                    help="batched: trajectories of the seeded subset the plain FP64 GPU path runs")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# Paper, Table 2: average CUDA run time (s) of the 3-D Hindmarsh-Rose model per
# number of steps N (unnamed GPU, parameters and precision not stated): context
# beside the Hindmarsh-Rose bench line, not a target.
PAPER_TABLE2_CUDA_S = {100000: 169.06, 500000: 1276.42, 1000000: 2670.56, 1500000: 4450.09,
                       2000000: 6639.45, 2500000: 9229.66, 3000000: 12226.39}


def workload(name, n=0):
    from paper_1611_08678_gb300 import workloads as wl
    if name == "chen_single":
        return (wl.chen_single(n) if n else wl.chen_single()), "fp64"
    if name == "lorenz_single":
        return (wl.lorenz_single(n) if n else wl.lorenz_single()), "fp64"
    if name == "hindmarsh_rose_single":
        return (wl.hindmarsh_rose_single(n) if n else wl.hindmarsh_rose_single()), "fp64"
    if name == "rossler_batched":
        return wl.rossler_batched(), "bf16x6"
    if name == "financial_batched":
        return wl.financial_batched(), "bf16x6"
    if name == "lorenz_adjoint":
        return wl.lorenz_adjoint()[0], "bf16x6"
    raise ValueError(name)


def is_single(name):
    return name.endswith("_single")


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        loaded = [x for x in sm if x > 0.5 * max(sm)] if sm else []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
def rel_err(y, ref):
    """max_n |y_n - ref_n|_inf / max(|ref_n|_inf, 1e-3 max_m |ref_m|_inf)"""
    import numpy as np
    nrm = np.abs(ref).max(axis=1)
    den = np.maximum(nrm, 1e-3 * nrm.max())
    return float(np.max(np.abs(y - ref).max(axis=1) / den))


def stats_rel_diff(y, ref):
    """Largest relative difference of the per-component min, max, mean and
    variance of y against ref (floors: 1e-3 of the range, std or variance)."""
    import numpy as np
    st = lambda a: np.stack([a.min(axis=0), a.max(axis=0), a.mean(axis=0), a.var(axis=0)])
    sy, sr = st(np.asarray(y)), st(np.asarray(ref))
    rng = np.ptp(ref, axis=0)
    scale = np.stack([rng, rng, ref.std(axis=0), ref.var(axis=0)])
    return float(np.max(np.abs(sy - sr) / np.maximum(np.abs(sr), 1e-3 * scale)))


def oracle_single_rate(w, n_sample):
    """Oracle (CPU, one thread) on the first n_sample steps of a single
    trajectory; returns (seconds, Y)."""
    import oracle
    t0 = time.perf_counter()
    Y, _ = oracle.solve(w.system, float(w.alpha[0]), float(w.h[0]), n_sample, w.params[0], w.y0[0])
    return time.perf_counter() - t0, Y


def single_cpu_baseline(w, n_sample):
    """Oracle MAC rate on the sample, scaled to full-workload trajectory-steps/s."""
    N, d = int(w.N[0]), w.d
    sec, Y = oracle_single_rate(w, n_sample)
    mac_rate = n_sample * (n_sample + 1) * d / sec
    steps_per_s = mac_rate / ((N + 1) * d)  # a full solve costs (N+1) d MACs per step on average
    return {"value": steps_per_s, "unit": "trajectory-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_sample} steps of the {N}-step trajectory on 1 host thread "
                      f"({sec:.2f} s), scaled by history MACs to the full solve",
            "history_mac_per_s": mac_rate}, Y


def bench_single(args, name, w, world, rank, local):
    import numpy as np
    import torch

    from paper_1611_08678_gb300 import abm
    N, d = int(w.N[0]), w.d
    alpha, h = float(w.alpha[0]), float(w.h[0])
    plan = abm.Plan(w.system, n_max=N)
    Y = torch.empty(N + 1, d, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(args.flush_mib * (1 << 20) // 4, dtype=torch.float32, device="cuda")

    def step():
        plan.solve(alpha, h, N, w.params[0], w.y0[0], Y=Y, sync=False, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    plan.sync(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between timed steps (outside the event pair)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    plan.sync(stream)  # raises on any device-side error
    per_step = [a.elapsed_time(b) / 1e3 for a, b in ev]
    total = sum(per_step)
    t = torch.tensor([total], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_max = float(t.item())
    steps_total = args.steps * N * world
    value = steps_total / total_max
    macs = N * (N + 1) * d
    mean_launch = total / args.steps
    achieved = 2.0 * macs / mean_launch / 1e12

    # e2e: one C-ABI call with host buffers (abm_solve_host): params / y0 from
    # host memory (passed by value), the solution written to pinned host
    # memory, every step.
    Yh = torch.empty(N + 1, d, dtype=torch.float64, pin_memory=True)
    p_host = np.ascontiguousarray(w.params[0], dtype=np.float64)
    y0_host = np.ascontiguousarray(w.y0[0], dtype=np.float64)
    e2e_steps = max(2, args.steps // 2)
    plan.solve_host(alpha, h, N, p_host, y0_host, Y=Yh, stream=stream)  # allocates the plan's device copy
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        plan.solve_host(alpha, h, N, p_host, y0_host, Y=Yh, sync=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.sync(stream)
    e2e_sec = e0.elapsed_time(e1) / 1e3
    e2e = {"value": e2e_steps * N * world / e2e_sec, "unit": "trajectory-steps/s",
           "h2d_bytes_per_step": int((w.params.shape[1] + d) * 8), "d2h_bytes_per_step": int((N + 1) * d * 8),
           "entry_point": "abm_solve_host"}

    out = {
        "metric": "trajectory-steps/s (plain FP64 path; history MAC/s beside)",
        "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name, "system": w.system, "alpha": alpha, "h": h, "N": N, "d": d,
                   "trajectories_per_gpu": 1, "parallelism": f"replicas{world}",
                   "l2": f"flushed between timed steps ({args.flush_mib} MiB write)",
                   "path": "abm_solve: one cooperative persistent launch per solve"},
        "history_mac_per_s": macs * args.steps * world / total_max,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get(name),
                     "kernel": "single_persistent_kernel", "flops_per_launch": 2.0 * macs,
                     "peak_source": "GB300 nominal dense FP64, 1.25 TFLOP/s (of nominal)"},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if w.system == "hindmarsh_rose" and N in PAPER_TABLE2_CUDA_S:
        out["paper_context"] = {"table2_cuda_seconds": PAPER_TABLE2_CUDA_S[N],
                                "this_run_seconds": total_max / args.steps,
                                "note": "paper's unnamed GPU, precision and parameters unstated: context only"}
    if rank == 0 and not args.no_cpu_baseline:
        n_sample = min(N, 1 << 16)  # about 10 s of oracle work on one host core
        cb, Yo = single_cpu_baseline(w, n_sample)
        out["cpu_baseline"] = cb
        # stated error of this run against the oracle, over its pointwise window
        t_win = 3.0 if w.system == "chen" else 5.0
        nwin = min(n_sample, int(round(t_win / h)))
        Yc = Y[: n_sample + 1].cpu().numpy()
        out["max_rel_err_vs_oracle"] = rel_err(Yc[: nwin + 1], Yo[: nwin + 1])
        out["error_window"] = f"t <= {t_win}"
        if n_sample > nwin + 1:
            # beyond the pointwise window (a chaotic flow decorrelates): per
            # component min, max, mean and variance against the oracle's,
            # relative to each statistic's scale
            out["statistics_beyond_window"] = {
                "window": f"t in ({t_win}, {n_sample * h:g}]",
                "max_rel_diff": stats_rel_diff(Yc[nwin + 1:], Yo[nwin + 1: n_sample + 1]),
                "measure": "max over components of |stat - stat_oracle| / max(|stat_oracle|, 1e-3 scale) for "
                           "min, max (scale: range), mean (scale: std) and variance"}
    return out


def shard_indices(M, rank, world, N=None):
    """Trajectories of one rank: round-robin over the trajectories ordered by
    N (descending), so every rank gets a similar share of the O(N^2) work."""
    import numpy as np
    order = np.argsort(-np.asarray(N), kind="stable") if N is not None else np.arange(M)
    return np.sort(order[rank::world])


def tile_schedule(w, per_tile=32):
    """Column tiles the library forms (alpha groups, N descending, 32 per tile):
    list of (n_tile, bucket, N of its trajectories)."""
    import numpy as np
    tiles = []
    for g, a in enumerate(np.unique(w.alpha)):
        idx = np.where(w.alpha == a)[0]
        Ns = np.sort(w.N[idx])[::-1]
        for q in range(0, len(Ns), per_tile):
            tiles.append((int(Ns[q]), g, Ns[q:q + per_tile]))
    return tiles


def tc_far(prec):
    """Far history on the tensor cores (BF16 split pieces)."""
    return prec in ("bf16x3", "bf16x6")


def far_shape(prec):
    """(split products, 16-bit pieces per operand, kernel name) of a tensor-core precision."""
    return {"bf16x3": (3, 2, "far_tc_kernel<3> (BF16x3)"),
            "bf16x6": (6, 3, "far_tc_kernel<6> (BF16x6)")}.get(prec, (6, 3, "far_tc_kernel<6> (BF16x6)"))


def far_work(w, nprod, npieces=None, B=64):
    """Per whole solve: algorithmic far flops (each trajectory's own targets
    n < N_i times its far rows [1, s)), raw tensor flops the MMAs execute
    (padded 128 x 96 tiles, all split products) and the operand bytes the far
    kernel streams from HBM (BF16 history pieces per active tile, Toeplitz
    pieces per active alpha group)."""
    import numpy as np
    tiles = tile_schedule(w)
    nmax = max(t[0] for t in tiles)
    npieces = npieces or (2 if nprod == 3 else 3)
    alg = raw = byts = 0.0
    for j in range((nmax + B - 1) // B):
        s = j * B
        if s <= 1:
            continue
        act = [t for t in tiles if t[0] > s]
        if not act:
            break
        for t in act:
            targets = np.clip(t[2] - s, 0, B)
            alg += 2.0 * 2 * (s - 1) * w.d * float(targets.sum())
        raw += len(act) * 2.0 * 128 * 96 * s * nprod
        byts += len(act) * s * 96 * 2 * npieces + len({t[1] for t in act}) * 128 * s * 2 * npieces
    return alg, raw, byts


def stratified(w, n):
    """n trajectories spread evenly over the N-sorted list (all of them when
    n >= M); sorted indices."""
    import numpy as np
    if n >= w.M:
        return np.arange(w.M)
    order = np.argsort(w.N, kind="stable")
    return np.sort(order[np.linspace(0, w.M - 1, n).astype(int)])


def oracle_windows(w, idx, passes=1, t_win=5.0):
    """The oracle on trajectories idx over their pointwise window t <= t_win
    (threads over the host cores): {i: Y}."""
    import concurrent.futures as cf

    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def run(i):
        n = min(int(w.N[i]), int(round(t_win / w.h[i])))
        return oracle.solve(w.system, float(w.alpha[i]), float(w.h[i]), n, w.params[i], w.y0[i], passes=passes)[0]

    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        return dict(zip([int(i) for i in idx], ex.map(run, idx)))


def arm_errors(Y, idx_local, idx_global, ref):
    """Pointwise (O8) and normwise errors of device results Y[idx_local]
    against the oracle windows ref[idx_global]."""
    import numpy as np
    Yc = Y[torch_index(idx_local)].cpu().numpy()
    errs, nerrs = [], []
    for row, g in zip(Yc, idx_global):
        r = ref[int(g)]
        errs.append(rel_err(row[: len(r)], r))
        nerrs.append(float(np.abs(row[: len(r)] - r).max() / np.abs(r).max()))
    return float(max(errs)), float(max(nerrs))


def torch_index(idx):
    import torch
    return torch.as_tensor(list(idx), dtype=torch.long, device="cuda")


def time_batched(w, prec, steps, warmup, passes, tuned, params=None, y0=None, Y=None, clocks=None,
                 sync_ranks=False):
    """Solves the batch with one plan of precision prec: warmup untimed solves,
    then `steps` timed ones (CUDA events on the launching stream around each
    solve, per-kernel events inside).  Returns a dict with the plan (open),
    per-step seconds, kernel times and the output buffer."""
    import torch

    from paper_1611_08678_gb300 import abm
    N = w.N
    ldY = int(N.max()) + 1
    plan = abm.Plan(w.system, n_max=int(N.max()), max_batch=w.M, prec=prec, profile=True,
                    corrector_passes=passes, near_warps=tuned.get("near_warps", 0),
                    far_split=tuned.get("far_split", 0), near_split=tuned.get("near_split", 0))
    params = params if params is not None else torch.as_tensor(w.params, device="cuda")
    y0 = y0 if y0 is not None else torch.as_tensor(w.y0, device="cuda")
    if Y is None:
        Y = torch.empty(w.M, ldY, w.d, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.solve_batched(w.alpha, w.h, N, params, y0, Y=Y, ldY=ldY, sync=False, stream=stream)

    for _ in range(warmup):
        step()
    plan.sync(stream)
    for k in abm.KERNEL_KINDS:
        plan.kernel_times(k, reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if sync_ranks:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    for k in range(steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if sync_ranks:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks is not None else None
    plan.sync(stream)
    times = {k: plan.kernel_times(k, reset=True) for k in abm.KERNEL_KINDS}
    per_step = [a.elapsed_time(b) / 1e3 for a, b in ev]
    return {"plan": plan, "per_step": per_step, "total": sum(per_step), "times": times, "Y": Y,
            "params": params, "y0": y0, "ldY": ldY, "clocks": clk}


def far_roofline(name, w, prec, times, steps):
    """Roofline object of the far kernel from its live per-launch times."""
    nprod, npieces, kname = far_shape(prec)
    far_n, far_ms = times["far"]
    far_sec = far_ms / 1e3 / steps  # per solve
    alg, raw, byts = far_work(w, nprod, npieces)
    if tc_far(prec):
        return {"bound": "hbm", "achieved": byts / far_sec / 1e9, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                "frac": byts / far_sec / 1e9 / HBM_PEAK_GBS,
                "traffic": (NCU_TRAFFIC_RATIO[f"{name}_{prec}"] * byts / max(1, far_n / steps)
                            if f"{name}_{prec}" in NCU_TRAFFIC_RATIO else None),
                "kernel": kname, "launches_per_solve": far_n / steps,
                "bytes_per_launch": byts / max(1, far_n / steps),
                "algorithmic_tflops": alg / far_sec / 1e12,
                "tensor_tflops_raw": raw / far_sec / 1e12, "tensor_peak_tflops": BF16_PEAK_TFLOPS,
                "tensor_frac": raw / far_sec / 1e12 / BF16_PEAK_TFLOPS,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs / bf16_tflops (of measured)"}
    if prec == "fp64":
        ach = alg / far_sec / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "batched_far_fp64_kernel",
                "launches_per_solve": far_n / steps, "flops_per_solve": alg,
                "peak_source": "GB300 nominal dense FP64, 1.25 TFLOP/s (of nominal)"}
    ach = alg / far_sec / 1e12
    return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "batched_far_fp32_kernel",
            "launches_per_solve": far_n / steps, "flops_per_solve": alg,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (of nominal)"}


def bench_batched(args, name, w, prec, world, rank, local):
    import numpy as np
    import torch

    from paper_1611_08678_gb300 import abm
    shard = w.subset(shard_indices(w.M, rank, world, w.N)) if world > 1 else w
    N = shard.N
    ldY = int(N.max()) + 1
    tuned = {"near_warps": 0, "far_split": 0, "near_split": 0}
    if args.knobs:
        fs, nw, ns = (int(v) for v in args.knobs.split(","))
        tuned = {"far_split": fs, "near_warps": nw, "near_split": ns, "cached": False, "results": []}
    elif tc_far(prec) and not args.no_tune:
        from paper_1611_08678_gb300 import autotune
        tuned = autotune.tune_batched(shard, prec)  # untimed; cached per shape
    passes = args.corrector_passes
    clocks = ClockSampler(local)
    run = time_batched(shard, prec, args.steps, max(args.warmup, 3), passes, tuned, clocks=clocks,
                       sync_ranks=world > 1)
    plan, Y, params, y0, times = run["plan"], run["Y"], run["params"], run["y0"], run["times"]
    stream = torch.cuda.current_stream()
    total = run["total"]
    t = torch.tensor([total], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_max = float(t.item())
    steps_all = float(w.N.sum()) * args.steps  # all ranks together
    value = steps_all / total_max
    macs_all = w.history_macs() * args.steps
    roof = far_roofline(name, shard, prec, times, args.steps)

    # e2e through the host-buffer entry point: inputs from pinned host memory,
    # every trajectory's rows 0..N_i back to pinned host memory, the copies
    # made by the library inside the call (copy-out overlapping later tiles)
    e2e_steps = 2
    p_host = torch.as_tensor(shard.params).pin_memory()
    y_host = torch.as_tensor(shard.y0).pin_memory()
    Yh = torch.empty(Y.shape, dtype=torch.float64, pin_memory=True)
    plan.solve_batched_host(shard.alpha, shard.h, N, p_host, y_host, Y=Yh, ldY=ldY, stream=stream)  # allocation
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        plan.solve_batched_host(shard.alpha, shard.h, N, p_host, y_host, Y=Yh, ldY=ldY, stream=stream, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.sync(stream)
    e2e_sec = e0.elapsed_time(e1) / 1e3
    e2e = {"value": float(shard.N.sum()) * e2e_steps * world / e2e_sec, "unit": "trajectory-steps/s",
           "h2d_bytes_per_step": int(p_host.numel() * 8 + y_host.numel() * 8),
           "d2h_bytes_per_step": int((shard.N + 1).sum()) * shard.d * 8,
           "entry_point": "abm_solve_batched_host"}
    del Yh

    # the same solve replayed from a captured CUDA graph (device-resident
    # inputs, no per-kernel events); the timed value above keeps the events
    # that give the roofline its kernel times
    plan.close()  # one workspace at a time
    gplan = abm.Plan(shard.system, n_max=int(N.max()), max_batch=shard.M, prec=prec, use_graph=True,
                     corrector_passes=passes, near_warps=tuned["near_warps"], far_split=tuned["far_split"],
                     near_split=tuned.get("near_split", 0))
    gsteps = max(1, min(args.steps, 3))
    for _ in range(2):  # capture, then one replay
        gplan.solve_batched(shard.alpha, shard.h, N, params, y0, Y=Y, ldY=ldY, sync=False, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(gsteps):
        gplan.solve_batched(shard.alpha, shard.h, N, params, y0, Y=Y, ldY=ldY, sync=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    gplan.sync(stream)
    g_ms = e0.elapsed_time(e1) / gsteps
    gplan.close()
    graph = {"ms_per_step": g_ms, "value": float(shard.N.sum()) * world / (g_ms / 1e3), "steps": gsteps}

    out = {
        "metric": "trajectory-steps/s and history MAC/s vs plain FP64 GPU path at stated error",
        "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"f64 state, {prec} far",
        "data": "synthetic",
        "config": {"workload": name, "system": w.system, "trajectories": int(w.M), "trajectories_per_gpu": int(shard.M),
                   "corrector_passes": passes,
                   "N_range": [int(w.N.min()), int(w.N.max())], "sum_N": int(w.N.sum()),
                   "alphas": sorted(set(float(a) for a in w.alpha)), "far_precision": prec,
                   "parallelism": f"trajectory shards x{world}",
                   "tuned": {"far_split": tuned["far_split"], "near_warps": tuned["near_warps"],
                             "near_split": tuned.get("near_split", 0), "cached": bool(tuned.get("cached", False)),
                             "timed_candidates": len(tuned.get("results", []))},
                   "l2": "inputs larger than L2 (f history of all trajectories, several GB)"},
        "history_mac_per_s": macs_all / total_max,
        "roofline": roof,
        "kernel_ms_per_solve": {k: v[1] / args.steps for k, v in times.items() if v[0]},
        # device time per solve outside every kernel of the library (launch
        # gaps between the ~2 launches per time tile), from the same events
        "launch_gaps_ms_per_solve": total / args.steps * 1e3 - sum(v[1] for v in times.values()) / args.steps,
        "e2e": e2e,
        "graph_replay": graph,
        "gpu_launches": int(sum(v[0] for v in times.values())),
        "clocks": run["clocks"],
    }
    if rank != 0 or world > 1:
        return out

    # ---- the error of this run and of the other arms against the oracle ----
    # error sample: 16 trajectories stratified by N (inside the FP64 comparator
    # subset, so every arm is compared on the same trajectories)
    sub_idx = stratified(shard, args.comparator_trajectories)
    err_idx = sub_idx[stratified(shard.subset(sub_idx), 16)]
    ref = oracle_windows(shard, err_idx, passes=passes)
    e_pt, e_nw = arm_errors(Y, err_idx, err_idx, ref)
    out["max_rel_err_vs_oracle"] = e_pt
    out["max_normwise_err_vs_oracle"] = e_nw
    out["error_window"] = f"t <= 5 on {len(err_idx)} trajectories stratified by N"
    del run, plan, Y
    torch.cuda.empty_cache()

    # ---- the plain FP64 GPU path: same library, far history in FP64 ----
    if not args.no_comparator and prec != "fp64":
        sub = shard.subset(sub_idx)
        cr = time_batched(sub, "fp64", 1, 1, passes, {})
        far_n, far_ms = cr["times"]["far"]
        near_ms = cr["times"]["near"][1]
        alg_sub = far_work(sub, 6, 3)[0]
        alg_full = far_work(shard, 6, 3)[0]
        # far history extrapolated by far-history multiply-adds (the FP64 far
        # kernel keeps the GPU's FP64 pipe busy at this subset size already);
        # the near steps taken from the full-size run above, which runs the
        # same near kernel plus the BF16 split stores (an upper bound)
        full_near_sec = out["kernel_ms_per_solve"].get("near", near_ms) / 1e3
        est_sec = far_ms / 1e3 * alg_full / alg_sub + full_near_sec
        pos = {int(g): k for k, g in enumerate(sub_idx)}
        c_pt, c_nw = arm_errors(cr["Y"], [pos[int(g)] for g in err_idx], err_idx, ref)
        comp = {"value": float(shard.N.sum()) / est_sec, "unit": "trajectory-steps/s",
                "history_mac_per_s": shard.history_macs() / est_sec, "sec_per_solve": est_sec,
                "max_rel_err_vs_oracle": c_pt, "max_normwise_err_vs_oracle": c_nw,
                "far_roofline": far_roofline(name, sub, "fp64", cr["times"], 1),
                "measured": {"trajectories": int(sub.M), "sum_N": int(sub.N.sum()), "ms_per_solve": cr["total"] * 1e3,
                             "far_ms": far_ms, "near_ms": near_ms},
                "method": f"plain FP64 path (abm_solve_batched, prec fp64) timed on {sub.M} trajectories "
                          f"stratified by N; far time scaled by far-history multiply-adds "
                          f"({alg_full / alg_sub:.1f}x) to the whole workload, near time of the full-size run "
                          "added: an extrapolation"}
        out["plain_fp64_gpu"] = comp
        out["speedup_vs_plain_fp64"] = value / comp["value"]
        cr["plan"].close()
        del cr
        torch.cuda.empty_cache()

    # ---- further precision arms on the full workload ----
    arms = {}
    for arm in [a for a in (args.arms or "").split(",") if a and a != prec]:
        if arm == "fp64":
            continue  # the comparator above
        ar = time_batched(shard, arm, 2, 1, passes, tuned if tc_far(arm) else {})
        a_pt, a_nw = arm_errors(ar["Y"], err_idx, err_idx, ref)
        arms[arm] = {"value": float(shard.N.sum()) * 2 / ar["total"], "unit": "trajectory-steps/s",
                     "ms_per_solve": ar["total"] / 2 * 1e3, "max_rel_err_vs_oracle": a_pt,
                     "max_normwise_err_vs_oracle": a_nw,
                     "kernel_ms_per_solve": {k: v[1] / 2 for k, v in ar["times"].items() if v[0]},
                     "roofline": far_roofline(name, shard, arm, ar["times"], 2)}
        ar["plan"].close()
        del ar
        torch.cuda.empty_cache()
    if arms:
        out["arms"] = arms
    if not args.no_cpu_baseline:
        out.update(batched_cpu_baseline(w, passes=passes))
    return out


def batched_cpu_baseline(w, n_sub=16, passes=1):
    """Oracle on a seeded subset (stratified by N), threads over the host
    cores; scaled by history MACs to the whole workload."""
    import concurrent.futures as cf

    import oracle
    pick = stratified(w, n_sub)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def run(i):
        return oracle.solve(w.system, float(w.alpha[i]), float(w.h[i]), int(w.N[i]), w.params[i], w.y0[i],
                            passes=passes)[0]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(run, pick))
    sec = time.perf_counter() - t0
    sub = w.subset(pick)
    mac_rate = sub.history_macs() / sec
    value = mac_rate * float(w.N.sum()) / w.history_macs()
    return {"cpu_baseline": {"value": value, "unit": "trajectory-steps/s", "cores": int(cores), "kind": "oracle",
                             "sample": f"{len(pick)} whole trajectories stratified by N ({int(sub.N.sum())} steps, "
                                       f"{sec:.1f} s on {cores} threads), scaled by history MACs to the workload",
                             "history_mac_per_s": mac_rate}}


def bench_adjoint(args, name, prec, world, rank, local):
    """Forward solve + loss partials + adjoint (dL/dparams, dL/dy0) per step:
    1024 fractional Lorenz trajectories, N = 2^14, loss = mean squared distance
    to the trajectories of perturbed parameters."""
    import numpy as np
    import torch

    from paper_1611_08678_gb300 import abm, workloads
    w_all, tparams_all = workloads.lorenz_adjoint()
    idx = shard_indices(w_all.M, rank, world, w_all.N) if world > 1 else np.arange(w_all.M)
    w, tparams = w_all.subset(idx), tparams_all[idx]
    N, M, d = int(w.N.max()), w.M, w.d
    # launch shapes: pinned by --knobs, else tuned on the forward solve (the
    # adjoint's far and near launches take the same plan options)
    tuned = {"far_split": 0, "near_warps": 0, "near_split": 0}
    if args.knobs:
        tuned = dict(zip(("far_split", "near_warps", "near_split"), (int(v) for v in args.knobs.split(","))))
    elif tc_far(prec) and not args.no_tune:
        from paper_1611_08678_gb300 import autotune
        tuned = autotune.tune_batched(w, prec)  # untimed; cached per shape
    plan = abm.Plan("lorenz", n_max=N, max_batch=M, prec=prec, profile=True, far_split=tuned["far_split"],
                    near_warps=tuned["near_warps"], near_split=tuned["near_split"])
    params = torch.as_tensor(w.params, device="cuda")
    y0 = torch.as_tensor(w.y0, device="cuda")
    Y = torch.zeros(M, N + 1, d, dtype=torch.float64, device="cuda")
    YP = torch.zeros_like(Y)
    Yt = plan.solve_batched(w.alpha, w.h, w.N, torch.as_tensor(tparams, device="cuda"), y0)  # targets
    scale = 2.0 / ((N + 1) * d)
    stream = torch.cuda.current_stream()

    def step():
        plan.solve_batched(w.alpha, w.h, w.N, params, y0, Y=Y, YP=YP, sync=False, stream=stream)
        G = (Y - Yt) * scale
        return plan.adjoint(w.alpha, w.h, w.N, params, y0, Y, YP, G, sync=False, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    plan.sync(stream)
    for k in abm.KERNEL_KINDS:
        plan.kernel_times(k, reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        ev[k][0].record(stream)
        dp, dy0 = step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    plan.sync(stream)
    times = {k: plan.kernel_times(k, reset=True) for k in abm.KERNEL_KINDS}
    total = sum(a.elapsed_time(b) / 1e3 for a, b in ev)
    t = torch.tensor([total], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    total_max = float(t.item())
    value = float(w_all.N.sum()) * args.steps / total_max
    nprod, npieces, kname = far_shape(prec)
    far_n, far_ms = times["far"]
    alg, raw, byts = far_work(w, nprod, npieces)
    far_sec = far_ms / 1e3 / args.steps
    out = {
        "metric": "trajectory-steps/s of forward + adjoint (history MAC/s beside; gradient error vs oracle stated)",
        "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"f64 state, {prec} far", "data": "synthetic",
        "config": {"workload": name, "system": "lorenz", "trajectories": int(w_all.M), "N": N,
                   "far_precision": prec, "parallelism": f"trajectory shards x{world}",
                   "tuned": {k: int(tuned[k]) for k in ("far_split", "near_warps", "near_split")},
                   "l2": "inputs larger than L2 (histories of 1024 trajectories, several GB)"},
        "history_mac_per_s": 2 * w_all.history_macs() * args.steps / total_max,
        "roofline": {"bound": "hbm", "achieved": byts / far_sec / 1e9, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                     "frac": byts / far_sec / 1e9 / HBM_PEAK_GBS, "traffic": None,
                     "kernel": f"{kname} (forward launches)",
                     "tensor_tflops_raw": raw / far_sec / 1e12, "tensor_frac": raw / far_sec / 1e12 / BF16_PEAK_TFLOPS},
        "kernel_ms_per_solve": {k: v[1] / args.steps for k, v in times.items() if v[0]},
        "gpu_launches": int(sum(v[0] for v in times.values())),
        "clocks": clk,
    }
    # e2e: inputs from pinned host memory, gradients back to the host
    p_host = torch.as_tensor(w.params).pin_memory()
    y_host = torch.as_tensor(w.y0).pin_memory()
    dp_h = torch.empty(M, 3, dtype=torch.float64, pin_memory=True)
    dy_h = torch.empty(M, d, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(2):
        params.copy_(p_host, non_blocking=True)
        y0.copy_(y_host, non_blocking=True)
        dp, dy0 = step()
        dp_h.copy_(dp, non_blocking=True)
        dy_h.copy_(dy0, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    out["e2e"] = {"value": float(w.N.sum()) * 2 * world / (e0.elapsed_time(e1) / 1e3), "unit": "trajectory-steps/s",
                  "h2d_bytes_per_step": int((p_host.numel() + y_host.numel()) * 8),
                  "d2h_bytes_per_step": int((dp_h.numel() + dy_h.numel()) * 8)}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        Yn, Ytn = Y.cpu().numpy(), Yt.cpu().numpy()
        dpn, dyn = dp.cpu().numpy(), dy0.cpu().numpy()
        errs, t0 = [], time.perf_counter()
        for i in (0, M - 1):
            Gi = (Yn[i] - Ytn[i]) * scale
            op, oy = oracle.tangent("lorenz", float(w.alpha[i]), float(w.h[i]), N, w.params[i], w.y0[i], Gi)
            errs.append(max(np.max(np.abs(dpn[i] - op)) / np.max(np.abs(op)),
                            np.max(np.abs(dyn[i] - oy)) / np.max(np.abs(oy))))
        sec = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 2 * N / sec, "unit": "trajectory-steps/s", "cores": 1, "kind": "oracle",
                               "sample": f"tangent-linear gradient of 2 trajectories ({sec:.1f} s, 1 host thread)"}
        out["max_rel_err_vs_oracle"] = float(max(errs))
        out["error_window"] = "gradients dL/dparams, dL/dy0 of 2 trajectories vs the oracle tangent-linear gradient"
    return out


def bench_reference(args, name, w, world, rank):
    """The oracle, as it stands, on the host cores: each step a bounded sample."""
    if rank != 0:
        return None
    if name == "lorenz_adjoint":
        return {"impl": "reference", "unavailable": "the reference arm times forward solves; the adjoint "
                                                    "workload's oracle gradient is timed in cpu_baseline"}
    if not is_single(name):
        return bench_reference_batched(args, name, w, world)
    N, d = int(w.N[0]), w.d
    n_sample = min(N, 1 << 14)
    rates = []
    for k in range(args.warmup + args.steps):
        sec, _ = oracle_single_rate(w, n_sample)
        if k >= args.warmup:
            rates.append(n_sample * (n_sample + 1) * d / sec)
    mac_rate = statistics.mean(rates)
    value = mac_rate / ((N + 1) * d)
    return {"impl": "reference", "metric": "trajectory-steps/s (plain FP64 path; history MAC/s beside)",
            "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": n_sample * (n_sample + 1) * d / mac_rate * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": name, "system": w.system, "N": N, "d": d},
            "history_mac_per_s": mac_rate,
            "cpu_baseline": {"value": value, "unit": "trajectory-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {n_sample} steps per step, 1 host thread, scaled by history "
                                       f"MACs to the {N}-step solve"},
            "e2e": {"value": value, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def bench_reference_batched(args, name, w, world, n_traj=16, n_prefix=1 << 14):
    """The oracle on a batched workload: each step solves the first n_prefix
    steps of n_traj trajectories stratified by N (threads over the host
    cores); the history-MAC rate is scaled to the whole workload."""
    import concurrent.futures as cf

    import oracle
    pick = stratified(w, n_traj)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    lens = {int(i): min(int(w.N[i]), n_prefix) for i in pick}
    macs = float(sum(n * (n + 1) for n in lens.values()) * w.d)

    def run(i):
        oracle.solve(w.system, float(w.alpha[i]), float(w.h[i]), lens[int(i)], w.params[i], w.y0[i],
                     passes=args.corrector_passes)

    rates, secs = [], []
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            list(ex.map(run, pick))
            sec = time.perf_counter() - t0
            if k >= args.warmup:
                rates.append(macs / sec)
                secs.append(sec)
    mac_rate = statistics.mean(rates)
    value = mac_rate * float(w.N.sum()) / w.history_macs()
    sample = (f"first {n_prefix} steps of {len(pick)} trajectories stratified by N per step, {cores} host threads, "
              f"scaled by history MACs to the whole workload")
    return {"impl": "reference", "metric": "trajectory-steps/s and history MAC/s vs plain FP64 GPU path at stated error",
            "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "system": w.system, "trajectories": int(w.M),
                       "N_range": [int(w.N.min()), int(w.N.max())], "sum_N": int(w.N.sum())},
            "history_mac_per_s": mac_rate,
            "cpu_baseline": {"value": value, "unit": "trajectory-steps/s", "cores": int(cores), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    args = parse_args(argv)
    world, rank, local = dist_env()
    w, default_prec = workload(args.workload, args.n)
    prec = args.prec or default_prec
    if args.trajectories and not is_single(args.workload) and args.workload != "lorenz_adjoint":
        import numpy as np
        w = w.subset(np.arange(min(args.trajectories, w.M)))
    if args.impl == "reference":
        out = bench_reference(args, args.workload, w, world, rank)
        if out is not None:
            print(json.dumps(out))
        return 0
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl")
    if is_single(args.workload):
        out = bench_single(args, args.workload, w, world, rank, local)
    elif args.workload == "lorenz_adjoint":
        out = bench_adjoint(args, args.workload, prec, world, rank, local)
    else:
        out = bench_batched(args, args.workload, w, prec, world, rank, local)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
