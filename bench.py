#!/usr/bin/env python
"""Benchmark of the fractional ABM history convolution on GB300.

Default workload: the fractional Chen system as one long trajectory
(a=35, b=3, c=28, alpha=0.9, y0=(-9,-5,14), h=0.001, N=2^18, d=3), plain FP64
path (abm_solve: one cooperative persistent launch per solve).  One "step" =
one whole solve.  Metric: trajectory-steps/s (history MAC/s reported beside).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chen_single|lorenz_single|rossler_batched|financial_batched]

Multi-GPU (torchrun, one rank per GPU): single-trajectory workloads run one
replica per rank (the path does not shard); batched workloads shard the
trajectories across ranks.  Both are weak scaling with no data-path
collective; the timing is the max over ranks.

The oracle (plain FP64 CPU implementation under oracle/) is executed here only
for the cpu_baseline leg and for --impl reference.
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

# Nominal FP64 rate of GB300 (profiling recipe: 1.25 TFLOP/s) - the peak of
# the ALU-bound FP64 path.  The measured HBM / bf16 peaks are read from
# MEASURED_PEAKS.json for the HBM/tensor-bound kernels.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flop x max clock


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0  # profiling recipe fallback


HBM_PEAK_GBS, BF16_PEAK_TFLOPS = _measured_peaks()

# DRAM bytes per launch of the dominant kernel from one ncu capture (see
# profiles/); None when the kernel changed since the counters were taken.
NCU_TRAFFIC = {
    "chen_single": 6780160 + 96000,  # profiles/single_persistent_kernel_chen_N262144.md
}
# Batched far kernel: DRAM bytes (read + write) of one captured launch over the
# algorithmic operand bytes of that launch, per workload and precision, from
# an ncu capture of the current kernel (profiles/far_tc_kernel_rossler_batched.md,
# profiles/far_tc_kernel_financial_batched.md: 512-trajectory cases); the bench
# line scales it to its own average launch, since DRAM bytes grow with the
# operand bytes.
NCU_TRAFFIC_RATIO = {
    "rossler_batched_bf16x6": (414428928 + 3322880) / 413564928,
    "financial_batched_bf16x6": (385732352 + 3349248) / 384024576,
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="chen_single",
                    choices=["chen_single", "lorenz_single", "hindmarsh_rose_single", "rossler_batched",
                             "financial_batched", "lorenz_adjoint"])
    ap.add_argument("--n", type=int, default=0, help="single-trajectory workloads: number of steps N")
    ap.add_argument("--prec", default=None, help="far-history precision of batched workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mib", type=int, default=256)
    ap.add_argument("--no-tune", action="store_true", help="batched: skip the autotuner (library defaults)")
    ap.add_argument("--corrector-passes", type=int, default=1,
                    help="batched: corrector passes per step (1 = PECE, m > 1 = P(EC)^m E)")
    ap.add_argument("--trajectories", type=int, default=0,
                    help="batched workloads: first M trajectories only (small cases for profiling)")
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

    # e2e: the public call with host buffers: params / y0 from pinned host
    # memory (by value through the ABI), the solution copied back to pinned
    # host memory, every step.
    Yh = torch.empty(N + 1, d, dtype=torch.float64, pin_memory=True)
    p_host = torch.tensor(w.params[0], dtype=torch.float64).pin_memory()
    y0_host = torch.tensor(w.y0[0], dtype=torch.float64).pin_memory()
    e2e_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        plan.solve(alpha, h, N, p_host.numpy(), y0_host.numpy(), Y=Y, sync=False, stream=stream)
        Yh.copy_(Y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.sync(stream)
    e2e_sec = e0.elapsed_time(e1) / 1e3
    e2e = {"value": e2e_steps * N * world / e2e_sec, "unit": "trajectory-steps/s",
           "h2d_bytes_per_step": int((w.params.shape[1] + d) * 8), "d2h_bytes_per_step": int((N + 1) * d * 8)}

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
                     "peak_source": "FP64 nominal 1.25 TFLOP/s (profiling recipe)"},
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
        out["max_rel_err_vs_oracle"] = rel_err(Y[: nwin + 1].cpu().numpy(), Yo[: nwin + 1])
        out["error_window"] = f"t <= {t_win}"
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


def bench_batched(args, name, w, prec, world, rank, local):
    import numpy as np
    import torch

    from paper_1611_08678_gb300 import abm
    shard = w.subset(shard_indices(w.M, rank, world, w.N)) if world > 1 else w
    N = shard.N
    ldY = int(N.max()) + 1
    tuned = {"near_warps": 0, "far_split": 0}
    if tc_far(prec) and not args.no_tune:
        from paper_1611_08678_gb300 import autotune
        tuned = autotune.tune_batched(shard, prec)  # untimed; cached per shape
    plan = abm.Plan(shard.system, n_max=int(N.max()), max_batch=shard.M, prec=prec, profile=True,
                    corrector_passes=args.corrector_passes,
                    near_warps=tuned["near_warps"], far_split=tuned["far_split"])
    params = torch.as_tensor(shard.params, device="cuda")
    y0 = torch.as_tensor(shard.y0, device="cuda")
    Y = torch.empty(shard.M, ldY, shard.d, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.solve_batched(shard.alpha, shard.h, N, params, y0, Y=Y, ldY=ldY, sync=False, stream=stream)

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
        step()
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
    steps_all = float(w.N.sum()) * args.steps  # all ranks together
    value = steps_all / total_max
    macs_all = w.history_macs() * args.steps

    nprod, npieces, kname = far_shape(prec)
    far_n, far_ms = times["far"]
    near_n, near_ms = times["near"]
    if tc_far(prec):
        alg, raw, byts = far_work(shard, nprod, npieces)
        far_sec = far_ms / 1e3 / args.steps  # per solve
        roof = {"bound": "hbm", "achieved": byts / far_sec / 1e9, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                "frac": byts / far_sec / 1e9 / HBM_PEAK_GBS,
                "traffic": (NCU_TRAFFIC_RATIO[f"{name}_{prec}"] * byts / max(1, far_n / args.steps)
                            if f"{name}_{prec}" in NCU_TRAFFIC_RATIO else None),
                "kernel": kname, "launches_per_solve": far_n / args.steps,
                "bytes_per_launch": byts / max(1, far_n / args.steps),
                "algorithmic_tflops": alg / far_sec / 1e12,
                "tensor_tflops_raw": raw / far_sec / 1e12, "tensor_peak_tflops": BF16_PEAK_TFLOPS,
                "tensor_frac": raw / far_sec / 1e12 / BF16_PEAK_TFLOPS,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs / bf16_tflops (of measured)"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None,
                "kernel": "batched far (SIMT)"}

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

    # the same solve replayed from a captured CUDA graph (device-resident
    # inputs, no per-kernel events); the timed value above keeps the events
    # that give the roofline its kernel times
    plan.close()  # one workspace at a time
    gplan = abm.Plan(shard.system, n_max=int(N.max()), max_batch=shard.M, prec=prec, use_graph=True,
                     corrector_passes=args.corrector_passes,
                     near_warps=tuned["near_warps"], far_split=tuned["far_split"])
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
        "metric": "trajectory-steps/s (history MAC/s beside; error vs FP64 oracle stated)",
        "value": value, "unit": "trajectory-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": f"f64 state, {prec} far",
        "data": "synthetic",
        "config": {"workload": name, "system": w.system, "trajectories": int(w.M), "trajectories_per_gpu": int(shard.M),
                   "corrector_passes": args.corrector_passes,
                   "N_range": [int(w.N.min()), int(w.N.max())], "sum_N": int(w.N.sum()),
                   "alphas": sorted(set(float(a) for a in w.alpha)), "far_precision": prec,
                   "parallelism": f"trajectory shards x{world}",
                   "tuned": {"near_warps": tuned["near_warps"], "far_split": tuned["far_split"],
                             "cached": bool(tuned.get("cached", False))},
                   "l2": "inputs larger than L2 (f history of all trajectories, several GB)"},
        "history_mac_per_s": macs_all / total_max,
        "roofline": roof,
        "kernel_ms_per_solve": {k: v[1] / args.steps for k, v in times.items() if v[0]},
        "e2e": e2e,
        "graph_replay": graph,
        "gpu_launches": int(sum(v[0] for v in times.values())),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out.update(batched_cpu_baseline(w, Y if world == 1 else None, passes=args.corrector_passes))
    return out


def batched_cpu_baseline(w, Y=None, n_sub=16, passes=1):
    """Oracle on a seeded subset (stratified by N), threads over the host
    cores; scaled by history MACs to the whole workload.  With Y (this run's
    GPU result, single rank) also the stated error over t <= 5."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    order = np.argsort(w.N)
    pick = order[np.linspace(0, w.M - 1, n_sub).astype(int)]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def run(i):
        return oracle.solve(w.system, float(w.alpha[i]), float(w.h[i]), int(w.N[i]), w.params[i], w.y0[i],
                            passes=passes)[0]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(run, pick))
    sec = time.perf_counter() - t0
    sub = w.subset(pick)
    mac_rate = sub.history_macs() / sec
    value = mac_rate * float(w.N.sum()) / w.history_macs()
    out = {"cpu_baseline": {"value": value, "unit": "trajectory-steps/s", "cores": int(cores), "kind": "oracle",
                            "sample": f"{n_sub} trajectories stratified by N ({int(sub.N.sum())} steps, "
                                      f"{sec:.1f} s on {cores} threads), scaled by history MACs to the workload",
                            "history_mac_per_s": mac_rate}}
    if Y is not None:
        # pointwise (the 1e-11 measure), normwise per trajectory, and, as the
        # scale of the flow's own conditioning, the oracle's divergence from
        # itself when y0 is perturbed at the FP32 rounding level (2^-24)
        errs, nerrs, cond = [], [], []
        Yc = Y.cpu().numpy()
        for i, ref in zip(pick, res):
            n = min(int(w.N[i]), int(round(5.0 / w.h[i])))
            errs.append(rel_err(Yc[i, : n + 1], ref[: n + 1]))
            nerrs.append(float(np.abs(Yc[i, : n + 1] - ref[: n + 1]).max() / np.abs(ref[: n + 1]).max()))
            y0p = np.asarray(w.y0[i], float) * (1.0 + 2.0 ** -24)
            refp = oracle.solve(w.system, float(w.alpha[i]), float(w.h[i]), n, w.params[i], y0p, passes=passes)[0]
            cond.append(rel_err(refp, ref[: n + 1]))
        out["max_rel_err_vs_oracle"] = float(max(errs))
        out["max_normwise_err_vs_oracle"] = float(max(nerrs))
        out["oracle_self_divergence_y0_2^-24"] = float(max(cond))
        out["error_window"] = f"t <= 5 on the {n_sub} oracle trajectories"
    return out


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
    plan = abm.Plan("lorenz", n_max=N, max_batch=M, prec=prec, profile=True)
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
    if not is_single(name):
        return {"impl": "reference", "unavailable": "reference arm implemented for single-trajectory workloads"}
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
