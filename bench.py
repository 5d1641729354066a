#!/usr/bin/env python
"""Benchmark: population updates per second of the fused RLBM step on GB300.

Default workload (one benchmark step): the 2D Riemann problem on a 2048 x 2048
grid (copy-out walls), quadrature N = 2 (3 radial Gauss-Laguerre nodes) x
K = 48 angles = 144 populations per site, Kn = 0.05 (tau = 102.4), 2000 time
steps: 1.21e12 population updates.  Populations are stored in FP16 relative to
the rest equilibrium (s = f / f_rest, stochastic rounding), accumulated in
FP32, with the Landau frame solved in double-float.  The 2.4 GB of
populations are far above the 129 MB L2, so the step kernel streams from HBM.
Inputs are synthetic: four quadrant states (n, T) = (1, 1), (0.5, 0.8),
(0.25, 0.6), (0.5, 0.8), u = 0, each jittered by 1 % from the seed.

The scaled 1D shock tube (8192 x 4, N = 3 x K = 64, four Kn, 4000 steps, FP32)
is `--workload shock1d_8192x4_N3K64`; its 67 MB working set stays in the L2,
and its line says so ("bound": "l2").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision fp32|fp64|fp16|bf16] [--impl ours|reference]

One JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle (the
method's plain definition) on the host cores on a bounded sample of the same
workload.  Under torchrun each rank runs its own replica of the problem set
(independent problems, no collective on the data path), weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2011_06856_gb300 import workloads as W  # noqa: E402

FALLBACK_HBM_GBS = 6800.0
METRIC = "population-updates/s"
L2_BYTES = 129e6


def kn_json(kn_list):
    """Kn values for the JSON line (tau -> inf, free streaming, as the string "inf")."""
    return [k if math.isfinite(k) else "inf" for k in kn_list]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="riemann2d_2048_N2K48",
                    choices=sorted(W.WORKLOADS) + ["batch256", "closure4096", "closure4096_4000steps"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp16", "bf16", "fp16n", "bf16n"])
    ap.add_argument("--timesteps", type=int, default=None,
                    help="override time steps per problem (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default=None, choices=["per-tile", "tma", "pair", "pair-bulk", "pair-tma"],
                    help="pin the step kernel (with --tile-p) instead of autotuning; for profiling runs")
    ap.add_argument("--tile-p", type=int, default=None, help="populations per warp with --kernel")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over the ranks of the job (the job takes as long as its
    slowest rank); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, max_total_ms: float) -> float:
    """Whole-job rate: the units every rank processed in the timed steps over
    the slowest rank's time (weak scaling: every rank has the same work)."""
    return units_per_rank_step * steps * world / (max_total_ms * 1e-3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as fh:
                d = json.load(fh)
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("rlbm_device.cuh", "rlbm_launch.cuh", "rlbm_args.h", "rlbm_pair.cuh", "rlbm_df64.cuh",
              "rlbm_pair_tma.cuh", "rlbm_tma.cuh"):
        with open(os.path.join(ROOT, "paper_2011_06856_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, precision: str, kernel: str, tile_p: int):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the summary is missing, covers another kernel or tiling, or
    the kernel sources changed since."""
    path = os.path.join(ROOT, "profiles", f"rlbm_step_{workload}_{precision}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    k = re.search(r"step_kernel:\s*(\S+)\s+P=(\d+)", text)
    if not m or not s or s.group(1) != kernel_source_hash():
        return None
    if not k or k.group(1) != kernel or int(k.group(2)) != tile_p:
        return None
    return float(m.group(1))


def fp64_roof(dev):
    """The FP64 rate of this GPU, measured here: a cuBLAS DGEMM (torch.matmul of
    two 4096 x 4096 FP64 matrices, best of 5, CUDA events).  MEASURED_PEAKS.json
    carries no FP64 figure."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12, "measured here: cuBLAS DGEMM 4096^3, best of 5"


def fp64_flops_per_update(N: int, two_d: bool, npop: int) -> float:
    """FP64 FLOPs (FMA = 2) the method needs per population update in FP64:
    streaming 9 (2D) or 3 (1D), angular sums 9, equilibrium 1 + 4N, omega 4,
    relaxation 3; plus about 500 per site for the per-site part (moment fold,
    Landau frame, equilibrium coefficients), counted once per site and shared
    by its npop populations (the per-tile kernel repeats it in every warp:
    that repetition is not the method's work and is not counted)."""
    return (9 if two_d else 3) + 9 + (1 + 4 * N) + 4 + 3 + 500.0 / npop


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_statistics(w: W.Workload, kn_list, budget_s: float = 12.0):
    """The quantum-statistics oracle (Python, one site at a time) on a bounded
    sample: a strip of 8 sites of the workload's first row, time steps until the
    budget is spent."""
    import oracle as O
    from oracle import statistics as S
    kind, g = W.statistics(w)
    eps = {"fd": S.FD, "be": S.BE}[kind]
    q = O.Quadrature(w.N, w.K)
    fl = W.workload_fields(w)
    sl = (slice(0, 1), slice(0, 8))
    f = S.init(q, fl.n[sl], fl.T[sl], fl.bx[sl], fl.by[sl], eps, g)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        f = S.run(q, f, W.tau_from_kn(kn_list[steps % len(kn_list)], w.nx), 1, w.bcx, w.bcy, eps, g)
        steps += 1
    dt = time.perf_counter() - t0
    updates = 8 * w.npop * steps
    return {"value": updates / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"8 sites of {w.nx}x{w.ny} N={w.N} K={w.K}, {kind} statistic, {steps} time steps "
                      f"({updates:.3e} updates, {dt:.1f} s, FP64, Python per site)"}


def cpu_baseline(w: W.Workload, kn_list, budget_s: float = 12.0):
    """Time the FP64 oracle (as it stands) on the host cores on a bounded sample:
    the full grid and quadrature of the workload, a few time steps per Kn."""
    if W.statistics(w)[0] != "mj":
        return cpu_baseline_statistics(w, kn_list, budget_s)
    import oracle as O
    q = O.Quadrature(w.N, w.K, onlattice=bool(w.extra.get("onlattice")))
    fl = W.workload_fields(w)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    # calibrate with one step, then fill the budget
    t0 = time.perf_counter()
    q.run(f0, W.tau_from_kn(kn_list[0], w.nx, W.light_speed(w)), 1, w.bcx, w.bcy)
    t1 = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(t1, 1e-6) / len(kn_list)))
    t0 = time.perf_counter()
    for kn in kn_list:
        q.run(f0, W.tau_from_kn(kn, w.nx, W.light_speed(w)), steps, w.bcx, w.bcy)
    dt = time.perf_counter() - t0
    updates = w.sites * w.npop * steps * len(kn_list)
    return {"value": updates / dt, "unit": METRIC, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{w.nx}x{w.ny} N={w.N} K={w.K}, {steps} time steps x {len(kn_list)} Kn "
                      f"({updates:.3e} updates, {dt:.1f} s, FP64)"}


def run_reference(args, w: W.Workload, precision: str):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    kn_list = list(w.kn)
    cb = cpu_baseline(w, kn_list, budget_s=8.0)
    if W.statistics(w)[0] != "mj":  # the Python statistics oracle: the baseline's sample is the timed work
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC,
                "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": w.name, "grid": [w.nx, w.ny], "N": w.N, "K": w.K, "npop": w.npop,
                           "kn": kn_json(kn_list), "precision": "fp64", "device": "host (oracle)"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    # timed steps: each a bounded sample of the workload
    import oracle as O
    q = O.Quadrature(w.N, w.K, onlattice=bool(w.extra.get("onlattice")))
    fl = W.workload_fields(w)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    t0 = time.perf_counter()
    q.run(f0, W.tau_from_kn(kn_list[0], w.nx, W.light_speed(w)), 1, w.bcx, w.bcy)
    per = time.perf_counter() - t0
    steps_per = max(1, int(6.0 / max(per, 1e-6) / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        q.run(f0, W.tau_from_kn(kn_list[0], w.nx, W.light_speed(w)), steps_per, w.bcx, w.bcy)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        q.run(f0, W.tau_from_kn(kn_list[s % len(kn_list)], w.nx, W.light_speed(w)), steps_per, w.bcx, w.bcy)
        times.append(time.perf_counter() - t0)
    upd = w.sites * w.npop * steps_per
    value = upd * len(times) / sum(times)
    cb["value"] = value
    cb["sample"] = f"{w.nx}x{w.ny} N={w.N} K={w.K}, {steps_per} time steps per timed step, FP64"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": [w.nx, w.ny], "N": w.N, "K": w.K,
                       "npop": w.npop, "kn": kn_json(kn_list), "time_steps_per_problem": steps_per,
                       "precision": "fp64", "device": "host cores (oracle)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """256 uneven independent problems (N = 2, FP32), all advanced `--timesteps`
    time steps (default 100; the full problem set runs 1000) per benchmark step,
    in the execution mode the batch autotuner picks (one persistent cooperative
    launch, or every problem's own step kernel on a pool of streams)."""
    import torch
    from paper_2011_06856_gb300 import build as B
    from paper_2011_06856_gb300 import rlbm as R
    B.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    probs = W.batch_problems(256)
    specs = [(p.nx, p.ny, p.bcx, p.bcy, p.K, W.tau_from_kn(p.kn, p.nx)) for p in probs]
    stream = torch.cuda.Stream()
    b = R.Batch(specs, N=2, precision="fp32", stream=stream)
    best = b.autotune(2)
    for p, pb in zip(b.problems, probs):
        fl = W.shock_tube(pb.nx, pb.ny, pb.left, pb.right)
        p.init_fields(fl)
    steps = args.timesteps or 100
    upd = b.population_updates_per_step * steps
    alg_bytes = 2 * 4 * b.population_updates_per_step
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            b.step(steps)
        b.sync()
        clk = ClockSampler(local)
        clk.start()
        ms = []
        l0 = b.kernel_launches
        for _ in range(args.steps):
            flush.random_(0, 255)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        b.sync()
        clocks = clk.stop()
        launches = b.kernel_launches - l0
        # the other execution mode, timed once after the measurement (outside the timed
        # region): one persistent launch against the stream pool
        mode_used = b.mode
        other = "persistent" if mode_used == "streams" else "streams"
        b.set_mode(other)
        b.step(steps)
        b.sync()
        flush.random_(0, 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        e1.synchronize()
        other_ms = e0.elapsed_time(e1) / steps
        b.set_mode(mode_used)
    total = max_over_ranks(float(np.sum(ms)), world, torch.device("cuda", local))
    value = job_throughput(upd, args.steps, world, total)
    peak, src = measured_peaks()
    achieved = alg_bytes * steps * args.steps / (total * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch256", "problems": len(probs), "N": 2,
                       "time_steps_per_bench_step": steps,
                       "footprint_GB": sum(2 * 4 * nx * ny * K * 3 for (nx, ny, _, _, K, _) in specs) / 1e9,
                       "l2": "flushed between timed steps; working set far above L2",
                       "autotuned_ms_per_time_step": best, "batch_mode": mode_used,
                       "other_mode": {"mode": other, "ms_per_time_step": other_ms},
                       "ms_per_time_step": total / args.steps / steps},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": src, "traffic": None,
                         "kernel": "rlbm_batch_kernel" if mode_used == "persistent"
                         else "per-problem step kernels (rlbm_pair_kernel / rlbm_kernel)"},
            "cpu_baseline": None,
            "e2e": None, "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        dist.destroy_process_group()


def run_closure(args):
    """Learned closure at the deployment size: time per step of the fine plain run
    (K = 128), the coarse plain run (K = 24) and the coarse run with the fused
    correction, on a 4096^2 Riemann problem (FP32), after a training on
    128^2 runs of the method.  Reports corrected-coarse population updates/s."""
    import torch
    from paper_2011_06856_gb300 import build as B
    from paper_2011_06856_gb300 import closure as CL
    from paper_2011_06856_gb300 import rlbm as R
    B.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:  # replicas: every rank runs the whole workload
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = 4096
    cl = R.Closure(2, 24, seed=7)
    X, T = CL.generate(cl, 128, 128, kns=(0.02, 0.1, 0.5, 2.0), steps=32, every=2)
    CL.train(cl, X, T, iters=4000, batch=16384, lr=2e-3, decay=True)
    del X, T
    fl = W.riemann_2d(n, n, CL.RIEMANN, jitter=0.01)
    kn = 0.3
    feat = CL.kn_feature(W.tau_from_kn(kn, n), 128)  # trained on 128^2 runs
    times = {}
    for name, K, corrected in (("fine_K128", 128, False), ("coarse_K24", 24, False),
                               ("coarse_K24_closure", 24, True)):
        sim = R.Simulation(n, n, 2, K, W.tau_from_kn(kn, n), "fp32", W.BC_COPYOUT, W.BC_COPYOUT,
                           stream=cl.stream)
        sim.init_fields(fl)
        sim.autotune(4)
        nst = 20

        def run(k):
            for _ in range(k):
                sim.step(1)
                if corrected:
                    cl.apply(sim, feat)
        run(3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cl.stream)
        run(nst)
        e1.record(cl.stream)
        e1.synchronize()
        times[name] = e0.elapsed_time(e1) / nst
        sim.close()
    # accuracy at the training size: a Riemann problem not in the training set
    acc = {}
    for kn_e in (0.3, 1.0):
        mf, mc, ml = CL.deploy(cl, 128, 128, kn_e, 64)
        acc[f"kn{kn_e}"] = {"plain_coarse_rel_l2_n_eps": [CL.rel_l2(mc[i], mf[i]) for i in (0, 1)],
                            "corrected_rel_l2_n_eps": [CL.rel_l2(ml[i], mf[i]) for i in (0, 1)]}
    upd = n * n * 72
    t_corr = max_over_ranks(times["coarse_K24_closure"], world, torch.device("cuda", local))
    value = job_throughput(upd, 1, world, t_corr)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": 20, "warmup": 3,
            "ms_per_step": times["coarse_K24_closure"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (bf16 network weights)", "data": "synthetic",
            "config": {"workload": "closure4096", "grid": [n, n], "N": 2, "K_coarse": 24,
                       "K_fine": 128, "kn": kn, "ms_per_time_step": times,
                       "fine_over_corrected_time": times["fine_K128"] / times["coarse_K24_closure"],
                       "accuracy_vs_fine_128sq_64_steps": acc,
                       "training": "tensor-core kernels, 4000 Adam steps of 16384 columns from 128^2 runs "
                                   "at Kn 0.02, 0.1, 0.5, 2 (32 steps each)"},
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Training runs of the config-5 closure: 1024^2 Riemann problems at four Kn,
# snapshots every `every` steps over `steps` steps (1024 steps of a 1024^2
# grid span the physical time of the 4000 deployed steps at 4096^2).
CLOSURE_LONG_TRAIN = {"grid": 1024, "kn": (0.01, 0.1, 1.0, 5.0), "steps": 1024, "every": 64}


def run_closure_long(args):
    """The learned closure trained on 1024^2 runs and deployed on 4096^2 for 4000 steps.
    Training data: 1024^2 four-quadrant Riemann runs at K = 128 (3 x 128 angles)
    and Kn in {0.01, 0.1, 1, 5}, a snapshot every 64 of 1024 steps; the network
    is trained on the GPU by the library's tensor-core kernels.  Deployment: a
    4096^2 Riemann problem (not in the training set) at K = 24 for 4000 steps with
    the correction after every step, judged against the plain K = 128 run of the
    same problem (relative L2 of n and eps).  The plain FP32 method at
    K in {24, 32, 48, 64} gives its time to solution at the stated 1e-3.
    Reports the corrected run's population updates/s."""
    import torch
    from paper_2011_06856_gb300 import build as B
    from paper_2011_06856_gb300 import closure as CL
    from paper_2011_06856_gb300 import rlbm as R
    B.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:  # replicas: every rank runs the whole workload
        import torch.distributed as dist
        dist.init_process_group("nccl")
    t0 = time.perf_counter()
    cl = R.Closure(2, 24, seed=7)
    tr = CLOSURE_LONG_TRAIN
    X, T = CL.generate(cl, tr["grid"], 128, tr["kn"], tr["steps"], every=tr["every"])
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = CL.train(cl, X, T, iters=8000, batch=65536, lr=2e-3, decay=True)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    columns = int(X.shape[1])
    del X, T
    torch.cuda.empty_cache()
    n, steps, kn = 4096, 4000, 1.0
    feat = CL.kn_feature(W.tau_from_kn(kn, n), CLOSURE_LONG_TRAIN["grid"])
    fl = W.riemann_2d(n, n, CL.RIEMANN, jitter=0.01, seed=99)
    runs = {}
    for name, K, corrected in (("plain_K128", 128, False), ("corrected_K24", 24, True), ("plain_K24", 24, False),
                               ("plain_K32", 32, False), ("plain_K48", 48, False), ("plain_K64", 64, False)):
        sim = R.Simulation(n, n, 2, K, W.tau_from_kn(kn, n), "fp32", W.BC_COPYOUT, W.BC_COPYOUT, stream=cl.stream)
        sim.init_fields(fl)
        sim.autotune(4)
        sim.init_fields(fl)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cl.stream)
        if corrected:
            for _ in range(steps):
                sim.step(1)
                cl.apply(sim, feat)
        else:
            sim.step(steps)
        e1.record(cl.stream)
        e1.synchronize()
        runs[name] = {"K": K, "s": e0.elapsed_time(e1) * 1e-3, "kernel": sim.step_kernel, "m": sim.moments()}
        sim.close()
    ref = runs["plain_K128"]["m"]
    out = {}
    for name, r in runs.items():
        e = [CL.rel_l2(r["m"][i], ref[i]) for i in (0, 1)]
        out[name] = {"K": r["K"], "seconds": r["s"], "step_kernel": r["kernel"], "rel_l2_n_eps_vs_K128": e}
    tol = 1e-3
    meets = {k: v["seconds"] for k, v in out.items() if k != "plain_K128" and max(v["rel_l2_n_eps_vs_K128"]) <= tol}
    plain_meets = {k: v for k, v in meets.items() if k.startswith("plain")}
    t_corr = runs["corrected_K24"]["s"]
    t_corr = max_over_ranks(t_corr, world, torch.device("cuda", local))
    value = job_throughput(n * n * 72 * steps, 1, world, t_corr * 1e3)
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": t_corr * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (bf16 network weights)", "data": "synthetic",
            "config": {"workload": "closure4096_4000steps", "grid": [n, n], "N": 2, "K_coarse": 24, "K_reference": 128,
                       "kn": kn, "time_steps": steps, "runs": out, "stated_accuracy": tol,
                       "plain_runs_meeting_accuracy": plain_meets, "corrected_meets_accuracy":
                       max(out["corrected_K24"]["rel_l2_n_eps_vs_K128"]) <= tol,
                       "fastest_plain_meeting_accuracy_s": min(plain_meets.values()) if plain_meets else None,
                       "kn_feature": feat,
                       "training": {"grid": [tr["grid"], tr["grid"]], "K_fine": 128, "kn": list(tr["kn"]),
                                    "steps": tr["steps"], "snapshot_every": tr["every"], "columns": columns,
                                    "adam_steps": 8000, "batch": 65536, "generate_s": gen_s, "train_s": train_s,
                                    "loss_first_last": [float(losses[0]), float(losses[-1])]}},
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference" and args.workload not in W.WORKLOADS:
        args.workload = "shock1d_8192x4_N3K64"
    if args.workload == "batch256" and args.impl == "ours":
        run_batch(args)
        return
    if args.workload == "closure4096" and args.impl == "ours":
        run_closure(args)
        return
    if args.workload == "closure4096_4000steps" and args.impl == "ours":
        run_closure_long(args)
        return
    w = W.WORKLOADS[args.workload]
    precision = args.precision or w.precision
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, w, precision)
        return

    # CPU baseline first (before any GPU call), rank 0 at N = 1 only
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, list(w.kn))

    import torch
    import torch.distributed as dist
    from paper_2011_06856_gb300 import build as B
    from paper_2011_06856_gb300 import rlbm as R

    B.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)

    steps_pp = args.timesteps or w.steps
    kn_list = list(w.kn)
    fl = W.workload_fields(w)
    d_fields = [torch.tensor(a, dtype=torch.float64, device=dev).contiguous()
                for a in (fl.n, fl.T, fl.bx, fl.by)]
    # the Kn problems are independent: each runs on its own stream, forked from and
    # joined back to the timing stream, so their (latency-bound) kernels overlap
    stream = torch.cuda.Stream(device=dev)
    pstreams = [torch.cuda.Stream(device=dev) for _ in kn_list]
    sims = [R.Simulation(w.nx, w.ny, w.N, w.K, W.tau_from_kn(kn, w.nx, W.light_speed(w)), precision, w.bcx, w.bcy,
                         stream=ps, onlattice=bool(w.extra.get("onlattice")))
            for kn, ps in zip(kn_list, pstreams)]
    outs = [torch.empty((6, w.ny, w.nx), dtype=torch.float64, device=dev) for _ in kn_list]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    # tiling chosen by the library's autotuner (cached per problem shape)
    kind, gdeg = W.statistics(w)
    with torch.cuda.stream(stream):
        for sim in sims:
            if kind != "mj":
                sim.set_statistics(kind, gdeg)
            sim.init_device(*d_fields)
            if args.kernel:
                sim.set_tiling(args.tile_p or sim.tile_populations, args.kernel)
            else:
                sim.autotune(8)
    tiling = {"populations_per_warp": sims[0].tile_populations, "kernel": sims[0].step_kernel,
              "population_groups_per_warp": sims[0].population_groups}
    kernel_names = {"per-tile": "rlbm_kernel<MODE_STEP>", "tma": "rlbm_step_tma",
                    "pair": "rlbm_pair_kernel", "pair-bulk": "rlbm_pair_kernel (bulk-staged)",
                    "pair-tma": "rlbm_pair_tma_kernel"}

    def kernel_name(sim):
        if sim.statistics != "mj":
            return "rlbm_kernel<MODE_STEP | MODE_Q>"
        if sim.onlattice:
            return "rlbm_kernel<MODE_STEP_LATTICE>"
        if sim.population_groups > 1:
            return {"pair": "rlbm_pair_groups_kernel",
                    "per-tile": "rlbm_kernel<MODE_STEP> (population groups)"}[sim.step_kernel]
        return kernel_names[sim.step_kernel]

    # the step launches are timed inside the timed region, on the streams they
    # are issued on: events before and after every problem's run of steps; the
    # span from the first start to the last end covers all step launches of
    # the bench step (the problems run concurrently)
    kspans = []

    def one_step(timed=False):
        fork = torch.cuda.Event(enable_timing=timed)
        fork.record(stream)
        marks = []
        for sim, ps, out in zip(sims, pstreams, outs):
            ps.wait_event(fork)
            sim.init_device(*d_fields)
            if timed:
                k0 = torch.cuda.Event(enable_timing=True)
                k1 = torch.cuda.Event(enable_timing=True)
                k0.record(ps)
            sim.step(steps_pp)
            if timed:
                k1.record(ps)
                marks.append((k0, k1))
            sim.moments_device(out)
            join = torch.cuda.Event()
            join.record(ps)
            stream.wait_event(join)
        if timed:
            kspans.append((fork, marks))

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        barrier()
        l0 = sum(s.kernel_launches for s in sims)
        clk = ClockSampler(local)
        clk.start()
        ev = []
        barrier()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.random_(0, 255)  # L2 flush outside the events, on the same stream
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(timed=True)
            e1.record(stream)
            ev.append((e0, e1))
        barrier()
        t_wall = time.perf_counter() - t_wall
        clocks = clk.stop()
        launches = sum(s.kernel_launches for s in sims) - l0
        ms = [a.elapsed_time(b) for a, b in ev]

        # time per step launch over the timed region: the span of the step
        # launches of every bench step over the launches in it
        span_ms = 0.0
        for fork, marks in kspans:
            span_ms += (max(fork.elapsed_time(k1) for _, k1 in marks) -
                        min(fork.elapsed_time(k0) for k0, _ in marks))
        kernel_ms = span_ms / (len(kspans) * steps_pp * len(sims))

        # end to end through the public API with host buffers
        host_fields = [np.ascontiguousarray(a) for a in (fl.n, fl.T, fl.bx, fl.by)]
        barrier()
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            for sim in sims:
                sim.init(*host_fields)
                sim.step(steps_pp)
                sim.moments()
        barrier()
        e2e_s = (time.perf_counter() - t0) / e2e_steps

    total_ms = max_over_ranks(float(np.sum(ms)), world, dev)
    upd_per_step = w.sites * w.npop * steps_pp * len(kn_list)
    value = job_throughput(upd_per_step, args.steps, world, total_ms)
    storage = R.STORAGE_BYTES[precision]
    alg_bytes = 2 * storage * w.sites * w.npop
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    peak, peak_src = measured_peaks()
    e2e_value = upd_per_step * world / e2e_s
    S = w.sites
    working_set = 2 * storage * S * w.npop
    l2_resident = working_set < L2_BYTES
    roofline = {"bound": "l2" if l2_resident else "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "traffic": profiled_traffic(w.name, precision, sims[0].step_kernel, sims[0].tile_populations),
                "kernel": kernel_name(sims[0]), "kernel_ms": kernel_ms,
                "kernel_timing": f"CUDA events around every problem's {steps_pp} steps on its own stream, "
                                 f"inside each timed step: span of the step launches / launches in it",
                "alg_bytes_per_launch": alg_bytes}
    if l2_resident:
        roofline["note"] = (f"working set {working_set / 1e6:.0f} MB stays in the 129 MB L2 within a step: "
                            f"frac is the algorithmic rate over the HBM peak, not an HBM measurement")
    if precision == "fp64" and sims[0].step_kernel == "per-tile":
        # FP64 storage: bound by the FP64 pipe, reported against the FP64 rate measured here
        fpu = fp64_flops_per_update(w.N, w.ny > 1, w.npop)
        tf_peak, tf_src = fp64_roof(dev)
        tf = w.sites * w.npop / (kernel_ms * 1e-3) * fpu / 1e12
        roofline = {"bound": "alu", "achieved": tf, "peak": tf_peak, "unit": "TFLOP/s", "frac": tf / tf_peak,
                    "peak_source": tf_src, "flops_per_update": fpu, "kernel": roofline["kernel"],
                    "kernel_ms": kernel_ms, "traffic": roofline["traffic"], "hbm": {
                        k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "alg_bytes_per_launch")}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32",
                      "bf16": "bf16-storage/f32", "fp16n": "f16-storage/f32",
                      "bf16n": "bf16-storage/f32"}[precision],
            "data": "synthetic",
            "config": {"workload": w.name, "grid": [w.nx, w.ny], "N": w.N, "K": w.K,
                       "quadrature": "on-lattice, stencil vectors of length 5" if w.extra.get("onlattice")
                       else "off-lattice product rule",
                       "statistics": {"mj": "Maxwell-Juttner", "fd": "Fermi-Dirac", "be": "Bose-Einstein"}[kind]
                       + ("" if kind == "mj" else f", g = {gdeg}"),
                       "npop": w.npop, "kn": kn_json(kn_list), "time_steps_per_problem": steps_pp,
                       "problems_per_step": len(kn_list), "precision": precision,
                       "bc": ["copy-out" if w.bcx else "periodic", "copy-out" if w.bcy else "periodic"],
                       "l2": f"flushed between timed steps (256 MB write); working set "
                             f"{working_set / 1e6:.0f} MB {'fits' if working_set < 129e6 else 'exceeds'} "
                             f"the 129 MB L2 within a step",
                       "parallelism": f"replicas x{world} (independent problems)",
                       "concurrency": f"the {len(kn_list)} Kn problems on {len(kn_list)} streams",
                       "tiling": tiling},
            "roofline": roofline,
            "cpu_baseline": cb,
            "e2e": {"value": e2e_value, "unit": METRIC,
                    "h2d_bytes_per_step": 4 * 8 * S * len(kn_list),
                    "d2h_bytes_per_step": 6 * 8 * S * len(kn_list)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    for s in sims:
        s.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
