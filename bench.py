#!/usr/bin/env python3
"""Benchmark of the QMC-slicing fast kernel sum on GB300.

One step = one full sum s = (1/P) sum_p [spread -> FFT filter -> interpolate]
over one batch of synthetic inputs already resident in HBM (all stages of the
hot path: projection of x and y, spread, FFT filter, interpolation, slice
reduction).  The default workload is the MNIST-shaped d=784 problem:
N=M=60000, P=2048 orthogonal directions, Laplace kernel (median rule),
N_ft=1024, W=8.

Prints ONE JSON line (rank 0).  Metric: Gpoint-slices/s = (N+M) P / time / 1e9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mnist_laplace|small_gauss|gauss64_negdist] [--proj fp32|...]
                  [--no-error-check] [--no-cpu-baseline]

With several GPUs (torchrun), every rank runs an independent replica of the
workload ("replicas only": the sum needs no exchange between GPUs); the
value is the total point-slices of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
import warnings

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sliced kernel-sum ms & Gpoint-slices/s at fixed rel. error vs plain FP32"
UNIT = "Gpoint-slices/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_problem(name: str, P: int = 0, N: int = 0):
    """The named workload; P / N > 0 shrink it (small cases for profiler captures)."""
    from paper_2410_01316_gb300 import workloads as W

    if name == "mnist_laplace":
        kw = {}
        if P:
            kw["P"] = P
        if N:
            kw["N"] = kw["M"] = N
        return W.mnist_laplace(**kw)
    if name in ("mnist_matern3", "mnist_matern7"):
        kw = {"nu": 1.5 if name == "mnist_matern3" else 3.5}
        if P:
            kw["P"] = P
        if N:
            kw["N"] = kw["M"] = N
        return W.mnist_matern(**kw)
    if name == "small_gauss":
        return W.small_gauss()
    if name == "gauss64_negdist":
        kw = {}
        if P:
            kw["P"] = P
        if N:
            kw["N"] = kw["M"] = N
        return W.gauss64_negdist(**kw)
    raise SystemExit(f"unknown workload {name}")


def workload_desc(prob, proj):
    return (f"{prob.name}: d={prob.d} N={prob.N} M={prob.M} P={prob.P} kernel={prob.kernel} "
            f"N_ft={prob.n_ft} W={prob.window} proj={proj}")


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
def smi_gpu_id(dev) -> str:
    """nvidia-smi id of a torch device (its UUID; falls back to the ordinal)."""
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index)


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# oracle legs (CPU)
# ---------------------------------------------------------------------------
def oracle_sample_rate(prob, n_slices: int, n_targets: int, threads: int = 0, seed: int = 99):
    """Time the FP64 oracle on a bounded sample of the workload: the first
    n_slices directions, all N sources, n_targets sampled targets.  Returns
    (Gpoint-slices/s, seconds, description)."""
    import oracle

    rng = np.random.default_rng(seed)
    idx = rng.choice(prob.M, min(n_targets, prob.M), replace=False)
    y = np.ascontiguousarray(prob.y[idx])
    xi = np.ascontiguousarray(prob.xi[:n_slices])
    t = oracle.tau(prob.kernel, prob.kparam, prob.R)
    c = oracle.coeffs(prob.kernel, prob.kparam, prob.d, t, prob.n_ft, nu=prob.kparam2)
    t0 = time.perf_counter()
    oracle.o1_sum(prob.x, prob.w, y, xi, t, c, threads)
    dt = time.perf_counter() - t0
    ps = (prob.N + y.shape[0]) * xi.shape[0]
    desc = f"{xi.shape[0]} of {prob.P} slices, all {prob.N} sources, {y.shape[0]} of {prob.M} targets"
    return ps / dt / 1e9, dt, desc


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return
    prob = make_problem(args.workload)
    n_slices = max(1, min(prob.P, args.ref_slices))
    rates = []
    for i in range(args.warmup + args.steps):
        r, dt, desc = oracle_sample_rate(prob, n_slices, args.ref_targets, seed=1000 + i)
        if i >= args.warmup:
            rates.append((r, dt))
    tot_ps = sum(r * dt for r, dt in rates)
    tot_t = sum(dt for _, dt in rates)
    value = tot_ps / tot_t
    cores = host_cores()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(prob, "oracle-fp64-direct-ndft"), "sample_per_step": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2410_01316_gb300 import QSPlan
    from paper_2410_01316_gb300 import build as qbuild

    qbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = make_problem(args.workload, args.P, args.N)
    proj = args.proj
    plan = QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, window=prob.window,
                  proj=proj, max_n=prob.N, max_m=prob.M, kparam2=prob.kparam2)
    x = torch.from_numpy(prob.x).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    w = torch.from_numpy(prob.w).to(dev)
    s = torch.empty(prob.M, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    if args.spread_variant:
        plan.set_variant(args.spread_variant)
        spread_variant = args.spread_variant
    else:
        spread_variant = plan.autotune(x, w)
    if args.gemm != "auto" and plan.proj in ("bf16x3", "tf32"):
        plan.set_gemm(args.gemm == "pair")
    gemm = ("pair" if plan.gemm_pair() else "single") if plan.proj in ("bf16x3", "tf32") else None
    for _ in range(args.warmup):
        plan.sum(x, w, y, out=s)
    plan.check()

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    plan.set_timing(True)
    dist_barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    step_ms, stage_acc = [], {}
    for _ in range(args.steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        plan.sum(x, w, y, out=s)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for k, v in plan.stage_times().items():
            stage_acc[k] = stage_acc.get(k, 0.0) + v
    torch.cuda.synchronize()
    clocks = sampler.stop()
    dist_barrier(world)
    plan.set_timing(False)
    status = plan.status()

    t_local = sum(step_ms) / 1e3
    t_max = dist_max(t_local, world, dev)
    ms_per_step = 1e3 * t_max / args.steps
    ps_step = prob.point_slices
    value = ps_step * args.steps * world / t_max / 1e9
    stages = {k: v / args.steps for k, v in stage_acc.items()}

    # ---- end to end through the host-buffer entry point (pinned host memory)
    xh = torch.from_numpy(prob.x).pin_memory().numpy()
    yh = torch.from_numpy(prob.y).pin_memory().numpy()
    wh = torch.from_numpy(prob.w).pin_memory().numpy()
    sh = torch.empty(prob.M, dtype=torch.float32).pin_memory().numpy()
    plan.sum_host(xh, wh, yh, out=sh)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.sum_host(xh, wh, yh, out=sh)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_t = dist_max(sum(e2e_ms) / 1e3, world, dev)
    h2d = (prob.N + prob.M) * prob.d * 4 + prob.N * 4
    d2h = prob.M * 4

    line = None
    if rank == 0:
        peaks, peak_src = _peaks()
        props = torch.cuda.get_device_properties(dev)
        sm_count = props.multi_processor_count
        roof, stage_roofs = roofline(prob, plan, stages, clocks, peaks, peak_src, sm_count)
        err = None
        err_desc = None
        if not args.no_error_check:
            err, err_desc = error_vs_oracle(prob, s, args.error_targets)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(prob, plan.proj), "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (256 MB write); inputs also exceed L2",
                       "rel_err_vs_oracle": err, "rel_err_sample": err_desc,
                       "rel_err_norm": "max_m |s - s_oracle| / (sum|w| max|F|)",
                       "stage_ms": {k: round(v, 4) for k, v in stages.items()},
                       "spread_variant": spread_variant,
                       "gemm": gemm,
                       "gemm_ctas": plan.gemm_ctas() if gemm else None,
                       "device_status": int(status)},
            "roofline": roof,
            "stage_rooflines": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()
                                    if kk in ("bound", "achieved", "peak", "unit", "frac", "ms", "hbm_achieved_gbs",
                                              "hbm_frac")}
                                for k, v in stage_roofs.items()},
            "clocks": clocks,
            "e2e": {"value": ps_step * args.steps * world / e2e_t / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * e2e_t / args.steps},
            "gpu_launches": args.steps * launches_per_step(plan),
        }
        if proj != "fp32" and not args.no_fp32_compare:
            line["config"]["plain_fp32"] = plain_fp32_compare(prob, x, w, y, flush, args, err_idx_err=not args.no_error_check)
        if world == 1 and not args.no_cpu_baseline:
            r, dt, desc = oracle_sample_rate(prob, args.cpu_slices, args.cpu_targets)
            line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                                    "sample": desc, "seconds": dt}
            # the paper's CPU timings are single-threaded (Sec. 4.3)
            r1, dt1, desc1 = oracle_sample_rate(prob, args.cpu1_slices, args.cpu1_targets, threads=1)
            line["cpu_baseline_1thread"] = {"value": r1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                            "sample": desc1, "seconds": dt1}
        if world == 1 and args.workload == "mnist_laplace" and not args.no_extra_configs:
            line["config"]["precision_forms"] = precision_forms(args, flush, clocks, peaks, peak_src, sm_count)
            line["config"]["small_gauss"] = small_gauss_latency(args)
            line["config"]["other_workloads"] = other_workloads(args, rank, world, local_rank)
        print(json.dumps(line), flush=True)
    plan.close()


def other_workloads(args, rank, world, local_rank):
    """Short runs of the other workloads for the default line (each as its own bench line would
    report it, with 3 timed steps after 2 warm-ups; the sorted path's error on 8 sampled targets):
    the 256-problem batch, the d = 16 MMD flow, sorting slicing on the d = 64 workload and the
    distance-design optimiser.  A failure is recorded in place of the record, not raised, so that
    the headline line is still printed."""
    import copy

    sub = copy.copy(args)
    sub.steps, sub.warmup, sub.P, sub.N = 3, 2, 0, 0
    sub.error_targets, sub.no_error_check, sub.proj = 8, False, "bf16x3"
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "roofline", "clocks", "gpu_launches")
    out = {}
    for name, fn in (("batch256", run_batch), ("mmd_flow16", run_mmd_flow), ("distance_design", run_design),
                     ("gauss64_negdist_sorted", None)):
        try:
            if fn is None:
                sub.workload = "gauss64_negdist"
                rec = run_sorted(sub, rank, world, local_rank, emit=False)
            else:
                sub.workload = name
                rec = fn(sub, rank, world, local_rank, emit=False)
            out[name] = {k: rec[k] for k in keep if k in rec}
            out[name]["config"] = rec.get("config", {})
        except Exception as exc:  # recorded in the line; the headline stays valid
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def run_sorted(args, rank, world, local_rank, emit=True):
    """Sorting slicing (exact sliced negative-distance sums, qs_sum_sorted) on a negdist workload,
    with the Fourier path (qs_sum) on the same problem for comparison; both against the exact
    sliced oracle O3 on sampled targets."""
    import torch

    import oracle
    from paper_2410_01316_gb300 import QSPlan
    from paper_2410_01316_gb300 import build as qbuild

    qbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = make_problem(args.workload, args.P, args.N)
    if prob.kernel != "negdist":
        raise SystemExit("--sorted needs a negative-distance workload")
    plan = QSPlan(prob.d, "negdist", prob.P, prob.n_ft, prob.R, dirs=prob.xi, proj=args.proj, max_n=prob.N,
                  max_m=prob.M)
    x, y, w = (torch.from_numpy(a).to(dev) for a in (prob.x, prob.y, prob.w))
    s = torch.empty(prob.M, dtype=torch.float32, device=dev)
    sf = torch.empty(prob.M, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.sum_sorted(x, w, y, out=s)
        plan.sum(x, w, y, out=sf)
    plan.check()

    def timed(fn):
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    torch.cuda.synchronize()
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    ms_sorted = timed(lambda: plan.sum_sorted(x, w, y, out=s))
    clocks = sampler.stop()
    ms_fourier = timed(lambda: plan.sum(x, w, y, out=sf))
    status = plan.status()
    ps = prob.point_slices
    line = None
    if rank == 0:
        peaks, peak_src = _peaks()
        L = prob.N + prob.M
        by = float(L) * prob.P * (4 * 20 + 24)
        achieved = by / (ms_sorted / 1e3) / 1e9
        err = err_f = None
        desc = None
        if not args.no_error_check:
            idx = np.random.default_rng(4242).choice(prob.M, min(args.error_targets, prob.M), replace=False)
            xi = plan.directions()
            ref = oracle.o3_sliced("negdist", 0.0, prob.x, prob.w, np.ascontiguousarray(prob.y[idx]), xi)
            norm = float(np.abs(prob.w.astype(np.float64)).sum()) * prob.R
            err = float(np.max(np.abs(s.cpu().numpy().astype(np.float64)[idx] - ref)) / norm)
            err_f = float(np.max(np.abs(sf.cpu().numpy().astype(np.float64)[idx] - ref)) / norm)
            desc = f"{idx.size} sampled targets vs the exact sliced sum (O3), all sources and slices"
        line = {"metric": METRIC, "value": ps / (ms_sorted / 1e3) / 1e9, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_sorted, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_desc(prob, "sorted (exact 1D sums)"),
                           "l2": "flushed between steps (256 MB write); inputs also exceed L2",
                           "rel_err_vs_exact_sliced": err, "rel_err_sample": desc,
                           "fourier_path": {"ms_per_step": ms_fourier, "value": ps / (ms_fourier / 1e3) / 1e9,
                                            "proj": args.proj, "rel_err_vs_exact_sliced": err_f},
                           "device_status": int(status)},
                "roofline": {"kernel": "sorted sum (radix co-sort + scans)", "bound": "hbm", "achieved": achieved,
                             "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                             "traffic": None,
                             "algorithmic": "co-sort traffic: 4 radix passes x 20 B (key + payload read and "
                                            "written, key read for the histogram) + 24 B (projection, tile sums, "
                                            f"evaluation) per point-slice = {by:.3e} B",
                             "peak_source": f"hbm_gbs ({peak_src})"},
                "clocks": clocks}
        if emit:
            print(json.dumps(line), flush=True)
    plan.close()
    return line


def plain_fp32_compare(prob, x, w, y, flush, args, err_idx_err=True):
    """Same workload through the plain FP32 form (SIMT projection), timed the
    same way, for the 'vs plain FP32' part of the metric."""
    import torch

    from paper_2410_01316_gb300 import QSPlan

    steps = max(3, min(args.steps, 5))
    with QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, window=prob.window,
                proj="fp32", max_n=prob.N, max_m=prob.M, kparam2=prob.kparam2) as plan:
        s = torch.empty(prob.M, dtype=torch.float32, device=x.device)
        for _ in range(2):
            plan.sum(x, w, y, out=s)
        stream = torch.cuda.current_stream()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.sum(x, w, y, out=s)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        plan.check()
        out = {"value": prob.point_slices / (sum(ms) / len(ms) / 1e3) / 1e9, "unit": UNIT,
               "ms_per_step": sum(ms) / len(ms), "steps": steps}
        if err_idx_err:
            out["rel_err_vs_oracle"], _ = error_vs_oracle(prob, s, args.error_targets)
        return out


def precision_forms(args, flush, clocks, peaks, peak_src, sm_count):
    """The precision-form workload (d = 64, N = M = 2e5, x, y ~ N(0, I), w ~ N(0, 1),
    negative distance, P = 4096 Sobol directions, N_ft = 2048) in every projection
    form (FP32 SIMT, TF32 and BF16x3 tensor-core GEMMs; spread, FFT and interpolation
    in FP32 throughout), each timed like the headline and with its error against the
    FP64 oracle.  The oracle's cost does not depend on how many targets are sampled
    (every slice needs the full adjoint NDFT of all 2e5 sources), so each form's error
    is measured on a plan over the first `pf_error_slices` of the 4096 directions, the
    same sources and 64 sampled targets: the same kernels on the same data, a subset
    of the slices."""
    import torch

    import oracle
    from paper_2410_01316_gb300 import QSPlan

    prob = make_problem("gauss64_negdist")
    dev = flush.device
    x = torch.from_numpy(prob.x).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    w = torch.from_numpy(prob.w).to(dev)
    s = torch.empty(prob.M, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    n_sub = max(1, min(prob.P, args.pf_error_slices))
    idx = np.random.default_rng(4242).choice(prob.M, 64, replace=False)
    t_ = oracle.tau(prob.kernel, prob.kparam, prob.R)
    c = oracle.coeffs(prob.kernel, prob.kparam, prob.d, t_, prob.n_ft)
    t0 = time.perf_counter()
    ref = oracle.o1_sum(prob.x, prob.w, np.ascontiguousarray(prob.y[idx]), np.ascontiguousarray(prob.xi[:n_sub]),
                        t_, c)
    oracle_s = time.perf_counter() - t0
    norm = float(np.abs(prob.w.astype(np.float64)).sum()) * prob.R
    out = {"workload": workload_desc(prob, "per form"),
           "rel_err_sample": f"plan over the first {n_sub} of the {prob.P} directions, all {prob.N} sources, "
                             f"64 sampled targets (oracle {oracle_s:.1f} s)",
           "rel_err_norm": "max_m |s - s_oracle| / (sum|w| R)",
           "l2": "flushed between steps (256 MB write); inputs also exceed L2", "forms": {}}
    steps = max(3, min(args.steps, 5))
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    # fp32_fused: the projections formed inside the spread and interpolation (no projection
    # buffer in HBM), the unfused forms' alternative for d <= 64
    for form in ("fp32", "tf32", "bf16x3", "fp32_fused"):
        with QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, window=prob.window,
                    proj=form, max_n=prob.N, max_m=prob.M) as plan:
            variant = plan.autotune(x, w)
            gemm = ("pair" if plan.gemm_pair() else "single") if form in ("bf16x3", "tf32") else None
            for _ in range(max(3, args.warmup)):
                plan.sum(x, w, y, out=s)
            plan.check()
            plan.set_timing(True)
            ms, stage_acc = [], {}
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.sum(x, w, y, out=s)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                for k, v in plan.stage_times().items():
                    stage_acc[k] = stage_acc.get(k, 0.0) + v
            plan.set_timing(False)
            status = plan.status()
            stages = {k: v / steps for k, v in stage_acc.items()}
            _, rl = roofline(prob, plan, stages, clocks, peaks, peak_src, sm_count)
        with QSPlan(prob.d, prob.kernel, n_sub, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi[:n_sub],
                    window=prob.window, proj=form, max_n=prob.N, max_m=prob.M) as sp:
            sp.sum(x, w, y, out=s)
            sp.check()
            err = float(np.max(np.abs(s.cpu().numpy().astype(np.float64)[idx] - ref))) / norm
        t = sum(ms) / len(ms)
        # HBM bytes the form must move: inputs and output, plus, unfused, the projection buffer
        # written by the GEMM and read by the spread and interpolation (4 B per point-slice each way)
        io = 4.0 * ((prob.N + prob.M) * prob.d + prob.N + prob.M)
        u_rt = 0.0 if form == "fp32_fused" else 8.0 * (prob.N + prob.M) * prob.P
        out["forms"][form] = {
            "ms_per_step": t, "value": prob.point_slices / (t / 1e3) / 1e9, "unit": UNIT,
            "hbm_bytes_inputs_outputs": io, "hbm_bytes_projection_round_trip": u_rt,
            "rel_err_vs_oracle": err, "steps": steps, "spread_variant": variant, "gemm": gemm,
            "device_status": int(status), "stage_ms": {k: round(v, 4) for k, v in stages.items()},
            "stage_rooflines": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in v.items()
                                    if kk in ("bound", "achieved", "peak", "unit", "frac", "ms", "hbm_achieved_gbs",
                                              "hbm_frac")}
                                for k, v in rl.items()}}
    out["clocks"] = sampler.stop()
    f = out["forms"]
    out["bf16x3_speedup_vs_fp32"] = f["fp32"]["ms_per_step"] / f["bf16x3"]["ms_per_step"]
    return out


def small_gauss_latency(args):
    """The small d = 3 workload (N = M = 1000, Gauss sigma = 0.5, P = 64 spherical
    Fibonacci, N_ft = 256, Kaiser-Bessel window of width 8, fused FP32 projection):
    launch-bound, so reported as microseconds per call, directly and as a
    CUDA-graph replay of one call."""
    import torch

    from paper_2410_01316_gb300 import QSPlan

    prob = make_problem("small_gauss")
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(prob.x).to(dev)
    y = torch.from_numpy(prob.y).to(dev)
    w = torch.from_numpy(prob.w).to(dev)
    s = torch.empty(prob.M, dtype=torch.float32, device=dev)
    reps = 200
    with QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs=prob.xi, window=prob.window,
                proj="fp32_fused", max_n=prob.N, max_m=prob.M, window_kind="kb") as plan:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(5):
                plan.sum(x, w, y, out=s, stream=side)
            side.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(side)
            for _ in range(reps):
                plan.sum(x, w, y, out=s, stream=side)
            e1.record(side)
            e1.synchronize()
            direct_us = 1e3 * e0.elapsed_time(e1) / reps
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                plan.sum(x, w, y, out=s, stream=side)
            for _ in range(5):
                g.replay()
            side.synchronize()
            e0.record(side)
            for _ in range(reps):
                g.replay()
            e1.record(side)
            e1.synchronize()
            graph_us = 1e3 * e0.elapsed_time(e1) / reps
        plan.check()
    err, desc = error_vs_oracle(prob, s, prob.M)
    return {"workload": workload_desc(prob, "fp32_fused"), "us_per_call": direct_us, "us_per_graph_replay": graph_us,
            "calls": reps, "launches_per_call": 4, "rel_err_vs_oracle": err, "rel_err_sample": desc,
            "window": "Kaiser-Bessel, W = 8 taps (the oracle has no window)"}


def run_gpu_compare(args, rank, world, local_rank):
    """The paper's GPU-comparison shape (App. H, "GPU Comparison"): d = 30, N = M = 960000
    PCA-shaped points summed against themselves with unit weights, P = 5120 distance QMC
    directions (QS_DIR_DISTANCE), for the Gauss, Laplace, Matern (nu = 3/2) and negative
    distance kernels with the paper's N_ft.  A step = the four sums; per kernel: ms,
    Gpoint-slices/s, the error against the oracle (on a plan over the first
    `pf_error_slices` directions, 64 sampled targets) and the relative L1 error of the
    full sum against the exact kernel sum on those targets (the paper's error measure)."""
    import torch

    import oracle
    from paper_2410_01316_gb300 import QSPlan
    from paper_2410_01316_gb300 import build as qbuild
    from paper_2410_01316_gb300 import workloads as W

    qbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kernels = ("gauss", "laplace", "matern", "negdist")
    per, tot_ps, tot_ms = {}, 0, 0.0
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    for kern in kernels:
        prob = W.gpu_compare30(kern, P=args.P or 5120)
        x = torch.from_numpy(prob.x).to(dev)
        w = torch.from_numpy(prob.w).to(dev)
        s = torch.empty(prob.M, dtype=torch.float32, device=dev)
        with QSPlan(prob.d, prob.kernel, prob.P, prob.n_ft, prob.R, prob.kparam, dirs="distance", seed=7,
                    window=prob.window, proj="auto", max_n=prob.N, max_m=prob.M, kparam2=prob.kparam2) as plan:
            variant = plan.autotune(x, w)
            for _ in range(max(3, args.warmup)):
                plan.sum(x, w, x, out=s)
            plan.check()
            ms = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.sum(x, w, x, out=s)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            status = plan.status()
            xi = plan.directions()
            proj = plan.proj
        t = sum(ms) / len(ms)
        tot_ps += prob.point_slices
        tot_ms += t
        rec = {"ms_per_step": t, "value": prob.point_slices / (t / 1e3) / 1e9, "unit": UNIT, "N_ft": prob.n_ft,
               "kparam": prob.kparam, "proj": proj, "spread_variant": variant, "device_status": int(status)}
        if not args.no_error_check:
            idx = np.random.default_rng(4242).choice(prob.M, 64, replace=False)
            yi = np.ascontiguousarray(prob.x[idx])
            sg = s.cpu().numpy().astype(np.float64)[idx]
            exact = oracle.o2_exact(prob.kernel, prob.kparam, prob.x, prob.w, yi, nu=prob.kparam2)
            rec["rel_l1_vs_exact"] = float(np.abs(sg - exact).sum() / np.abs(exact).sum())
            n_sub = max(1, min(prob.P, args.pf_error_slices))
            with QSPlan(prob.d, prob.kernel, n_sub, prob.n_ft, prob.R, prob.kparam, dirs=xi[:n_sub],
                        window=prob.window, proj="auto", max_n=prob.N, max_m=prob.M, kparam2=prob.kparam2) as sp:
                sp.sum(x, w, x, out=s)
                sp.check()
                sub = s.cpu().numpy().astype(np.float64)[idx]
            tt = oracle.tau(prob.kernel, prob.kparam, prob.R)
            c = oracle.coeffs(prob.kernel, prob.kparam, prob.d, tt, prob.n_ft, nu=prob.kparam2)
            ref = oracle.o1_sum(prob.x, prob.w, yi, np.ascontiguousarray(xi[:n_sub]), tt, c)
            norm = float(prob.N) * (prob.R if prob.kernel == "negdist" else 1.0)
            rec["rel_err_vs_oracle"] = float(np.max(np.abs(sub - ref))) / norm
            rec["rel_err_sample"] = f"plan over the first {n_sub} of the {prob.P} directions, 64 sampled targets"
        per[kern] = rec
        del x, w, s
    clocks = sampler.stop()
    line = {"metric": METRIC, "value": tot_ps / (tot_ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gpu_compare30: d=30, N=M=960000 PCA-shaped points (independent N(0, 1/j) "
                                   "coordinates) summed against themselves, w = 1, P=5120 distance QMC directions, "
                                   "median rule; one step = the Gauss, Laplace, Matern and negative distance sums",
                       "kernels": per, "l2": "flushed between steps (256 MB write); inputs also exceed L2"},
            "clocks": clocks, "gpu_launches": args.steps * 4 * 6}
    if rank == 0:
        print(json.dumps(line), flush=True)


def slicing_rate_study(dims=(3, 10, 50), kernels=("negdist", "gauss", "laplace"), Ps=None, reps=50, n_x=1000,
                       iters=1000, designs=("iid", "orthogonal", "sobol", "distance"), seed=20241007):
    """Slicing error |F(|x|) - (1/P) sum_p f(|<xi_p, x>|)| (Sec. 4.2, eq. approximation)
    for x ~ N(0, 0.1 I), averaged over n_x samples of x and `reps` realisations of the
    directions, and its rate r (error ~ P^-r, a least-squares line in the log-log plot,
    as for Table tab:rates).  Designs: iid, orthogonal, scrambled Sobol (Sec. 4.1) and
    the library's distance QMC design (qs_distance_design on the GPU, from a seeded
    orthogonal start), randomised by a Haar rotation per realisation (App. D).  The
    sliced estimate is the oracle's closed-form sliced sum (one source at the origin),
    so only kernels whose f the oracle has in closed form enter: the negative distance
    in any d, Gauss and Laplace at d = 3.  Kernel parameters: median rule on |x|."""
    import torch

    import oracle
    from paper_2410_01316_gb300 import distance_design
    from paper_2410_01316_gb300 import workloads as W

    Ps = Ps or [5 * 2 ** k for k in range(1, 9)]
    out = {}
    for d in dims:
        rng = np.random.default_rng(seed + d)
        xs = W.gaussian(rng, n_x, d, scale=math.sqrt(0.1))
        med = float(np.median(np.linalg.norm(xs.astype(np.float64), axis=1)))
        origin = np.zeros((1, d), dtype=np.float32)
        base = {}
        if "distance" in designs:
            for P in Ps:
                xi0 = torch.from_numpy(W.directions_orthogonal(np.random.default_rng(seed + P), P, d)).cuda()
                distance_design(xi0, iters=iters)
                base[P] = xi0.cpu().numpy()
        for kern in kernels:
            if kern != "negdist" and d != 3:
                continue
            kp = {"negdist": 0.0, "gauss": med, "laplace": 1.0 / med}[kern]
            exact = np.array([oracle.F(kern, kp, float(r)) for r in np.linalg.norm(xs.astype(np.float64), axis=1)])
            res = {}
            for des in designs:
                errs = []
                for P in Ps:
                    e = 0.0
                    for rep in range(reps):
                        r = np.random.default_rng([seed, d, P, rep])
                        if des == "iid":
                            xi = W.directions_iid(r, P, d)
                        elif des == "orthogonal":
                            xi = W.directions_orthogonal(r, P, d)
                        elif des == "sobol":
                            with warnings.catch_warnings():  # P = 5 2^k is not a power of two
                                warnings.simplefilter("ignore")
                                xi = W.directions_sobol(r, P, d)
                        else:
                            xi = W.random_rotation(r, base[P])
                        est = oracle.o3_sliced(kern, kp, origin, None, xs, xi)
                        e += float(np.mean(np.abs(est - exact)))
                    errs.append(e / reps)
                slope = np.polyfit(np.log(Ps), np.log(errs), 1)[0]
                res[des] = {"rate": float(-slope), "errors": errs}
            out[f"{kern}_d{d}"] = {"kparam": kp, "P": list(Ps), "designs": res}
    return out


def run_rates(args, rank, world, local_rank):
    """Slicing-error rates of the direction designs (Sec. 4.2, Table tab:rates): one JSON
    line with the fitted rate r per kernel, dimension and design.  Not a throughput run."""
    import torch

    from paper_2410_01316_gb300 import build as qbuild

    qbuild.build()
    torch.cuda.set_device(local_rank)
    t0 = time.perf_counter()
    study = slicing_rate_study(reps=args.rate_reps)
    line = {"metric": "slicing error rate r (error ~ P^-r)", "workload": "slicing_rates: x ~ N(0, 0.1 I), d in "
            "{3, 10, 50}, P = 5 2^k (k = 1..8), iid / orthogonal / scrambled Sobol / distance QMC (library, "
            "randomly rotated) directions, median rule on |x|", "reps": args.rate_reps, "samples_x": 1000,
            "paper_rates_distance": {"gauss_d3": 2.10, "laplace_d3": 1.26, "negdist": [1.27, 0.71, 0.70]},
            "rates": {k: {des: round(v["rate"], 3) for des, v in r["designs"].items()} for k, r in study.items()},
            "study": study, "seconds": time.perf_counter() - t0}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_mmd_flow(args, rank, world, local_rank, emit=True):
    """MMD gradient flow with the negative distance kernel (App. H, MMD flows):
    particles y move by explicit Euler steps y <- y - h M grad_y G(y), where
    G(y) = MMD^2 between the particles and the fixed targets x, and the
    gradient is one qs_grad call over the joint sources [y; x] with weights
    [1/M^2; -1/(MN)].  A step = one gradient + one update."""
    import torch

    from paper_2410_01316_gb300 import QSPlan
    from paper_2410_01316_gb300 import build as qbuild
    from paper_2410_01316_gb300 import workloads as W

    qbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    st = W.mmd_flow16()
    x = torch.from_numpy(st["x"]).to(dev)
    y0 = torch.from_numpy(st["y"]).to(dev)
    N, M, d, P, n_ft = x.shape[0], y0.shape[0], st["d"], st["P"], st["n_ft"]
    xi = W.make_directions("orthogonal", P, d, st["seed"] + 11)
    R = 1.25 * 2 * float(max(x.norm(dim=1).max(), y0.norm(dim=1).max()))
    plan = QSPlan(d, "negdist", P, n_ft, R, dirs=xi, proj="fp32", max_n=N + M, max_m=N + M)
    z = torch.cat([y0, x]).contiguous()          # sources; z[:M] are the moving particles
    y = z[:M]
    wz = torch.cat([torch.full((M,), 1.0 / (M * M)), torch.full((N,), -1.0 / (M * N))]).float().to(dev)
    we = torch.cat([torch.full((M,), 0.5 / (M * M)), torch.full((N,), -1.0 / (M * N))]).float().to(dev)
    wx = torch.full((N,), 0.5 / (N * N), dtype=torch.float32, device=dev)
    h = 1.0
    gy = torch.empty((M, d), dtype=torch.float32, device=dev)
    from paper_2410_01316_gb300 import _lib
    import ctypes

    def step():
        _lib.check(plan._lib.qs_grad(plan._handle, z.data_ptr(), N + M, wz.data_ptr(), y.data_ptr(), M, None,
                                     None, None, gy.data_ptr(), torch.cuda.current_stream().cuda_stream), "qs_grad")
        y.add_(gy, alpha=-h * M)

    def mmd2():
        yc = y.contiguous()
        a = plan.sum(z, we, yc).double().sum()
        b = plan.sum(x, wx, x).double().sum()
        return float(a + b)

    curve = [(0, mmd2())]
    for _ in range(args.warmup):
        step()
    y.copy_(y0)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    ms = []
    for i in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        if (i + 1) % 10 == 0:
            curve.append((i + 1, mmd2()))
    clocks = sampler.stop()
    status = plan.status()
    t = sum(ms) / 1e3
    ps = (N + M + M) * P
    line = {"metric": METRIC, "value": ps * args.steps / t / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"mmd_flow16: d={d} N={N} targets, M={M} particles, P={P} orthogonal, "
                                   f"negdist, N_ft={n_ft}, Euler h={h} on M grad (gradient over {N + M} sources)",
                       "mmd2_curve": curve, "device_status": int(status),
                       "point_slices_per_step": f"(N + M sources + M targets) P = {ps}"},
            "clocks": clocks, "gpu_launches": args.steps * 4}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    plan.close()
    return line


def run_design(args, rank, world, local, emit=True):
    """Distance QMC design generator (Sec. 4.1 "Distance"; eq. distance-sym) at the paper's largest
    reported size, d = 200 and P = 5000: Adam steps per second.  One step = Gram matrix + pairwise
    weights + (B - A) Xi + Adam/renormalise, i.e. 4 P^2 d flop in two contractions on the tcgen05
    GEMM in BF16x3 (12 P^2 d BF16 flop); the roofline divides that by the whole step's time and the
    measured BF16 peak (the weights, operand splits and update take about as long as the GEMMs)."""
    import torch

    from paper_2410_01316_gb300 import build as qbuild
    from paper_2410_01316_gb300 import directions, distance_design, distance_energy

    qbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d, P = 200, (args.P or 5000)
    iters = 50
    x0 = torch.from_numpy(directions("orthogonal", d, P, seed=20241006)).to(dev)
    e_orth = distance_energy(x0)
    x = x0.clone()
    for _ in range(args.warmup):
        distance_design(x, iters=5)
    x.copy_(x0)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    ms, energies = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        energies.append(distance_design(x, iters=iters))
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    t = sum(ms) / 1e3
    n_it = iters * args.steps
    flops = 3 * 4.0 * P * P * d
    peaks, peak_src = _peaks()
    peak = peaks["bf16_tflops"]
    achieved = flops * n_it / t / 1e12
    line = {"metric": "distance QMC design: Adam steps per second", "value": n_it / t, "unit": "steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / n_it,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"distance_design: d={d} P={P}, {iters} Adam steps per timed call "
                                   f"(workspace allocation included), start = seeded orthogonal design",
                       "energy_start": e_orth, "energy_after": energies},
            "roofline": {"kernel": "design step", "bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "algorithmic": f"3 x 4 P^2 d = {flops:.3e} BF16 flop per step (two P x P x d "
                                        "contractions in BF16x3 on tcgen05) over the whole step, which also "
                                        "holds the pairwise weights, the operand splits, the range "
                                        "reduction and the Adam update",
                         "peak_source": f"bf16_tflops ({peak_src}, burst)"},
            "clocks": clocks, "gpu_launches": n_it * 5 + args.steps * 4}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def run_batch(args, rank, world, local_rank, emit=True):
    """One persistent, graph-captured launch over 256 independent problems."""
    import torch

    from paper_2410_01316_gb300 import QSBatch, QSPlan
    from paper_2410_01316_gb300 import build as qbuild

    qbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2410_01316_gb300 import workloads as W

    probs = W.batch256_problems()
    plans = [QSPlan(p.d, p.kernel, p.P, p.n_ft, p.R, p.kparam, dirs=p.xi, proj="auto", max_n=p.N,
                    max_m=p.M) for p in probs]
    data = [(torch.from_numpy(p.x).to(dev), torch.from_numpy(p.w).to(dev), torch.from_numpy(p.y).to(dev),
             torch.empty(p.M, dtype=torch.float32, device=dev)) for p in probs]
    ps = sum(p.point_slices for p in probs)
    batch = QSBatch(plans)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        # the library's tuner picks the mode (persistent kernel or concurrent per-problem
        # pipelines) and the persistent kernel's interpolation tiling
        best_tpt = batch.autotune(data, stream=stream)
        batch.sum(data, stream=stream)
        torch.cuda.synchronize()
        # both modes timed for the record (graph replays of one call each)
        mode_ms = {}
        for name, conc in (("persistent", False), ("concurrent", True)):
            batch.set_mode(conc)
            if not conc:
                batch.set_tiling(best_tpt if best_tpt else 4)
            gm = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gm, stream=stream):
                batch.sum(data, stream=stream)
            gm.replay()
            tm = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gm.replay()
                e1.record(stream)
                e1.synchronize()
                tm.append(e0.elapsed_time(e1))
            mode_ms[name] = min(tm)
            del gm
        batch.set_mode(best_tpt == 0)
        if best_tpt:
            batch.set_tiling(best_tpt)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            batch.sum(data, stream=stream)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(smi_gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    ms = []
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    batch.check()
    # the same problems as 256 separate qs_sum calls on one stream
    seq = []
    for rep in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for pl, (x, w, y, out) in zip(plans, data):
            pl.sum(x, w, y, out=out)
        e1.record()
        e1.synchronize()
        seq.append(e0.elapsed_time(e1))
    t = sum(ms) / len(ms)
    # per-problem ideal: the problem's point-slices at the throughput one GPU-filling problem of its
    # d class reaches (N = M = 1e5, P = 256, N_ft = 512, the same projection form), summed
    rate_big = {}
    for dd in sorted({p.d for p in probs}):
        big = W.tiny(d=dd, N=100000, M=100000, P=256, kernel="gauss", kparam=1.5 * math.sqrt(dd), n_ft=512,
                     seed=77 + dd, dirs="fibonacci" if dd == 3 else "orthogonal")
        xb, wb, yb = (torch.from_numpy(a).to(dev) for a in (big.x, big.w, big.y))
        sb = torch.empty(big.M, device=dev)
        with QSPlan(big.d, big.kernel, big.P, big.n_ft, big.R, big.kparam, dirs=big.xi, proj="auto", max_n=big.N,
                    max_m=big.M) as bp:
            bp.autotune(xb, wb)
            for _ in range(3):
                bp.sum(xb, wb, yb, out=sb)
            tb = []
            for _ in range(5):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                bp.sum(xb, wb, yb, out=sb)
                e1.record()
                e1.synchronize()
                tb.append(e0.elapsed_time(e1))
        rate_big[dd] = big.point_slices / (min(tb) / 1e3)
    ideal_ms = 1e3 * sum(p.point_slices / rate_big[p.d] for p in probs)
    line = {"metric": METRIC, "value": ps / (t / 1e3) / 1e9, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch256: 256 Gauss problems, N, M log-uniform in [1e3, 1e5], d in {3,16,64}, "
                                   "N_ft in {256,512,1024}, P=256, one graph-captured qs_sum_batched call",
                       "point_slices": ps,
                       "mode": "concurrent per-problem pipelines on 8 streams" if best_tpt == 0 else
                               f"persistent kernel, {best_tpt} targets per thread",
                       "mode_ms": mode_ms,
                       "sequential_qs_sum_ms": min(seq),
                       "speedup_vs_sequential": min(seq) / t,
                       "ideal_ms": ideal_ms, "persistent_efficiency": ideal_ms / t,
                       "efficiency_definition": "sum over problems of point-slices / the Gpoint-slices/s of one "
                                                "GPU-filling problem of the same d (N = M = 1e5, P = 256, N_ft = 512), "
                                                "divided by the measured batched time",
                       "big_problem_gps": {str(k): v / 1e9 for k, v in rate_big.items()},
                       "l2": "flushed between steps"},
            "clocks": clocks, "gpu_launches": args.steps}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    batch.close()
    for pl in plans:
        pl.close()
    return line


def launches_per_step(plan) -> int:
    # [split x,] projection x, weight bound, spread+filter, [split y,] projection y,
    # interpolation, reduction
    if plan.proj in ("bf16x3", "tf32"):
        return 8
    return 6 if plan.proj == "fp32" else 4


# DRAM bytes (read + write) per launch from one ncu capture of the default workload itself
# (d = 784, N = M = 60000, P = 2048, N_ft = 1024, BF16x3 on the SM-pair GEMM, momentwin32
# spread, 8 targets per interpolation thread; profiles/traffic_mnist_laplace.md).  Only for
# that configuration and the kernels as captured.
TRAFFIC_MNIST = {"project_x": 636.4e6, "project_y": 633.4e6, "spread_filter": 504.3e6, "interp": 520.4e6}


def _traffic(prob, plan, name):
    if (prob.d, prob.N, prob.M, prob.P, prob.n_ft, plan.proj) != (784, 60000, 60000, 2048, 1024, "bf16x3"):
        return None
    if name == "spread_filter" and plan.variant() != "momentwin32":
        return None
    if name.startswith("project") and not plan.gemm_pair():
        return None
    return TRAFFIC_MNIST.get(name)


def stage_rooflines(prob, plan, stages, clocks, peaks, peak_src, sm_count):
    """Roofline entry per stage, from the in-stream stage events (ms)."""
    mhz = clocks.get("sm_mhz") or 2070.0
    fp32_peak = sm_count * 128 * 2 * mhz * 1e6 / 1e12
    N, M, P, d, W, G = prob.N, prob.M, prob.P, prob.d, prob.window, plan.G
    out = {}

    def add(name, bound, achieved, peak, unit, what, source):
        out[name] = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak if peak else None, "traffic": _traffic(prob, plan, name),
                     "algorithmic": what,
                     "peak_source": source, "ms": stages[name]}

    for name, rows in (("project_x", N), ("project_y", M)):
        t = stages.get(name, 0.0) / 1e3
        if t <= 0 or plan.proj == "fp32_fused":  # the fused form projects inside the spread and interpolation
            continue
        if plan.proj == "bf16x3":
            fl = 6.0 * rows * P * d
            add(name, "tensor", fl / t / 1e12, peaks["bf16_tflops"], "TFLOP/s",
                f"6 {'N' if name == 'project_x' else 'M'} P d = {fl:.3e} BF16 flop (three products per FP32 product)",
                f"bf16_tflops burst ({peak_src})")
        elif plan.proj == "tf32":
            fl = 2.0 * rows * P * d
            add(name, "tensor", fl / t / 1e12, peaks["bf16_tflops"] * 1.1 / 2.25, "TFLOP/s",
                f"2 {'N' if name == 'project_x' else 'M'} P d = {fl:.3e} TF32 flop", f"bf16_tflops ({peak_src}) x 1.1/2.25 nominal TF32:BF16")
        else:
            fl = 2.0 * rows * P * d
            add(name, "alu", fl / t / 1e12, fp32_peak, "TFLOP/s",
                f"2 {'N' if name == 'project_x' else 'M'} P d = {fl:.3e} FP32 flop",
                f"{sm_count} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz")
    for name, rows in (("prep_x", N), ("prep_y", M)):
        t = stages.get(name, 0.0) / 1e3
        if t <= 0 or plan.proj not in ("bf16x3", "tf32"):  # only the tensor-core forms split operands
            continue
        by = rows * d * 8.0  # read FP32, write BF16 hi + lo (or TF32)
        add(name, "hbm", by / t / 1e9, peaks["hbm_gbs"], "GB/s", f"8 B per coordinate = {by:.3e} B",
            f"hbm_gbs ({peak_src})")
    unfused = plan.proj != "fp32_fused"

    def hbm(name, by, what):
        # the same stage against HBM: its algorithmic byte stream
        t_ = stages[name] / 1e3
        out[name].update({"hbm_bytes": by, "hbm_algorithmic": what, "hbm_achieved_gbs": by / t_ / 1e9,
                          "hbm_frac": by / t_ / 1e9 / peaks["hbm_gbs"]})

    # spread and interpolation: unfused, bound by their HBM stream (U, weights, rows); fused, by the
    # FP32 dot products of the projection they contain
    for name, by, what, rows in (
            ("spread_filter", 4.0 * N * P + 4.0 * N + 4.0 * P * G,
             "4 N P (U) + 4 N (w) read, 4 P G (filtered rows) written", N),
            ("interp", 4.0 * M * P + 4.0 * P * G, "4 M P (U) + 4 P G (filtered rows) read", M)):
        t = stages.get(name, 0.0) / 1e3
        if t <= 0:
            continue
        if unfused:
            add(name, "hbm", by / t / 1e9, peaks["hbm_gbs"], "GB/s", f"{what} = {by:.3e} B", f"hbm_gbs ({peak_src})")
            hbm(name, by, what)
        else:
            fl = 2.0 * rows * P * d
            add(name, "alu", fl / t / 1e12, fp32_peak, "TFLOP/s",
                f"2 {'N' if name == 'spread_filter' else 'M'} P d = {fl:.3e} FP32 flop (the projection inside the kernel)",
                f"{sm_count} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz")
    return out


# stages launched by the same kernel (one launch each per step)
KERNEL_STAGES = {"projection GEMM": ("project_x", "project_y"), "operand split": ("prep_x", "prep_y"),
                 "spread_filter": ("spread_filter",), "interp": ("interp",)}


def roofline(prob, plan, stages, clocks, peaks, peak_src, sm_count):
    """Roofline of the dominant kernel of the step: the kernel with the largest
    device time per step summed over its launches (the projection GEMM runs
    twice, once for the sources and once for the targets).  achieved = the
    algorithmic work of its launches / their summed duration; traffic = DRAM
    bytes per launch (mean over its launches)."""
    rl = stage_rooflines(prob, plan, stages, clocks, peaks, peak_src, sm_count)
    best, best_ms = None, -1.0
    for kern, names in KERNEL_STAGES.items():
        got = [rl[n] for n in names if n in rl]
        ms = sum(g["ms"] for g in got)
        if got and ms > best_ms:
            best, best_ms = (kern, got), ms
    kern, got = best
    first = got[0]
    work = sum(g["achieved"] * g["ms"] for g in got)  # achieved x ms = work / 1e3 in the unit's scale
    achieved = work / best_ms
    tr = [g["traffic"] for g in got]
    out = dict(first)
    out.update({"kernel": kern, "stages": [g["kernel"] for g in got], "launches": len(got),
                "achieved": achieved, "frac": achieved / first["peak"] if first["peak"] else None,
                "traffic": (sum(tr) / len(tr)) if all(t is not None for t in tr) else None,
                "ms": best_ms, "ms_per_launch": best_ms / len(got)})
    if kern == "projection GEMM":
        tc = "tc_project_pair" if plan.proj in ("bf16x3", "tf32") and plan.gemm_pair() else "tc_project_persistent"
        out["kernel"] = {"bf16x3": f"{tc}<BF16x3>", "tf32": f"{tc}<TF32>",
                         "fp32": "project_fp32_kernel"}.get(plan.proj, kern)
    if len(got) > 1:
        out["algorithmic"] = (" + ".join(g["algorithmic"].split(" = ")[0] for g in got)
                              + f" over {len(got)} launches ({', '.join(g['kernel'] for g in got)}); per launch: "
                              + "; ".join(g["algorithmic"].split(" = ", 1)[1] for g in got))
    return out, rl


def error_vs_oracle(prob, s, n_targets: int):
    import oracle

    idx = np.random.default_rng(4242).choice(prob.M, min(n_targets, prob.M), replace=False)
    t = oracle.tau(prob.kernel, prob.kparam, prob.R)
    c = oracle.coeffs(prob.kernel, prob.kparam, prob.d, t, prob.n_ft, nu=prob.kparam2)
    ref = oracle.o1_sum(prob.x, prob.w, np.ascontiguousarray(prob.y[idx]), prob.xi, t, c)
    sg = s.detach().cpu().numpy().astype(np.float64)[idx]
    norm = float(np.abs(prob.w.astype(np.float64)).sum()) * (prob.R if prob.kernel == "negdist" else 1.0)
    return float(np.max(np.abs(sg - ref)) / norm), f"{idx.size} sampled targets, all sources and slices"


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------
_PG = None


def dist_init():
    global _PG
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        _PG = dist
    return rank, world, local


def dist_barrier(world):
    if world > 1 and _PG is not None:
        _PG.barrier()


def dist_max(v: float, world: int, dev) -> float:
    if world == 1 or _PG is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64, device=dev)
    _PG.all_reduce(t, op=_PG.ReduceOp.MAX)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mnist_laplace")
    ap.add_argument("--proj", default="bf16x3")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip the same-run measurement of the plain FP32 form")
    ap.add_argument("--P", type=int, default=0, help="override the number of slices (profiling small cases)")
    ap.add_argument("--N", type=int, default=0, help="override N = M (profiling small cases)")
    ap.add_argument("--no-error-check", action="store_true")
    ap.add_argument("--spread-variant", default="", help="fix the spread variant instead of timing the family")
    ap.add_argument("--sorted", action="store_true", help="negdist workloads: exact sums by sorting slicing")
    ap.add_argument("--gemm", default="auto", choices=["auto", "pair", "single"],
                    help="tensor-core projection GEMM on SM pairs (cta_group::2) or one CTA per SM")
    ap.add_argument("--error-targets", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-slices", type=int, default=128)
    ap.add_argument("--cpu-targets", type=int, default=1024)
    ap.add_argument("--cpu1-slices", type=int, default=8, help="single-thread oracle sample: slices")
    ap.add_argument("--cpu1-targets", type=int, default=256, help="single-thread oracle sample: targets")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the precision-form (d = 64) and small d = 3 sub-records of the default workload")
    ap.add_argument("--pf-error-slices", type=int, default=64,
                    help="slices of the precision-form error check (oracle cost grows with them)")
    ap.add_argument("--rate-reps", type=int, default=50, help="slicing_rates: realisations per design and P")
    ap.add_argument("--ref-slices", type=int, default=16)
    ap.add_argument("--ref-targets", type=int, default=1024)
    args = ap.parse_args()
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "mmd_flow16":
        run_mmd_flow(args, rank, world, local)
    elif args.workload == "batch256":
        run_batch(args, rank, world, local)
    elif args.workload == "gpu_compare30":
        run_gpu_compare(args, rank, world, local)
    elif args.workload == "slicing_rates":
        run_rates(args, rank, world, local)
    elif args.workload == "distance_design":
        run_design(args, rank, world, local)
    elif args.sorted:
        run_sorted(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1 and _PG is not None:
        _PG.barrier()
        _PG.destroy_process_group()


if __name__ == "__main__":
    main()
