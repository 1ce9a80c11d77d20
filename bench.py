#!/usr/bin/env python
"""Benchmark of the AF-NS Runge-Kutta step on one B300 (or N replicas).

A "step" is one SSP-RK54 time step of the 2D smooth periodic Navier-Stokes
workload (1024 x 1024 cells, 4 point sites + cell averages, mu = 0.01, Pr = 0.72):
CFL reduction (Eq. (13)), five fused stage kernels (point residual, high- and
low-order face fluxes, smoothness and positivity limiters, point scaling
limiter, RK combination) with their ghost fills, and the restart-flag read
(Remark 3.2). The metric is cell-stage updates per second:
cells x 5 x steps / seconds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   (the CPU oracle, timed on a bounded sample)
  python bench.py --workload batch ...   (256 uneven problems, persistent kernel + graph)
  python bench.py --workload tube [--t-end T] ...   (walled shock tube 2000 x 1000)
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D cell-stage updates/s and HBM fraction, FP32-mixed vs FP64, at stated L1 error vs oracle"
UNIT = "cell-stage updates/s"
N_CELLS = 1024
# FP64 peak of one B300 (TFLOP/s) from its unit counts (the FP64 pipe is 1/64 of
# the FP32 rate on sm_103): 148 SMs x 2 FP64 FMA per SM per clock x 2 flops x
# 2.032 GHz (max SM clock)
FP64_DERIVED_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
# 148 SMs x 128 FP32 lanes x 2 flops x 2.032 GHz
FP32_DERIVED_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# DRAM bytes (read + write) per stage launch from ncu (one launch of a step of
# the benchmark flow at 1024x1024), keyed by the digest of the kernel sources and
# the launch configuration they were taken on; reported only while both match.
MEASURED_TRAFFIC = {
    "mixed:e71b91eac6336001:32x8x256": 87.646e6 + 42.031e6,
    "mixed:e71b91eac6336001:16x8x128": 88.048e6 + 43.877e6,
    "fp64:e71b91eac6336001:16x8x128": 137.804e6 + 91.294e6,
}


def kernel_digest(precision):
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2609_29081_b300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.startswith("stage2d") or f == "afns_dev.cuh":
            h.update(open(os.path.join(d, f), "rb").read())
    return precision + ":" + h.hexdigest()[:16]


def measure_alu_peaks():
    """FP64 and FP32 FMA-chain throughput measured on this GPU (TFLOP/s)."""
    from paper_2609_29081_b300._native import FP64, MIXED, alu_peak
    out = {}
    for name, p in (("fp64", FP64), ("fp32", MIXED)):
        try:
            out[name] = alu_peak(p)
        except Exception:
            out[name] = None
    return out


def stage_roofline(precision, cells, stage_ms, peaks, alu_pk, tuned=None):
    """Roofline of the stage kernel: the slower of the algorithmic HBM bytes at
    the measured copy bandwidth and the algorithmic flops at the measured FMA
    rate (FP64 path: FP64 flops; mixed path: FP32 flops, 256 B per cell-stage)."""
    sec = stage_ms / 1e3
    hbm = peaks.get("hbm_gbs")
    hbm_src = "of measured: MEASURED_PEAKS.json hbm_gbs" if hbm else "of fallback: 6400 GB/s"
    hbm = hbm or 6400.0
    key = "fp64" if precision == "fp64" else "fp32"
    derived = FP64_DERIVED_TFLOPS if precision == "fp64" else FP32_DERIVED_TFLOPS
    alu = alu_pk.get(key)
    alu_src = "of measured: %s FMA chains on this GPU (af_alu_peak)" % key.upper() if alu else \
        "of derived: unit counts x 2.032 GHz"
    alu = alu or derived
    bpc = BYTES_PER_CELL_STAGE_FP64 if precision == "fp64" else BYTES_PER_CELL_STAGE_MIXED
    t_hbm = bpc * cells / (hbm * 1e9)
    t_alu = FLOPS_PER_CELL_STAGE * cells / (alu * 1e12)
    dig = kernel_digest(precision)
    cfg = "%dx%dx%d" % (tuned["tile_x"], tuned["tile_y"], tuned["threads"]) if tuned else ""
    traffic = MEASURED_TRAFFIC.get(dig + ":" + cfg)
    kern = "k_stage2d<double>" if precision == "fp64" else "k_stage2d<float>"
    common = {"traffic": traffic, "kernel": kern, "kernel_digest": dig, "launch_config": cfg,
              "hbm_frac": t_hbm / sec, "alu_frac": t_alu / sec,
              "alu_peak_tflops": alu, "alu_peak_source": alu_src,
              "alu_peak_derived_tflops": derived, "hbm_peak_gbs": hbm}
    if t_alu >= t_hbm:
        achieved = FLOPS_PER_CELL_STAGE * cells / sec / 1e12
        r = {"bound": "alu", "achieved": achieved, "peak": alu, "unit": "TFLOP/s", "frac": achieved / alu,
             "work_per_cell": "%.0f flops (counted: oracle/opcount_smooth2d.json)" % FLOPS_PER_CELL_STAGE,
             "peak_source": alu_src}
    else:
        achieved = bpc * cells / sec / 1e9
        r = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
             "work_per_cell": "%.1f bytes" % bpc, "peak_source": hbm_src}
    r.update(common)
    return r


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


PREHEAT_S = 0.3


def preheat(step, warmup):
    """Run `warmup` untimed steps, then keep stepping (untimed) until the device
    has been busy for PREHEAT_S seconds; returns the number of steps run."""
    import torch
    t0 = time.perf_counter()
    n = 0
    while n < warmup or time.perf_counter() - t0 < PREHEAT_S:
        step()
        n += 1
    torch.cuda.synchronize()
    return n


def clocks_start():
    f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
    f.close()
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200",
                              "-i", os.environ.get("LOCAL_RANK", "0"), "-f", f.name],
                             stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    except Exception:
        p = None
    return p, f.name


def clocks_stop(p, path):
    out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    if p is None:
        return out
    time.sleep(0.3)
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    try:
        rows = [r.split(",") for r in open(path).read().strip().splitlines() if r.strip()]
        os.unlink(path)
    except Exception:
        return out
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        r = [x.strip() for x in r]
        try:
            sm.append(float(r[1]))
            mx.append(float(r[2]))
        except Exception:
            continue
        for k, nm in enumerate(names):
            if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                reasons.add(nm)
    if sm:
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        out = {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
               "samples": len(sm)}
    return out


def dist_setup(args):
    """One process per GPU (torchrun): NCCL for the GPU arms, gloo for the CPU
    reference arm; no collective touches the data path (replicas / independent
    problems), only the timing reduction."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if args.impl != "reference":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl" if args.impl != "reference" else "gloo")
        return dist, rank, ws
    return None, 0, 1


def reduce_over_ranks(dist, values, ops):
    """Reduce floats across ranks ("max" for times, "sum" for work) on the
    backend's device; returns them unchanged without a process group."""
    if not dist:
        return list(values)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    out = []
    for v, op in zip(values, ops):
        t = torch.tensor([float(v)], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
        out.append(float(t.item()))
    return out


def batch_seed(rank):
    """Problem-set seed of a rank in the batched arm: rank 0 runs the seed-5 set,
    every other rank an independent set of the same statistics (weak scaling)."""
    return 5 + rank


def workload_name(n):
    return ("2D smooth periodic NS %dx%d (rho=1+0.2sin(x+y), (u,v)=(1,0.5)+8-mode perturbation, p=1, mu=0.01, "
            "Pr=0.72), CFL steps, limiter s+pp" % (n, n))


def reference_arm(args, rank, ws):
    """The oracle as it stands, on the host cores: each timed step is one full
    SSP-RK54 step of the same flow on a 128 x 128 sample of the grid."""
    if rank != 0:
        return
    import oracle as O
    from paper_2609_29081_b300 import workloads as W
    n = 128
    w = W.smooth_2d(n)
    P = O.problem(2, n, n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    s = w.state.copy()
    for _ in range(args.warmup):
        O.step(P, s, O.dt_max(P, s))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(P, s, O.dt_max(P, s))
    sec = time.perf_counter() - t0
    val = n * n * 5 * args.steps / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n), "precision": "fp64 (oracle)",
                       "sample": "each timed step: one SSP-RK54 step of the same flow on a %dx%d grid" % (n, n)},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d SSP-RK54 steps on a %dx%d sample of the workload" % (args.steps, n, n)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, S, args):
    """The oracle's residual of one stage at full size, timed on the host, and the
    L1 distance of the GPU residual from it (bounded sample: one stage)."""
    import oracle as O
    P = O.problem(2, *w.n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    dt = O.dt_max(P, w.state)
    t0 = time.perf_counter()
    Lr, _ = O.residual(P, w.state, dt)
    sec = time.perf_counter() - t0
    return Lr, dt, {"value": w.cells / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": "one limited stage residual L(u) of the full %dx%d workload (%.1f s)"
                              % (w.n[0], w.n[1], sec)}


def host_description():
    """nproc and the CPU model of this host (from lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _oracle_sample_step(n):
    """One SSP-RK54 step of the benchmark flow on an n x n grid in the oracle
    (runs in a spawned worker process); returns its seconds."""
    import oracle as O
    from paper_2609_29081_b300 import workloads as W
    w = W.smooth_2d(n)
    P = O.problem(2, n, n, lo=w.lo, hi=w.hi, mu=w.mu, Pr=w.Pr, bc=w.bc, gamma=w.gamma)
    s = w.state.copy()
    t0 = time.perf_counter()
    O.step(P, s, O.dt_max(P, s))
    return time.perf_counter() - t0


def cpu_all_cores(n=128):
    """The oracle as it stands on every host core: nproc independent processes
    (spawned), each one SSP-RK54 step of the benchmark flow on an n x n sample;
    cell-stage updates of all of them over the wall time."""
    import multiprocessing as mp
    import oracle as O
    O.build()
    k = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(k) as pool:
        pool.map(_oracle_sample_step, [16] * k)          # workers up and the library loaded
        t0 = time.perf_counter()
        pool.map(_oracle_sample_step, [n] * k)
        sec = time.perf_counter() - t0
    return {"value": k * n * n * 5 / sec, "unit": UNIT, "cores": k, "kind": "oracle",
            "sample": "%d independent processes, each one SSP-RK54 step of the same flow on a %dx%d grid (%.1f s)"
                      % (k, n, n, sec)}


def tube_measure(args, steps, warmup):
    """Walled shock tube (2000 x 1000, no-slip walls, symmetry on top), mixed
    path, autotuned: `steps` timed CFL steps after the warm-up, with the extreme
    density and pressure of every DoF afterwards (sub-record of the default line)."""
    import torch
    from paper_2609_29081_b300 import Solver, workloads as W
    from paper_2609_29081_b300._native import MIXED
    w = W.shock_tube_2d((2000, 1000))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        S = Solver.from_workload(w, precision=MIXED, stream=stream)
        S.set_state(w.state)
        tuned = S.tune()
        warm = preheat(lambda: S.step(0.0), warmup)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        restarts = 0
        for _ in range(steps):
            restarts += S.step(0.0)[1]
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        st = W.split_sites(S.get_state(), 2, *w.n)
        S.close()
    pmin = min(float((0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])).min()) for U in st)
    rmin = min(float(U[0].min()) for U in st)
    return {"value": w.cells * 5 * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "warmup_steps_run": warm, "restarts": restarts, "tuned": tuned,
            "workload": "2D viscous shock tube, walled box [0,1]x[0,0.5], 2000x1000, mu=1e-3, Pr=0.73, "
                        "(120,0,0,120/1.4)|(1.2,0,0,1.2/1.4), no-slip x-lo/x-hi/y-lo, symmetry y-hi, mixed, "
                        "timed CFL steps following the warm-up steps from t = 0",
            "positivity": {"rho_min": rmin, "p_min": pmin}}


def tube_arm(args, dist, rank, ws):
    """2D viscous shock tube in a walled box (no-slip walls, symmetry on top),
    2000 x 1000 cells, Re = 1000: K timed CFL steps after the warm-up; with
    --t-end the whole run from t = 0 is timed as well (the paper's wall-clock
    figures for this problem are on 24 CPU cores, context only)."""
    import torch
    from paper_2609_29081_b300 import Solver, build, workloads as W
    from paper_2609_29081_b300._native import FP64, MIXED
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = W.shock_tube_2d((2000, 1000))
    prec = FP64 if args.precision == "fp64" else MIXED
    stream = torch.cuda.Stream()
    full = None
    with torch.cuda.stream(stream):
        S = Solver.from_workload(w, precision=prec, stream=stream)
        S.set_state(w.state)
        tuned = S.tune()
        if args.t_end > 0:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ns, nr = S.advance(args.t_end)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            full = {"t_end": args.t_end, "seconds": sec, "steps": ns, "restarts": nr,
                    "cell_stage_per_s": w.cells * 5 * ns / sec,
                    "paper_context": "AF on a 24-core Apple M3 Ultra: 8 h 35 min for this grid to t = 1"}
            S.set_state(w.state)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        cp, cpath = clocks_start()
        time.sleep(0.4)
        warm_done = preheat(lambda: S.step(0.0), args.warmup)
        S.set_profiling(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        restarts = 0
        for _ in range(args.steps):
            restarts += S.step(0.0)[1]
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = clocks_stop(cp, cpath)
        ms = reduce_over_ranks(dist, [ev0.elapsed_time(ev1)], ["max"])[0]
        prof = S.profile()
        S.set_profiling(False)
        st = W.split_sites(S.get_state(), 2, *w.n)
        pmin = min(float((0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])).min()) for U in st)
        rmin = min(float(U[0].min()) for U in st)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": w.cells * 5 * args.steps * ws / (ms / 1e3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "2D viscous shock tube, walled box [0,1]x[0,0.5], 2000x1000, mu=1e-3, "
                                   "Pr=0.73, (120,0,0,120/1.4)|(1.2,0,0,1.2/1.4), no-slip x-lo/x-hi/y-lo, "
                                   "symmetry y-hi, CFL steps, limiter s+pp",
                       "precision": args.precision, "tuned": tuned, "restarts": restarts,
                       "warmup_steps_run": warm_done, "l2": "inputs larger than L2"},
            "clocks": clocks, "gpu_launches": prof["launches"], "stage_ms": prof["stage_ms"] / max(prof["stage_launches"], 1),
            "positivity": {"rho_min": rmin, "p_min": pmin}}
    if full:
        line["full_run"] = full
    print(json.dumps(line), flush=True)


def ladder_arm(args, rank):
    """Grid-refinement ladder of the smooth periodic flow, 256^2 .. 2048^2, to
    --t-end (default: the time 200 FP64 CFL steps reach on 1024^2, the benchmark's
    run length), with the limiter s+pp and without limiter: relative L1 distance
    of the cell averages of N cells from the 2N solution restricted by 2x2
    averaging and the observed orders, for the FP64 and the mixed path, and the
    mixed path's distance from FP64 on every grid."""
    import torch
    from paper_2609_29081_b300 import Solver, build, workloads as W
    from paper_2609_29081_b300._native import FP64, MIXED
    build.build()
    if args.t_end > 0:
        t_end = args.t_end
    else:
        w = W.smooth_2d(1024)
        S = Solver.from_workload(w, precision=FP64)
        S.set_state(w.state)
        for _ in range(ACCURACY_STEPS):
            S.step(0.0)
        S.get_state()
        t_end = S.t
        S.close()
    ns = [256, 512, 1024, 2048]
    out = {"t_end": t_end}
    for lim_name, lim in (("s+pp", 2), ("none", 0)):
        res = {}
        for name, prec in (("mixed", MIXED), ("fp64", FP64)):
            sol, secs = {}, {}
            for n in ns:
                w = W.smooth_2d(n)
                S = Solver.from_workload(w, precision=prec, limiter=lim)
                S.set_state(w.state)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                steps, _ = S.advance(t_end)
                torch.cuda.synchronize()
                secs[n] = (time.perf_counter() - t0, steps)
                sol[n] = W.split_sites(S.get_state(), 2, n, n)[0]
                S.close()
                torch.cuda.empty_cache()
            err = []
            for n in ns[:-1]:
                f = sol[2 * n]
                r = 0.25 * (f[:, 0::2, 0::2] + f[:, 1::2, 0::2] + f[:, 0::2, 1::2] + f[:, 1::2, 1::2])
                err.append(float(np.abs(sol[n] - r).sum() / np.abs(r).sum()))
            res[name] = {"n": ns[:-1], "l1": err,
                         "orders": [float(np.log2(err[k] / err[k + 1])) for k in range(len(err) - 1)],
                         "seconds_steps": {str(n): secs[n] for n in ns}}
            if name == "mixed":
                mixed_sol = sol
            else:
                res["mixed_vs_fp64_l1"] = {str(n): float(np.abs(mixed_sol[n] - sol[n]).sum() / np.abs(sol[n]).sum())
                                           for n in ns}
        out[lim_name] = res
    if rank == 0:
        print(json.dumps({"workload": "2D smooth periodic NS refinement ladder, t_end=%g, limiter s+pp and none"
                                      % t_end, "ladder": out}), flush=True)


def batch_measure(args, dist, rank, ws, steps, warmup, nprob):
    """Batched form: nprob independent periodic problems of uneven sizes (mixed
    precision, persistent stage kernel, CUDA graph, autotuned configuration),
    timed over `steps` graph-replayed batch steps; the same problems advanced one
    by one in FP64 on a bounded sample. Restarted (rejected) problem steps count
    as time, not as updates."""
    import torch
    from paper_2609_29081_b300 import BatchSolver, Solver, build, workloads as W
    from paper_2609_29081_b300._native import FP64, MIXED
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wls = W.batch_problems(nprob=nprob, seed=batch_seed(rank))
    B = BatchSolver(wls, precision=MIXED)
    for i, w in enumerate(wls):
        B.set_state(i, w.state)
    cfg = B.tune()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    cp, cpath = clocks_start()
    time.sleep(0.4)
    warm_done = preheat(lambda: (B.step_all(1, graph=True), B.sync()), warmup)
    acc0 = [B.stats(i)["accepted"] for i in range(len(wls))]
    rst0 = [B.stats(i)["restarts"] for i in range(len(wls))]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(B.stream)
    B.step_all(steps, graph=True)
    ev1.record(B.stream)
    nlaunch = B.sync()
    torch.cuda.synchronize()
    clocks = clocks_stop(cp, cpath)
    ms = ev0.elapsed_time(ev1)
    st = [B.stats(i) for i in range(len(wls))]
    updates = sum(w.cells * 5 * (s["accepted"] - a0) for w, s, a0 in zip(wls, st, acc0))
    restarts = sum(s["restarts"] - r0 for s, r0 in zip(st, rst0))
    failed = sum(s["failed"] for s in st)
    B.close()
    ms, updates = reduce_over_ranks(dist, [ms, updates], ["max", "sum"])
    value = updates / (ms / 1e3)
    # FP64 one by one on a bounded sample (first 16 problems, 2 timed steps each)
    one_cells, one_ms = 0, 0.0
    for w in wls[:16]:
        S = Solver.from_workload(w, precision=FP64)
        S.set_state(w.state)
        S.step(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(2):
            S.step(0.0)
        torch.cuda.synchronize()
        one_ms += 1e3 * (time.perf_counter() - t0)
        one_cells += w.cells * 5 * 2
        S.close()
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs") or 6400.0
    alu = measure_alu_peaks().get("fp32") or FP32_DERIVED_TFLOPS
    sec = ms / 1e3
    t_hbm = updates * BYTES_PER_CELL_STAGE_MIXED / (hbm * 1e9)
    t_alu = updates * FLOPS_PER_CELL_STAGE / (alu * 1e12)
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": updates * FLOPS_PER_CELL_STAGE / sec / 1e12, "peak": alu,
                "unit": "TFLOP/s", "frac": t_alu / sec}
    else:
        roof = {"bound": "hbm", "achieved": updates * BYTES_PER_CELL_STAGE_MIXED / sec / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": t_hbm / sec}
    roof.update({"hbm_frac": t_hbm / sec, "alu_frac": t_alu / sec,
                 "work_per_cell": "%.0f flops (counted) / %.0f bytes per accepted cell-stage"
                                  % (FLOPS_PER_CELL_STAGE, BYTES_PER_CELL_STAGE_MIXED),
                 "time": "whole batch steps (CFL, ghost, stage and commit kernels, graph replay)",
                 "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs; FP32 FMA chains (af_alu_peak)"})
    return {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "warmup_steps_run": warm_done,
            "workload": "batched: %d periodic 2D problems, sides from {64..512}, mu log-uniform [1e-4,1e-2], "
                        "Mach 0.1-3, 25%% near-vacuum blasts (seed 5 + rank)" % len(wls),
            "cells": int(sum(w.cells for w in wls)), "tuned": cfg, "restarts": restarts, "failed": failed,
            "graph": True, "gpu_launches": nlaunch * steps, "clocks": clocks, "roofline": roof,
            "fp64_one_by_one": {"value": one_cells / (one_ms / 1e3), "unit": UNIT,
                                "sample": "first 16 problems, 2 FP64 steps each, one problem at a time"}}


def batch_arm(args, dist, rank, ws):
    """The batched workload as the bench line's headline (--workload batch)."""
    b = batch_measure(args, dist, rank, ws, args.steps, args.warmup, args.nprob)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": b["workload"], "cells": b["cells"], "tuned": b["tuned"],
                       "restarts": b["restarts"], "graph": True, "warmup_steps_run": b["warmup_steps_run"]},
            "roofline": b["roofline"], "clocks": b["clocks"], "gpu_launches": b["gpu_launches"],
            "fp64_one_by_one": b["fp64_one_by_one"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libafns")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the run in the other precision")
    ap.add_argument("--n", type=int, default=N_CELLS)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-contexts", type=int, default=E2E_CONTEXTS,
                    help="independent contexts of the pipelined end-to-end loop")
    ap.add_argument("--no-ladder", dest="ladder", action="store_false",
                    help="skip the accuracy ladder at the run length (128^2 .. 2048^2, FP64 and mixed)")
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="skip the batched sub-record of the default line")
    ap.add_argument("--no-tube", dest="tube", action="store_false",
                    help="skip the walled shock-tube sub-record of the default line")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "tube", "ladder"])
    ap.add_argument("--t-end", type=float, default=0.0)
    ap.add_argument("--nprob", type=int, default=256)
    ap.add_argument("--tile", type=lambda s: tuple(int(v) for v in s.split("x")), default=None,
                    help="fixed 2D launch configuration TXxTYxTHREADS (e.g. 16x8x128) instead of the autotuner")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    dist, rank, ws = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, rank, ws)
        return
    if args.workload == "batch":
        batch_arm(args, dist, rank, ws)
        return
    if args.workload == "tube":
        tube_arm(args, dist, rank, ws)
        return
    if args.workload == "ladder":
        ladder_arm(args, rank)
        return

    import torch
    from paper_2609_29081_b300 import build, workloads as W
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = W.smooth_2d(args.n)
    alu_pk = measure_alu_peaks()
    main_run = single_run(args, w, args.precision, dist, ws, e2e=True)
    other = "fp64" if args.precision == "mixed" else "mixed"
    cmp_run = single_run(args, w, other, dist, ws, e2e=False) if args.compare else None
    if rank != 0:
        return
    peaks = load_peaks()
    cells = w.cells
    r = main_run
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n),
                       "precision": args.precision, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "working set larger than L2: a stage reads 1-3 state buffers of %.0f MB and writes 1-2"
                             % (w.cells * (20 * 4 if args.precision == "mixed" else 16 * 8) / 1e6),
                       "restarts": r["restarts"], "tuned": r["tuned"], "warmup_steps_run": r["warm_done"]},
            "roofline": stage_roofline(args.precision, cells, r["stage_ms"], peaks, alu_pk, r["tuned"]),
            "clocks": r["clocks"],
            "e2e": {"value": r["e2e_pipe"]["value"], "unit": UNIT, "h2d_bytes_per_step": r["state_bytes"],
                    "d2h_bytes_per_step": r["state_bytes"], "ms_per_step": r["e2e_pipe"]["ms_per_step"],
                    "contexts": r["e2e_pipe"]["contexts"],
                    "what": ("%d independent contexts of the workload, each on its own stream and host thread; "
                             "every step of each: %s from pinned host memory, af_step, %s to pinned host memory "
                             "(uploads, steps and downloads of different contexts overlap)"
                             % (r["e2e_pipe"]["contexts"],
                                *(("af_set_state_f32", "af_get_state_f32") if args.precision == "mixed"
                                  else ("af_set_state", "af_get_state")))),
                    "one_context": {"value": r["e2e"], "ms_per_step_parts": r["e2e_parts_ms"],
                                    "what": "the same loop on one context, calls back to back"}},
            "gpu_launches": r["launches"],
            "stage_ms": r["stage_ms"]}
    if cmp_run:
        c = cmp_run
        line[other] = {"value": c["value"], "unit": UNIT, "ms_per_step": c["ms"] / args.steps,
                       "stage_ms": c["stage_ms"], "tuned": c["tuned"], "restarts": c["restarts"],
                       "roofline": stage_roofline(other, cells, c["stage_ms"], peaks, alu_pk, c["tuned"])}
    if args.ladder:
        acc = accuracy_ladder(args.n, ACCURACY_STEPS)
        key = str(args.n)
        line["accuracy"] = acc
        line["l1_mixed_vs_fp64"] = {"value": acc["mixed_vs_fp64_l1"][key],
                                    "linf": acc["mixed_vs_fp64_linf"][key],
                                    "discretisation_l1": acc["discretisation_l1"].get(key),
                                    "mixed_below_discretisation_up_to": acc["mixed_below_discretisation_up_to"],
                                    "what": "relative L1 / Linf distance of the cell averages after %d CFL "
                                            "steps (t = %.4g), mixed vs FP64, beside the FP64 discretisation "
                                            "error of the grid" % (ACCURACY_STEPS, acc["t_end"])}
    if not args.no_cpu:
        from paper_2609_29081_b300 import Solver
        from paper_2609_29081_b300._native import FP64, MIXED
        w0 = W.smooth_2d(args.n)
        S = Solver.from_workload(w0, precision=MIXED if args.precision == "mixed" else FP64)
        S.set_state(w0.state)
        Lr, dt, cb = cpu_baseline(w0, S, args)
        Lg, _ = S.residual(dt)
        S.close()
        # the first SSP-RK54 stage update u + b0 dt L of the cell averages, both sides
        b0 = 0.391752226571890
        u0 = W.split_sites(w0.state, 2, *w0.n)[0]
        avg_r = u0 + b0 * dt * W.split_sites(Lr, 2, *w0.n)[0]
        avg_g = u0 + b0 * dt * W.split_sites(Lg, 2, *w0.n)[0]
        line["cpu_baseline"] = cpu_all_cores()
        line["cpu_baseline"]["host"] = host_description()
        line["cpu_baseline"]["single_core"] = cb
        line["l1_vs_oracle"] = {"what": "relative L1 / Linf distance of the first stage update u + b0 dt L(u) of "
                                        "the cell averages, GPU (%s) vs oracle, full grid" % args.precision,
                                "value": float(np.abs(avg_g - avg_r).sum() / np.abs(avg_r).sum()),
                                "linf": float(np.abs(avg_g - avg_r).max() / np.abs(avg_r).max())}
    if args.tube:
        line["tube"] = tube_measure(args, min(args.steps, 10), args.warmup)
    if args.batch:
        b = batch_measure(args, None, 0, 1, args.steps, args.warmup, args.nprob)
        line["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "workload", "cells", "tuned",
                                           "restarts", "failed", "graph", "gpu_launches", "roofline",
                                           "fp64_one_by_one", "clocks")}
    print(json.dumps(line), flush=True)


ACCURACY_STEPS = 200   # the run length of the 2D smooth periodic configuration


def accuracy_ladder(n_main, steps, grids=(32, 64, 128, 256, 512, 1024, 2048)):
    """Accuracy of the mixed path at the configuration's run length (not timed).
    t_end is the time the FP64 path reaches in `steps` CFL steps on n_main^2; on
    every grid of the ladder both paths advance to t_end (the FP64 path equals
    the oracle to 1e-10, parity tests). Reported per grid N: the discretisation
    error, relative L1 distance of the FP64 cell averages from the 2N solution
    restricted by 2x2 averaging, and the mixed path's error, relative L1 (and
    Linf) distance of its cell averages from FP64's; and the largest grid on
    which the mixed error stays below the discretisation error."""
    from paper_2609_29081_b300 import Solver, workloads as W
    from paper_2609_29081_b300._native import FP64, MIXED
    import torch
    w = W.smooth_2d(n_main)
    S = Solver.from_workload(w, precision=FP64)
    S.set_state(w.state)
    for _ in range(steps):
        S.step(0.0)
    S.get_state()
    t_end = S.t
    S.close()
    sol = {"fp64": {}, "mixed": {}}
    nsteps = {}
    t0 = time.perf_counter()
    for n in grids:
        for name, p in (("fp64", FP64), ("mixed", MIXED)):
            wn = W.smooth_2d(n)
            S = Solver.from_workload(wn, precision=p)
            S.set_state(wn.state)
            k, _ = S.advance(t_end)
            sol[name][n] = W.split_sites(S.get_state(), 2, n, n)[0]
            nsteps[n] = k
            S.close()
            torch.cuda.empty_cache()
    disc, mixed, mixed_inf = {}, {}, {}
    for n in grids:
        f = sol["fp64"][n]
        d = np.abs(sol["mixed"][n] - f)
        mixed[n] = float(d.sum() / np.abs(f).sum())
        mixed_inf[n] = float(d.max() / np.abs(f).max())
        if 2 * n in sol["fp64"]:
            g = sol["fp64"][2 * n]
            r = 0.25 * (g[:, 0::2, 0::2] + g[:, 1::2, 0::2] + g[:, 0::2, 1::2] + g[:, 1::2, 1::2])
            disc[n] = float(np.abs(f - r).sum() / np.abs(r).sum())
    below = [n for n in disc if mixed[n] < disc[n]]
    return {"t_end": t_end, "steps_at": {str(n): nsteps[n] for n in grids},
            "discretisation_l1": {str(n): v for n, v in disc.items()},
            "mixed_vs_fp64_l1": {str(n): v for n, v in mixed.items()},
            "mixed_vs_fp64_linf": {str(n): v for n, v in mixed_inf.items()},
            "mixed_below_discretisation_up_to": max(below) if below else None,
            "seconds": time.perf_counter() - t0,
            "what": "cell averages at t_end = time of %d FP64 CFL steps on %d^2; discretisation error of grid N: "
                    "relative L1 distance from the 2N solution restricted by 2x2 averaging (FP64); mixed error: "
                    "relative L1 / Linf distance of the mixed cell averages from FP64's on the same grid"
                    % (steps, n_main)}


def tile_opts(args):
    if not args.tile:
        return {}
    return {"tile_x": args.tile[0], "tile_y": args.tile[1], "threads": args.tile[2]}


def single_run(args, w, precision, dist, ws, e2e):
    """Tune, warm up and time args.steps CFL steps of workload w in one precision;
    optionally the end-to-end loop through host buffers."""
    import torch
    from paper_2609_29081_b300 import Solver
    from paper_2609_29081_b300._native import FP64, MIXED
    prec = FP64 if precision == "fp64" else MIXED
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        S = Solver.from_workload(w, precision=prec, stream=stream, **tile_opts(args))
        S.set_state(w.state)
        out["tuned"] = S.tune() if not args.tile else {"tile_x": args.tile[0], "tile_y": args.tile[1],
                                                         "threads": args.tile[2], "fixed": True}
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        cp, cpath = clocks_start()
        time.sleep(0.4)
        # warm-up right before the timed region: W steps, then more untimed steps
        # until the GPU has been busy for PREHEAT_S (clocks up after the idle sleep)
        out["warm_done"] = preheat(lambda: S.step(0.0), args.warmup)
        S.set_profiling(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        restarts = 0
        for _ in range(args.steps):
            restarts += S.step(0.0)[1]
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        out["clocks"] = clocks_stop(cp, cpath)
        ms = ev0.elapsed_time(ev1)
        prof = S.profile()
        S.set_profiling(False)
        ms = reduce_over_ranks(dist, [ms], ["max"])[0]
        out.update(ms=ms, restarts=restarts, launches=prof["launches"],
                   stage_ms=prof["stage_ms"] / max(prof["stage_launches"], 1),
                   value=w.cells * 5 * args.steps * ws / (ms / 1e3))
        if e2e:
            # end to end through the public API with pinned host buffers (FP32
            # site arrays for the mixed path, FP64 for the FP64 path)
            f32 = precision == "mixed"
            host_in = torch.from_numpy(S.get_state_f32() if f32 else S.get_state()).pin_memory()
            host_out = torch.empty_like(host_in).pin_memory()
            put, get = (S.set_state_f32, S.get_state_f32) if f32 else (S.set_state, S.get_state)
            # untimed warm-up of the loop (the first transfers into freshly pinned
            # host buffers run at half speed)
            for _ in range(max(2, args.warmup)):
                put(host_in.numpy())
                S.step(0.0)
                get(host_out.numpy())
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            # each call returns with its work done (the uploads and downloads
            # synchronise the stream, the step reads its restart flag), so host
            # time stamps between them split the step into its three parts
            parts = [0.0, 0.0, 0.0]
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                ta = time.perf_counter()
                put(host_in.numpy())
                tb = time.perf_counter()
                S.step(0.0)
                tc = time.perf_counter()
                get(host_out.numpy())
                td = time.perf_counter()
                parts[0] += tb - ta
                parts[1] += tc - tb
                parts[2] += td - tc
            torch.cuda.synchronize()
            e2e_sec = time.perf_counter() - t0
            e2e_sec = reduce_over_ranks(dist, [e2e_sec], ["max"])[0]
            out["e2e"] = w.cells * 5 * args.e2e_steps * ws / e2e_sec
            out["e2e_parts_ms"] = {k: 1e3 * v / args.e2e_steps for k, v in zip(("upload", "step", "download"), parts)}
            out["state_bytes"] = host_in.numel() * host_in.element_size()
            tuned = out["tuned"]
        S.close()
    if e2e:
        out["e2e_pipe"] = e2e_pipelined(args, w, precision, dist, ws, tuned, args.e2e_contexts)
    return out


# Contexts of the pipelined end-to-end loop: while one context computes, another
# uploads and a third downloads (the copy engines and the SMs work at once).
E2E_CONTEXTS = 4


def e2e_pipelined(args, w, precision, dist, ws, tuned, nctx):
    """End to end through the public API with nctx independent contexts, each on
    its own CUDA stream and host thread: every step of every context uploads its
    state from pinned host memory, takes one CFL step and downloads the result to
    pinned host memory (the calls block their own thread; ctypes releases the GIL).
    Returns cell-stage updates/s over all contexts, timed from a common start to
    the last context's last download."""
    import threading
    import torch
    from paper_2609_29081_b300 import Solver
    from paper_2609_29081_b300._native import FP64, MIXED
    prec = FP64 if precision == "fp64" else MIXED
    f32 = precision == "mixed"
    dev = torch.cuda.current_device()
    topts = {"tile_x": tuned["tile_x"], "tile_y": tuned["tile_y"], "threads": tuned["threads"]}
    ctxs = []
    for _ in range(nctx):
        st = torch.cuda.Stream()
        S = Solver.from_workload(w, precision=prec, stream=st, **topts)
        S.set_state(w.state)
        hin = torch.from_numpy(S.get_state_f32() if f32 else S.get_state()).pin_memory()
        ctxs.append((S, hin, torch.empty_like(hin).pin_memory()))

    def loop(k, n, start, times):
        torch.cuda.set_device(dev)
        S, hin, hout = ctxs[k]
        put, get = (S.set_state_f32, S.get_state_f32) if f32 else (S.set_state, S.get_state)
        if start is not None:
            start.wait()
        for _ in range(n):
            put(hin.numpy())
            S.step(0.0)
            get(hout.numpy())
        times[k] = time.perf_counter()

    # untimed warm-up of every context's loop, one context at a time
    scratch = [0.0] * nctx
    for k in range(nctx):
        loop(k, max(2, args.warmup), None, scratch)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    start = threading.Barrier(nctx + 1)
    ends = [0.0] * nctx
    th = [threading.Thread(target=loop, args=(k, args.e2e_steps, start, ends)) for k in range(nctx)]
    for t in th:
        t.start()
    start.wait()
    t0 = time.perf_counter()
    for t in th:
        t.join()
    sec = max(ends) - t0
    sec = reduce_over_ranks(dist, [sec], ["max"])[0]
    for S, _, _ in ctxs:
        S.close()
    return {"value": w.cells * 5 * args.e2e_steps * nctx * ws / sec, "contexts": nctx,
            "ms_per_step": 1e3 * sec / (args.e2e_steps * nctx)}


# Algorithmic work of one 2D stage per cell. Flops: counted by the op-counting
# build of the oracle on this flow (oracle/opcount_smooth2d.json, written by
# oracle/count_ops.py): every distinct evaluation of the paper's formulas once,
# trivial operations (exact 0 / +-1 operands) left out. Bytes: the minimum HBM
# traffic of a stage, 3.2 state copies per stage on average over the five
# SSP-RK54 stages, of 16 FP64 words (FP64 path) or 16 FP32 words plus 4 FP32
# compensation words of the cell averages (mixed path).
def _counted_flops():
    with open(os.path.join(ROOT, "oracle", "opcount_smooth2d.json")) as f:
        return float(json.load(f)["flops_per_cell_stage"])


FLOPS_PER_CELL_STAGE = _counted_flops()
BYTES_PER_CELL_STAGE_MIXED = 3.2 * 20 * 4
BYTES_PER_CELL_STAGE_FP64 = 3.2 * 16 * 8


if __name__ == "__main__":
    main()
