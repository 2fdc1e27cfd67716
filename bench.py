#!/usr/bin/env python
"""Benchmark of the fused D3Q27 collide-and-stream step (MLUPS, % of HBM
roofline) on one GB300, with the FP64 oracle as the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One bench step is one lattice time step of the D3Q27 Taylor-Green + noise
workload (256^3 periodic, tau = 0.6, FP32 storage): one launch of the fused
step kernel.  Inputs are larger than L2 (two 1.8 GB state buffers), so no L2
flush is needed between steps.  With N > 1 (torchrun) every rank runs the
same workload on its own GPU (independent replicas: the method is not
sharded across GPUs here) and the slowest rank's time counts.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q27 fused step MLUPS and % of HBM roofline; adjoint/forward step-time ratio"
UNIT = "MLUPS"
# algorithmic bytes per cell update: every population read once and written
# once; BF16 adds its momentum references (a float4 per pair of cells, 8 B
# written and 8 B read per cell)
BYTES_PER_CELL = {("q27", "f32"): 216, ("q27", "f16"): 108, ("q27", "bf16"): 124,
                  ("q15", "f32"): 120, ("q15", "f16"): 60, ("q15", "bf16"): 76}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth (a copy reaches ~86 % of it)
KERNEL_SOURCES = ["lattice.cuh", "vec2.cuh", "collide_q27.cuh", "kernels.cuh"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=256, help="cube edge of the main workload")
    p.add_argument("--quick", action="store_true",
                   help="main measurement only (no e2e, sweeps, 16-bit or CPU baseline)")
    p.add_argument("--lattice", type=int, choices=[27, 15], default=27,
                   help="lattice of the main measurement (profiling runs)")
    p.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32",
                   help="storage of the main measurement (profiling runs)")
    p.add_argument("--inplace", action="store_true",
                   help="time the single-buffer in-place (AA) scheme as the main line")
    p.add_argument("--adjoint-only", action="store_true",
                   help="time only the adjoint workload at --size (profiling runs)")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for n in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1202_6081_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(size):
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, scaled to the workload's cells; None if the kernel changed."""
    path = os.path.join(ROOT, "profiles", "step_q27_f32_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d["dram_bytes_per_cell"] * size**3


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, maximum SM clock and the throttle reasons seen
        active, from the sampler's CSV lines (FIELDS order); None if no line
        parses."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(size, budget_s=15.0):
    """The FP64 oracle on this host's cores, on a bounded sample of the same
    workload: z-slabs of the size^3 Taylor-Green + noise field (periodic),
    stepped until about budget_s of CPU work has run."""
    import oracle
    import workloads as W
    oracle.build()
    Q = 27
    om = W.omegas(Q, 1 / 0.6)
    nz_s = 1
    shape = (nz_s, size, size)
    rho, u = W.taylor_green((size, size, size), u0=0.02, noise=1e-3)
    f = oracle.equilibrium(Q, rho[:nz_s], u[:, :nz_s], np.zeros(3))
    cores = oracle.max_threads()
    cells = size * size * nz_s

    def timed(nthreads, budget):
        t0 = time.perf_counter()
        oracle.run(Q, shape, f, np.zeros(3), om, 1, nthreads=nthreads)
        one = time.perf_counter() - t0
        steps = max(1, int(budget / max(one, 1e-3)))
        t0 = time.perf_counter()
        oracle.run(Q, shape, f, np.zeros(3), om, steps, nthreads=nthreads)
        return steps, time.perf_counter() - t0

    steps, dt = timed(cores, budget_s)
    steps1, dt1 = timed(1, budget_s / 3)
    oracle.run(Q, shape, f, np.zeros(3), om, 0, nthreads=cores)  # restore the thread count
    # the small configurations, all cores: 32^3 Taylor-Green x 100 steps in
    # full, and the first 100 steps of the 16 x 64 x 64 channel
    small = {}
    for name, Qs, shp, om_s, F, bc, n in (
            ("D3Q27 32^3 Taylor-Green, 100 steps", 27, (32, 32, 32), W.omegas(27, 1 / 0.6),
             np.zeros(3), 0, 100),
            ("D3Q15 16x64x64 channel, first 100 steps", 15, (64, 64, 16), W.omegas(15, 1 / 0.8),
             np.array([1e-6, 0.0, 0.0]), 3, 100),
            ("D3Q27 16x64x64 channel, first 100 steps", 27, (64, 64, 16), W.omegas(27, 1 / 0.8),
             np.array([1e-6, 0.0, 0.0]), 3, 100)):
        r0, u0 = W.taylor_green(shp, u0=0.02) if bc == 0 else (np.ones(shp),
                                                             np.zeros((3,) + shp))
        f0 = oracle.equilibrium(Qs, r0, u0, F)
        t0 = time.perf_counter()
        oracle.run(Qs, shp, f0, F, om_s, n, bc=bc, nthreads=cores)
        t = time.perf_counter() - t0
        small[name] = {"value": int(np.prod(shp)) * n / t / 1e6, "unit": UNIT,
                       "seconds": t}
    return {"value": cells * steps / dt / 1e6, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "%d steps of one %dx%dx%d z-slab of the %d^3 Taylor-Green+noise field "
                      "(periodic), D3Q27, tau=0.6, FP64, %.1f s" % (steps, size, size, nz_s,
                                                                   size, dt),
            "single_thread": {"value": cells * steps1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": "%d steps of the same slab, %.1f s" % (steps1, dt1)},
            "small_configs": small}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import workloads as W
    oracle.build()
    Q = 27
    size = args.size
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green((size, size, size), u0=0.02, noise=1e-3)
    # each reference step: one oracle step on a z-slab of the workload, the
    # slab sized so that warmup + steps end within about two minutes
    probe = (1, size, size)
    f1 = oracle.equilibrium(Q, rho[:1], u[:, :1], np.zeros(3))
    t0 = time.perf_counter()
    oracle.run(Q, probe, f1, np.zeros(3), om, 1)
    per_plane = time.perf_counter() - t0
    total_steps = args.steps + args.warmup
    budget = 120.0
    planes = max(1, min(size, int(budget / max(total_steps * per_plane, 1e-9))))
    cells_side = size
    if planes == 1 and total_steps * per_plane > budget:
        # shrink the slab's rows too
        frac = budget / (total_steps * per_plane)
        cells_side = max(8, int(size * frac))
    shape = (planes, cells_side, size)
    f = oracle.equilibrium(Q, rho[:planes, :cells_side], u[:, :planes, :cells_side],
                           np.zeros(3))
    for _ in range(args.warmup):
        f = oracle.run(Q, shape, f, np.zeros(3), om, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle.run(Q, shape, f, np.zeros(3), om, 1)
    dt = time.perf_counter() - t0
    cells = planes * cells_side * size
    value = cells * args.steps / dt / 1e6
    sample = ("each step: one oracle step on a %dx%dx%d slab of the %d^3 Taylor-Green+noise "
              "field (periodic), D3Q27, tau=0.6, FP64" % (size, cells_side, planes, size))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "D3Q27 Taylor-Green+noise %d^3 periodic, tau=0.6" % size,
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def make_solver(lbm, Q, size, storage, tau, inplace=False):
    import workloads as W
    shape = (size, size, size)
    om = W.omegas(Q, 1 / tau)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    S = lbm.Solver(Q, shape, om, storage=storage, inplace=inplace)
    S.init_equilibrium(rho, u)
    return S, rho, u


def time_steps(torch, S, steps, warmup, barrier=None):
    stream = torch.cuda.current_stream()
    S.step(warmup)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    S.step(steps)
    end.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return start.elapsed_time(end) / 1e3


def e2e_job(torch, lbm, size, steps):
    """Whole job through the public API from pinned host buffers: rho, u
    (FP64) in pinned host memory go to lbm_init_equilibrium, whose kernel
    reads them across the host link (no separate copy), `steps` steps, and
    lbm_macroscopic writes rho, u (FP32) straight into pinned host memory."""
    import workloads as W
    Q = 27
    shape = (size, size, size)
    N = size**3
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    h_rho = torch.from_numpy(rho).pin_memory()
    h_u = torch.from_numpy(u).pin_memory()
    o_rho = torch.empty(shape, dtype=torch.float32).pin_memory()
    o_u = torch.empty((3,) + shape, dtype=torch.float32).pin_memory()
    S = lbm.Solver(Q, shape, om)
    stream = torch.cuda.current_stream()

    def job():
        lbm.lbm_init_equilibrium(S.ctx, h_rho, h_u)  # kernel reads pinned host memory
        lbm.lbm_step(S.ctx, steps)
        lbm.lbm_macroscopic(S.ctx, o_rho, o_u)       # kernel writes pinned host memory
        stream.synchronize()

    job()  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    job()
    dt = time.perf_counter() - t0
    h2d = (8 + 24) * N
    d2h = (4 + 12) * N
    return {"value": N * steps / dt / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "job": "rho,u (FP64) read by the init kernel from pinned host memory + %d steps + "
                   "rho,u (FP32) written by the macroscopic kernel to pinned host memory" % steps}


def adjoint_timing(torch, lbm, size, steps=100, Q=27):
    """Adjoint step vs forward step at the adjoint workload (D3Q27 or D3Q15,
    size^3 periodic, tau = 0.6, per-cell force field), both by CUDA events;
    plus a whole checkpointed gradient (200 steps, checkpoint every 20).
    Algorithmic bytes of an adjoint step per cell: f_t, lam_{t+1} read and
    lam_t written (3 Q x 4 B), the force field read and dJ/dF read and
    written (36 B)."""
    import workloads as W
    from paper_1202_6081_gb300.autograd import kinetic_energy_after
    shape = (size, size, size)
    om = W.omegas(Q, 1 / 0.6)
    rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
    F = torch.as_tensor(W.gaussian_force_field(shape, rms=1e-5, sigma=4.0).astype(np.float32),
                        device="cuda").contiguous()
    S = lbm.Solver(Q, shape, om)
    S.set_force_field(F)
    S.init_equilibrium(rho, u)
    t_fwd = time_steps(torch, S, steps, 5) / steps
    f_t = S.current_buffer()
    lam = [S.new_adjoint_field(), S.new_adjoint_field()]
    gF = torch.zeros_like(F)
    stream = torch.cuda.current_stream()
    for i in range(5):
        S.adjoint_step(f_t, lam[i % 2], lam[1 - i % 2], gF)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        S.adjoint_step(f_t, lam[i % 2], lam[1 - i % 2], gF)
    e1.record(stream)
    torch.cuda.synchronize()
    t_adj = e0.elapsed_time(e1) / 1e3 / steps
    cells = size**3
    # whole gradient: forward with checkpoints, then backward (recompute + adjoint);
    # one untimed gradient first so the ring and checkpoint buffers are in
    # torch's allocator cache
    Fg = F.clone().requires_grad_()
    init = S.current_buffer().clone()
    S.load_buffer(init)
    kinetic_energy_after(S, Fg, 200, 20).backward()
    Fg.grad = None
    S.load_buffer(init)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J = kinetic_energy_after(S, Fg, 200, 20)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"workload": "D3Q%d %d^3 periodic, tau=0.6, force field, FP32" % (Q, size),
            "forward_ms_per_step": t_fwd * 1e3, "adjoint_ms_per_step": t_adj * 1e3,
            "adjoint_forward_ratio": t_adj / t_fwd,
            "adjoint_GB/s": (12 * Q + 36) * cells / t_adj / 1e9,
            "gradient_200_steps": {"forward_s": t1 - t0, "backward_s": t2 - t1,
                                   "backward_forward_ratio": (t2 - t1) / (t1 - t0)}}


def small_grids(torch, lbm, steps=4000):
    """Small grids are bound by launch cost: D3Q27 FP32 MLUPS with every step
    launched on its own and with runs of 32 steps launched as CUDA graphs."""
    import workloads as W
    out = {}
    om = W.omegas(27, 1 / 0.6)
    for name, shape, walls in (("32^3 periodic", (32, 32, 32), 0),
                               ("16x64x64 channel", (64, 64, 16), 3),
                               ("64^3 periodic", (64, 64, 64), 0),
                               ("128^3 periodic", (128, 128, 128), 0)):
        rho, u = W.taylor_green(shape, u0=0.02, noise=1e-3)
        row = {}
        for gs in (0, 32):
            S = lbm.Solver(27, shape, om, walls=walls)
            S.set_graph_steps(gs)
            S.init_equilibrium(rho, u)
            t = time_steps(torch, S, steps, 64)
            row["graphs" if gs else "single_launches"] = int(np.prod(shape)) * steps / t / 1e6
            del S
        out[name] = row
    return out


def max_over_ranks(torch, value, device):
    """The largest value over the ranks of the default process group (the
    slowest rank's time).  Timing only: no simulation data is exchanged."""
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells, steps, elapsed):
    """Cell updates of all ranks (independent replicas of the same workload)
    per second of the slowest rank, in millions."""
    return world * cells * steps / elapsed / 1e6


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    barrier = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        barrier = dist.barrier

    from paper_1202_6081_gb300 import build, lbm
    build()
    size = args.size
    if args.adjoint_only:
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_timing(torch, lbm, size, steps=args.steps,
                                                        Q=args.lattice)}), flush=True)
        return 0
    lat, st = args.lattice, args.storage
    S, _, _ = make_solver(lbm, lat, size, st, 0.6, inplace=args.inplace)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    elapsed = time_steps(torch, S, args.steps, args.warmup, barrier)
    clocks = sampler.stop() if sampler else None
    cons = S.conservation()
    if world > 1:
        elapsed = max_over_ranks(torch, elapsed, "cuda")
    cells = size**3
    value = whole_job_mlups(world, cells, args.steps, elapsed)
    peaks, peak_kind = measured_peaks()
    per_launch = elapsed / args.steps
    bpc = BYTES_PER_CELL.get(("q%d" % lat, st), (4 if st == "f32" else 2) * 2 * lat)
    alg_bytes = bpc * cells
    achieved = alg_bytes / per_launch / 1e9
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_launch * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "D3Q%d Taylor-Green+noise %d^3 periodic, tau=0.6, %s storage "
                               "of f-w%s" % (lat, size, st.upper(),
                                             ", in-place (AA) streaming" if args.inplace else ""),
                   "cells": cells, "l2": "no flush: inputs larger than L2 (%s%.1f GB state)"
                   % ("" if args.inplace else "2 x ", alg_bytes / 2 / 1e9),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": ncu_traffic(size) if (lat, st, args.inplace) == (27, "f32", False)
                     else None,
                     "peak_source": "%s hbm_gbs: the bandwidth of a plain device copy "
                                    "(frac is achieved / measured copy, not of the data sheet), "
                                    "%d B/cell algorithmic" % (peak_kind, bpc),
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "conservation": {"mass": cons[0], "momentum": list(cons[1:])},
    }
    del S
    torch.cuda.empty_cache()
    if rank == 0 and not args.quick:
        result["e2e"] = e2e_job(torch, lbm, size, args.steps)
        torch.cuda.empty_cache()
        sweep = {}
        for tau in (0.51, 0.6, 1.0):
            S, _, _ = make_solver(lbm, 27, size, "f32", tau)
            t = time_steps(torch, S, 200, 5)
            sweep["%g" % tau] = cells * 200 / t / 1e6
            del S
        result["tau_sweep_mlups"] = sweep
        torch.cuda.empty_cache()
        s16 = {}
        big = 512
        for st in ("f32", "f16", "bf16"):
            S, _, _ = make_solver(lbm, 27, big, st, 0.6)
            t = time_steps(torch, S, 100, 5)
            mlups = big**3 * 100 / t / 1e6
            bpc = BYTES_PER_CELL[("q27", st)]
            s16[st] = {"mlups": mlups, "GB/s": bpc * big**3 * 100 / t / 1e9,
                       "frac": bpc * big**3 * 100 / t / 1e9 / peak}
            del S
            torch.cuda.empty_cache()
        result["storage_512"] = s16
        q15 = {}
        for st in ("f32", "f16", "bf16"):
            S, _, _ = make_solver(lbm, 15, size, st, 0.6)
            t = time_steps(torch, S, 200, 5)
            bpc = BYTES_PER_CELL[("q15", st)]
            q15[st] = {"mlups": cells * 200 / t / 1e6, "GB/s": bpc * cells * 200 / t / 1e9,
                       "frac": bpc * cells * 200 / t / 1e9 / peak}
            del S
            torch.cuda.empty_cache()
        result["d3q15_%d" % size] = q15
        aa = {}
        for n, st in ((size, "f32"), (512, "f32"), (512, "f16")):
            S, _, _ = make_solver(lbm, 27, n, st, 0.6, inplace=True)
            t = time_steps(torch, S, 200 if n == size else 100, 6)
            k = 200 if n == size else 100
            bpc = BYTES_PER_CELL[("q27", st)]
            aa["%d_%s" % (n, st)] = {"mlups": n**3 * k / t / 1e6,
                                      "GB/s": bpc * n**3 * k / t / 1e9,
                                      "frac": bpc * n**3 * k / t / 1e9 / peak,
                                      "state_GB": bpc / 2 * n**3 / 1e9}
            del S
            torch.cuda.empty_cache()
        result["inplace_aa"] = aa
        result["small_grids"] = small_grids(torch, lbm)
        result["adjoint"] = adjoint_timing(torch, lbm, 128)
        result["adjoint_q15"] = adjoint_timing(torch, lbm, 128, Q=15)
        torch.cuda.empty_cache()
        result["cpu_baseline"] = cpu_baseline(size)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        try:
            return run_reference(args)
        except Exception as e:  # the oracle could not be built or run here
            if dist_env()[0] == 0:
                print(json.dumps({"impl": "reference",
                                  "unavailable": "FP64 oracle failed: %s" % str(e)[:200]}),
                      flush=True)
            return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
