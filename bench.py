"""Benchmark of the WENO-theta hot path on GB300.

Headline workload: the batched 1D Euler configuration, the largest that runs on one GPU.
4096 independent problems (gamma = 1.4), lengths N log-uniform in [256, 65536] (47.3 M cells
for seed 0), each on [-5, 5] with periodic or outflow boundaries (coin flip), seeded Riemann +
entropy-wave data, its own CFL 0.5 step and Lax-Friedrichs constants, 200 TVD-RK3 steps in
FP64, advanced through weno_theta_step_batched (one launch of the fused RHS + RK stage kernel
per RK stage over all problems, replayed from a CUDA graph).

One benchmark step = RK_PER_STEP (10) RK3 steps of the whole batch through one
weno_theta_step_batched call; 20 steps are the workload's 200 RK steps, timed from the initial
data (the warm-up steps run on a copy first).  value = cell-updates/s, one cell-update being
one cell advanced by a full RK3 step (three RHS evaluations).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its LPT share of the first N x 4096 problems of the same
seeded stream (weak scaling: about 4096 problems' cells per GPU, no data exchange); rank 0
prints one JSON line.  --impl reference times the CPU oracle (the plain reference
implementation of the method, OpenMP over problems) on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1504_00731_gb300 import distributed as D  # noqa: E402
from paper_1504_00731_gb300 import workloads as W  # noqa: E402

METRIC = "FP64 cell-updates/s per GB300 and % HBM roofline; batched & adjoint vs plain"
NPROB = 4096
CFL = 0.5
M = 3
RK_STEPS = 200            # RK steps of the workload
RK_PER_STEP = 10          # RK steps per benchmark step
WORKLOAD = "euler1d_batch4096_N-loguniform-256-65536_periodic-or-outflow_riemann-entropy_cfl0.5_200rk3"
# Arithmetic of one cell-update (one cell, one RK3 step) of 1D Euler, counted by the oracle's
# operation-counting instantiation (tests/test_flop_count.py keeps it honest): +, -, *, / and
# sqrt each count one flop.  It is the method's literal arithmetic; the fast policy executes
# fewer FP64 operations (FMA, closed-form restricted stencils, restriction and theta decided in
# FP32 where an error bound proves them), so a fraction by this count can pass 1 where the GPU
# is full.  frac_pipe (ncu) is the FP64 pipe's occupancy, which cannot.
FLOPS_PER_CELL_UPDATE = 3696.0
FLOPS_PER_CELL_UPDATE_2D = 10449.0
# Algorithmic memory bytes of one cell-update through the stage kernels: stage 1 reads u^n and
# writes u^(1), stage 2 reads u^(1) and u^n and writes u^(2), stage 3 reads u^(2) and u^n and
# writes u^(n+1): 8 m doubles = 64 m bytes per RK step (a third of it per launch, on average).
BYTES_PER_CELL_UPDATE_STAGES = 64.0 * M
# FP64 peak from unit counts: 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x 2.07 GHz
# (a microbenchmark reaches 94.7% of it: profiles/fp64_pipe_microbenchmark.md).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
FLOPS_NOTE = ("algorithmic flops: the oracle's count of the method's literal FP64 arithmetic; the fast policy "
              "executes fewer FP64 operations (FMA, closed-form restricted stencils, restriction and theta "
              "decided in FP32 where an error bound proves them), so this fraction can exceed 1; frac_pipe is "
              "the FP64 pipe's active share of elapsed cycles (ncu)")
L2_FLUSH_BYTES = 256 << 20
KERNEL_SOURCES = ("wt_kernels.cuh", "wt_math_fast.cuh", "wt_device.cuh", "wt_kernels_fast.cu", "wt_launch.h")
COUNTERS = {
    "batched": os.path.join(ROOT, "profiles", "stage1d_batched_euler_counters.json"),
    "stepblock": os.path.join(ROOT, "profiles", "stepblock1d_euler_N4096_counters.json"),
    "stage2d": os.path.join(ROOT, "profiles", "stage2d_euler_counters.json"),
    "adjoint": os.path.join(ROOT, "profiles", "adj_stage_euler_counters.json"),
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_hash(sources=KERNEL_SOURCES):
    """Hash of the kernel sources' code: comments and blank lines removed, so that a change to a
    comment does not retire counters taken on the same code (no string literal in these files
    holds a comment marker)."""
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1504_00731_gb300", "csrc", name)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def counters(kind):
    """ncu figures of a kernel from the committed summary, if the kernel sources are unchanged
    since they were taken; else None."""
    try:
        with open(COUNTERS[kind]) as f:
            c = json.load(f)
    except OSError:
        return None
    srcs = tuple(c.get("sources", KERNEL_SOURCES))
    if c.get("kernel_sha") != kernel_hash(srcs):
        return None
    return c


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_info():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "lscpu_model": model}


def config_dict(world):
    return {"workload": WORKLOAD, "problems_per_gpu": NPROB, "problems": NPROB * world, "n_min": 256,
            "n_max": 65536, "rk_steps": RK_STEPS, "rk_steps_per_step": RK_PER_STEP, "m": M, "cfl": CFL,
            "bc": "periodic or outflow per problem", "mode": "fast", "alpha_R": W.ALPHA_R_SEEDED, "eps": 1e-10,
            "seed": 0,
            "timed": "K benchmark steps = K x 10 RK steps from the initial data (K = 20: the whole 200-step run)",
            "l2": "inputs larger than L2 (1.13 GB of state per GPU against a 129 MB L2)",
            "parallelism": (f"LPT split of the first {world} x {NPROB} problems of the seed-0 stream over {world} "
                            "GPUs, no data exchange" if world > 1 else "one GPU")}


def stride_sample(lengths, every):
    """Every `every`-th problem in length order: a sample with the batch's length mix."""
    order = np.argsort(lengths, kind="stable")
    return np.sort(order[::every])


def cpu_baseline():
    """The oracle's CPU baseline, measured in a process of its own (no CUDA context or torch
    threads beside it), as cpu_baseline_here() reports it."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only"], capture_output=True,
                       text=True, timeout=900, cwd=ROOT)
    if r.returncode != 0:
        return {"value": None, "unit": "cell-updates/s", "cores": None, "kind": "oracle",
                "sample": "failed: " + (r.stderr.strip().splitlines() or ["?"])[-1]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_here(serial_every=32, serial_steps=8, par_every=4, par_steps=4):
    """The oracle, as it stands, on seeded samples of the same workload (every k-th problem in
    length order, so the sample keeps the batch's length mix): one core, and OpenMP over the
    problems on every core (the per-problem arithmetic is the same)."""
    import oracle as O

    O.lib()
    lengths = W.batch_lengths(NPROB, seed=0)
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    out = {}
    for name, every, steps, threads in (("serial", serial_every, serial_steps, 1),
                                        ("all_cores", par_every, par_steps, 0)):
        ids = stride_sample(lengths, every)
        b = W.euler_batch(NPROB, seed=0, problems=ids)
        t0 = time.perf_counter()
        O.run_batch(P, b.u, b.offsets, b.lengths, b.lo, b.hi, b.bc, cfl=CFL, n_steps=steps, threads=threads)
        el = time.perf_counter() - t0
        cells = int(b.lengths.sum())
        out[name] = {"value": cells * steps / el, "cores": 1 if threads == 1 else O.max_threads(), "seconds": el,
                     "sample": f"{len(ids)} of the {NPROB} problems (every {every}th by length, {cells} cells), "
                               f"{steps} RK3 steps from the initial data"}
    par = out["all_cores"]
    return {"value": par["value"], "unit": "cell-updates/s", "cores": par["cores"], "kind": "oracle",
            "sample": "all cores: " + par["sample"] + "; serial: " + out["serial"]["sample"],
            "serial": out["serial"], "all_cores": par, **host_info(), "openmp": O.openmp(),
            "build": "g++ -O2 -ffp-contract=off -fopenmp (OpenMP over independent problems)"}


# ---------------------------------------------------------------------------------------------
# Extra measurements (one GPU): the single-problem workload, 2D, adjoint, per-problem launches
# ---------------------------------------------------------------------------------------------

def segments(B, batch):
    segs = []
    for p in range(len(batch.lengths)):
        s = B.WtSegment()
        s.offset, s.n = int(batch.offsets[p]), int(batch.lengths[p])
        s.lo, s.hi = float(batch.lo[p]), float(batch.hi[p])
        s.bc_lo = s.bc_hi = int(batch.bc[p])
        segs.append(s)
    return segs


def pipe_block(kind, achieved_cell_updates_s, flops_per_cu):
    c = counters(kind)
    if c is None:
        return {"frac_pipe": None, "note": "no ncu counters for the current kernel sources"}
    out = {"frac_pipe": c["fp64_pipe_active_pct"] / 100.0,
           "fp64_pipe_source": c["source"],
           "fp64_thread_ops_per_cell_update": c.get("fp64_thread_ops_per_cell_update"),
           "fp64_warp_inst_per_cell_update": c.get("fp64_warp_inst_per_cell_update"),
           "method_flops_per_cell_update": flops_per_cu}
    if c.get("fp64_flops_per_cell_update"):
        ex = achieved_cell_updates_s * c["fp64_flops_per_cell_update"] / 1e9
        out["executed_fp64_gflops"] = ex
        out["frac_executed"] = ex / FP64_PEAK_GFLOPS
    return out


def single_problem_measure(B, dev, runs=10):
    """The single-problem 1D Euler workload (N = 4096 on [-5, 5], outflow, seeded Riemann +
    entropy wave, CFL 0.5, 2000 RK steps): one cooperative launch of the step-blocked kernel per
    run, L2 flushed between runs; e2e through host buffers."""
    import torch

    n, steps = 4096, 2000
    U0, x, dx = W.euler_c2(n, seed=0)
    prob = B.problem(B.WT_FLUX_EULER1D, bc=B.WT_BC_OUTFLOW, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    grid = B.grid_1d(n, -5.0, 5.0)
    ws = B.alloc_workspace(B.workspace_bytes(prob, grid), dev)
    src = torch.from_numpy(U0).to(dev)
    u = torch.empty_like(src)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(runs)]
    for _ in range(3):
        u.copy_(src)
        B.weno_theta_step(prob, grid, u, CFL, ws, max_steps=steps)
    tot, tot0 = 0.0, 0.0
    for maxs in (steps, 0):
        for k in range(runs):
            u.copy_(src)
            flush.zero_()
            ev[k][0].record(stream)
            B.weno_theta_step(prob, grid, u, CFL, ws, max_steps=maxs)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        s = sum(a.elapsed_time(b) for a, b in ev)
        if maxs:
            tot = s
        else:
            tot0 = s
    ms = tot / runs
    kernel_ms = (tot - tot0) / runs
    h = torch.from_numpy(U0.copy()).pin_memory()
    e2e = []
    for _ in range(3):
        hu = h.clone().pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.weno_theta_step(prob, grid, hu.numpy(), CFL, ws, max_steps=steps, stream=stream.cuda_stream)
        e2e.append(time.perf_counter() - t0)
    v = n * steps / (ms * 1e-3)
    ach = FLOPS_PER_CELL_UPDATE * n * steps / (kernel_ms * 1e-3) / 1e9
    return {"value": v, "unit": "cell-updates/s", "ms_per_run": ms, "kernel_ms": kernel_ms,
            "e2e_value": n * steps / float(np.mean(e2e)),
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": ach / FP64_PEAK_GFLOPS,
                         "kernel": "stepblock1d_kernel<FastMath, Euler1D, 27> (one cooperative launch per run)",
                         **pipe_block("stepblock", n * steps / (kernel_ms * 1e-3), FLOPS_PER_CELL_UPDATE)},
            "workload": "euler1d_riemann_entropy_N4096_outflow_cfl0.5_2000rk3 (seed 0)"}


def plain_vs_batched(B, dev, batch, steps=20):
    """Every problem of the batch through weno_theta_step one at a time (the per-problem
    launches the batched path replaces), `steps` RK steps each, with the automatic launch choice
    and with per-stage launches of the fused stage kernel; CUDA-event time around each call."""
    import torch

    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0 = torch.from_numpy(batch.u).to(dev)
    nmax = int(batch.lengths.max())
    out = {}
    for name, launch in (("plain_auto", B.WT_LAUNCH_AUTO), ("plain_stages", B.WT_LAUNCH_STAGES)):
        pmax = B.problem(B.WT_FLUX_EULER1D, bc=B.WT_BC_OUTFLOW, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED,
                         launch=launch)
        ws = B.alloc_workspace(B.workspace_bytes(pmax, B.grid_1d(nmax, -5.0, 5.0)), dev)
        tot_ms, cells = 0.0, 0
        per = np.zeros(len(batch.lengths))
        for p in range(len(batch.lengths)):
            o, n = int(batch.offsets[p]), int(batch.lengths[p])
            pb = B.problem(B.WT_FLUX_EULER1D, bc=int(batch.bc[p]), mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED,
                           launch=launch)
            g = B.grid_1d(n, -5.0, 5.0)
            us = u0[:, o:o + n].contiguous()
            if p < 8:  # graphs and kernels warm for the first sizes
                B.weno_theta_step(pb, g, us, CFL, ws, max_steps=1)
            e0.record(stream)
            B.weno_theta_step(pb, g, us, CFL, ws, max_steps=steps)
            e1.record(stream)
            e1.synchronize()
            per[p] = e0.elapsed_time(e1) * 1e-3
            tot_ms += per[p] * 1e3
            cells += n
        out[name] = {"value": cells * steps / (tot_ms * 1e-3), "seconds": tot_ms * 1e-3}
        # where the per-problem time goes, by problem length
        groups = []
        for lo_n, hi_n in ((0, 2048), (2048, 16384), (16384, 1 << 30)):
            sel = (batch.lengths >= lo_n) & (batch.lengths < hi_n)
            c, t = int(batch.lengths[sel].sum()), float(per[sel].sum())
            groups.append({"n_range": [lo_n, min(hi_n, 65536)], "problems": int(sel.sum()),
                           "cells_share": c / cells, "time_share": t / (tot_ms * 1e-3),
                           "rate": c * steps / t if t > 0 else None})
        out[name]["by_length"] = groups
        del ws
    return out


def euler2d_measure(B, dev, steps=5):
    """2D Euler, 4096 x 4096 periodic vortex / quadrant state, CFL 0.45, timed over `steps` RK
    steps of the 500-step workload (throughput per step does not depend on the count)."""
    import torch

    n = 4096
    U, dx, dy = W.euler2d_vortices(n, n, seed=0)
    prob = B.problem(B.WT_FLUX_EULER2D, bc=B.WT_BC_PERIODIC, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    g = B.grid_2d(n, n)
    ws = B.alloc_workspace(B.workspace_bytes(prob, g), dev)
    u0 = torch.from_numpy(U).to(dev)
    u = u0.clone()
    B.weno_theta_step(prob, g, u, 0.45, ws, max_steps=1)
    u.copy_(u0)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    B.weno_theta_step(prob, g, u, 0.45, ws, max_steps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    v = n * n * steps / t
    ach = v * FLOPS_PER_CELL_UPDATE_2D / 1e9
    return {"value": v, "unit": "cell-updates/s", "cells": n * n, "rk_steps_timed": steps,
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": ach / FP64_PEAK_GFLOPS, "kernel": "stage2d_kernel<FastMath, *>",
                         **pipe_block("stage2d", v, FLOPS_PER_CELL_UPDATE_2D)},
            "workload": "2D Euler 4096^2 periodic, 4 quadrants + 8 isentropic vortices, CFL 0.45"}


def adjoint_measure(B, dev, nprob=256, n=16384, steps=64, K=32, K_full=2):
    """Discrete adjoint of nprob x n 1D Euler cells through `steps` RK steps with checkpoints every
    K, against one plain forward run of the same problems through the batched entry point.
    The adjoint workload runs 1024 steps with checkpoints every 32: 32 segments, of which the
    forward pass records the last and the reverse sweep recomputes the other 31.  `steps`
    with checkpoints every K_full (64 / 2 = 32 segments) recomputes the same share and gives
    that workload's ratio; `steps` with K (2 segments) recomputes half."""
    import torch

    U0 = np.empty((nprob, 3, n))
    for p in range(nprob):
        U0[p] = W.euler_riemann(n, W.riemann_params(p))[0]
    prob = B.problem(B.WT_FLUX_EULER1D, bc=B.WT_BC_OUTFLOW, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    g = B.grid_1d(n, -5.0, 5.0)
    ws = B.alloc_workspace(max(B.adjoint_workspace_bytes(prob, g, nprob, steps, K),
                               B.adjoint_workspace_bytes(prob, g, nprob, steps, K_full)), dev)
    u0 = torch.from_numpy(U0).to(dev)
    uT, gT, g0 = torch.empty_like(u0), torch.zeros_like(u0), torch.empty_like(u0)
    gT[:, 0, :] = 1e-3
    B.weno_theta_adjoint(prob, g, nprob, u0, 0.5, 2, 2, gT, g0, ws, uT=uT)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_adj = {}
    for k in (K, K_full):
        torch.cuda.synchronize()
        e0.record(stream)
        B.weno_theta_adjoint(prob, g, nprob, u0, 0.5, steps, k, gT, g0, ws, uT=uT)
        e1.record(stream)
        torch.cuda.synchronize()
        t_adj[k] = e0.elapsed_time(e1) * 1e-3
    del ws
    segs = []
    for p in range(nprob):
        s = B.WtSegment()
        s.offset, s.n, s.lo, s.hi, s.bc_lo, s.bc_hi = p * n, n, -5.0, 5.0, 1, 1
        segs.append(s)
    wsb = B.alloc_workspace(B.workspace_bytes(prob, None, nprob * n, nprob), dev)
    packed = u0.permute(1, 0, 2).reshape(3, nprob * n).contiguous()
    u = packed.clone()
    B.weno_theta_step_batched(prob, segs, u, nprob * n, 0.5, 2, wsb)
    u = packed.clone()
    torch.cuda.synchronize()
    e0.record(stream)
    B.weno_theta_step_batched(prob, segs, u, nprob * n, 0.5, steps, wsb)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) * 1e-3
    seg_full = (steps + K_full - 1) // K_full
    return {"adjoint_over_forward": t_adj[K_full] / t_fwd, "adjoint_s": t_adj[K_full], "forward_s": t_fwd,
            "recomputed_share": f"{seg_full - 1} of {seg_full} segments (checkpoints every {K_full} of {steps} "
                                f"steps), as in 1024 steps with checkpoints every 32",
            "adjoint_over_forward_two_segments": t_adj[K] / t_fwd, "adjoint_s_two_segments": t_adj[K],
            "problems": nprob, "n": n, "rk_steps": steps, "checkpoint_every": K_full,
            "grad_finite": bool(torch.isfinite(g0).all()),
            "workload": "256 x 1D Euler N=16384 (seeded Riemann + entropy wave), outflow, CFL 0.5"}


def problems_measure(B, dev):
    """The small scalar workload (linear advection of sin(pi x), N = 200, periodic, CFL 0.4 to
    t = 2: 500 steps; latency-bound) and the test problems of Sec. 4.2 / 4.3 built on
    reflective walls and gravity: two interacting blast waves (TEST 5, N = 801, alpha_R = 10,
    the paper's run to t = 0.038), the Rayleigh-Taylor instability (TEST 6, 120 x 360,
    gravity 0.1, 2000 of the ~17600 steps to t = 9.5) and the implosion problem (TEST 7,
    400 x 400, alpha_R = 1, 1000 of the ~16200 steps to t = 5); fast mode, CFL 0.5 unless
    stated, cell-updates/s through weno_theta_step."""
    import torch

    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    cases = []
    U, x, dx = W.advection_sine(200)
    cases.append(("advection_sine_N200_cfl0.4_t2", U, B.problem(B.WT_FLUX_ADVECTION, bc=B.WT_BC_PERIODIC,
                                                                mode=B.WT_MODE_FAST), B.grid_1d(200, -1.0, 1.0),
                  dict(t_final=2.0, cfl=0.4)))
    U, x, dx = W.blast_waves(801)
    cases.append(("blast_waves_N801_t0.038", U, B.problem(B.WT_FLUX_EULER1D, bc=B.WT_BC_REFLECTIVE, mode=B.WT_MODE_FAST,
                                                          alpha_R=10.0), B.grid_1d(801, 0.0, 1.0),
                  dict(t_final=0.038)))
    U, dx, dy = W.rayleigh_taylor(120, 360)
    cases.append(("rayleigh_taylor_120x360_2000steps", U,
                  B.problem(B.WT_FLUX_EULER2D, bc=B.WT_BC_PERIODIC, bc_y=B.WT_BC_REFLECTIVE, mode=B.WT_MODE_FAST,
                            gravity=W.RT_GRAVITY), B.grid_2d(120, 360, (-0.25, -0.75), (0.25, 0.75)),
                  dict(max_steps=2000)))
    U, dx, dy = W.implosion(400)
    cases.append(("implosion_400x400_1000steps", U,
                  B.problem(B.WT_FLUX_EULER2D, bc=B.WT_BC_REFLECTIVE, bc_y=B.WT_BC_REFLECTIVE, mode=B.WT_MODE_FAST,
                            alpha_R=1.0), B.grid_2d(400, 400), dict(max_steps=1000)))
    for name, U, prob, grid, kw in cases:
        kw = dict(kw)
        cfl = kw.pop("cfl", 0.5)
        ws = B.alloc_workspace(B.workspace_bytes(prob, grid), dev)
        u0 = torch.from_numpy(np.ascontiguousarray(U)).to(dev)
        u = u0.clone()
        B.weno_theta_step(prob, grid, u, cfl, ws, max_steps=3)
        u.copy_(u0)
        torch.cuda.synchronize()
        e0.record(stream)
        t, steps = B.weno_theta_step(prob, grid, u, cfl, ws, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3
        cells = int(np.prod(U.shape[1:]))
        out[name] = {"value": cells * steps / sec, "unit": "cell-updates/s", "cells": cells, "rk_steps": steps,
                     "t_reached": t, "seconds": sec, "finite": bool(torch.isfinite(u).all())}
    return out


# ---------------------------------------------------------------------------------------------
# The reference arm: the CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------------------------

def run_reference(args):
    world, rank, _ = D.env()
    if rank != 0:
        return
    import oracle as O

    O.lib()
    every = 8  # 512 of the 4096 problems, every 8th by length: the batch's length mix
    ids = stride_sample(W.batch_lengths(NPROB, seed=0), every)
    b = W.euler_batch(NPROB, seed=0, problems=ids)
    P = O.problem(O.FLUX_EULER1D, alpha_R=W.ALPHA_R_SEEDED)
    cells = int(b.lengths.sum())

    def one(u):
        return O.run_batch(P, u, b.offsets, b.lengths, b.lo, b.hi, b.bc, cfl=CFL, n_steps=1, threads=0)[0]

    u = b.u
    for _ in range(args.warmup):
        u = one(u)
    u = b.u
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u = one(u)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = cells * args.steps / tot
    sample = (f"each benchmark step: 1 RK3 step of {len(ids)} of the {NPROB} problems (every {every}th by length, "
              f"{cells} cells), OpenMP over problems on {O.max_threads()} threads, from the initial data")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(max(args.gpus, 1)),
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": O.max_threads(), "kind": "oracle",
                         "sample": sample, **host_info()},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------------------------

def run_ours(args):
    import torch

    from paper_1504_00731_gb300 import binding as B
    from paper_1504_00731_gb300 import build as BLD

    world, rank, local = D.env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        BLD.build_library()
    if world > 1:
        dist.barrier()
    B.lib()

    # this rank's share: the LPT partition of the first world x 4096 problems of the stream
    lengths_all = W.batch_lengths(NPROB * world, seed=0)
    mine = D.lpt_partition(lengths_all, world)[rank] if world > 1 else np.arange(NPROB)
    batch = W.euler_batch(NPROB * world, seed=0, problems=mine)
    prob = B.problem(B.WT_FLUX_EULER1D, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
    segs = segments(B, batch)
    total = int(batch.u.shape[1])
    ws = B.alloc_workspace(B.workspace_bytes(prob, None, total, len(segs)), dev)
    src = torch.from_numpy(batch.u).to(dev)
    u = src.clone()
    stream = torch.cuda.current_stream(dev)

    def one_step(arr, k=RK_PER_STEP, strm=None):
        B.weno_theta_step_batched(prob, segs, arr, total, CFL, k, ws, stream=strm)

    for _ in range(args.warmup):  # the first call autotunes the tile and captures the graph
        one_step(u)
    torch.cuda.synchronize()
    u.copy_(src)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region: K benchmark steps (K x 10 RK steps) from the initial data
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        wall0 = time.perf_counter()
        ev_all0 = torch.cuda.Event(enable_timing=True)
        ev_all1 = torch.cuda.Event(enable_timing=True)
        ev_all0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            one_step(u)
            ev[k][1].record(stream)
        ev_all1.record(stream)
        barrier()
        wall = time.perf_counter() - wall0
    finite = bool(torch.isfinite(u).all())
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = ev_all0.elapsed_time(ev_all1)
    # the same calls with zero RK steps (state in, alphas, state out): the rest of each timed
    # call is the 3 x 10 launches of the batched stage kernel
    u0 = torch.empty_like(u)
    ms0 = []
    for k in range(min(args.steps, 5)):
        ev[k][0].record(stream)
        one_step(u0.copy_(src), k=0)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms0 = [ev[k][0].elapsed_time(ev[k][1]) for k in range(min(args.steps, 5))]
    launch_ms = (float(np.mean(step_ms)) - float(np.mean(ms0))) / (3 * RK_PER_STEP)
    tot_ms = D.max_over_ranks(tot_ms, dev)
    cells_all = D.sum_over_ranks(float(total), dev)
    ms_per_step = tot_ms / args.steps
    value = D.whole_job_rate(cells_all * RK_PER_STEP * args.steps, tot_ms * 1e-3)

    # ---- end to end through the public API with pinned host buffers (copies inside)
    h_src = torch.from_numpy(batch.u).pin_memory()
    h_u = torch.empty_like(h_src).pin_memory()
    h_u.copy_(h_src)
    e2e_steps = max(2, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        one_step(h_u.numpy(), strm=stream.cuda_stream)
    e2e_s = D.max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = D.whole_job_rate(cells_all * RK_PER_STEP * e2e_steps, e2e_s)
    del h_src, h_u

    if rank == 0:
        peaks = measured_peaks()
        cu_rate = total / (3 * launch_ms * 1e-3)  # cell-updates/s of the stage kernel alone (3 launches per RK step)
        achieved = FLOPS_PER_CELL_UPDATE * cu_rate / 1e9
        c = counters("batched")
        traffic = c["dram_bytes_per_cell_stage"] * total if c else None
        hbm_gbs = BYTES_PER_CELL_UPDATE_STAGES / 3 * total / (launch_ms * 1e-3) / 1e9
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(world),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
                         "kernel": "stage1d_batched_kernel<FastMath, Euler1D, stage, T> (one launch per RK stage over "
                                   "every problem; T chosen by the autotuner)",
                         "launch_ms": launch_ms, "flops_per_launch": FLOPS_PER_CELL_UPDATE / 3 * total,
                         "cells_per_launch": total,
                         "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (unit counts and max clock); "
                                        "microbenchmark 94.7% of it", "flops_note": FLOPS_NOTE,
                         **pipe_block("batched", cu_rate, FLOPS_PER_CELL_UPDATE),
                         "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": hbm_peak, "frac": hbm_gbs / hbm_peak,
                                 "bytes_per_cell_update": BYTES_PER_CELL_UPDATE_STAGES,
                                 "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}},
            "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": int(batch.u.nbytes),
                    "d2h_bytes_per_step": int(batch.u.nbytes), "steps": e2e_steps,
                    "how": "weno_theta_step_batched on pinned host arrays: the library copies the state in, runs 10 "
                           "RK steps and copies it out, every step"},
            # per benchmark step: pack, alphas, 3 x 10 stage launches, unpack
            "gpu_launches": args.steps * (3 + 3 * RK_PER_STEP),
            "clocks": clk.summary(),
            "wall_s_timed_region": wall,
            "state_finite": finite,
        }
        if world == 1 and not args.no_extras:
            ex = {}
            pv = plain_vs_batched(B, dev, batch)
            # the most any kernel issuing this kernel's FP64 instructions could reach: every SMSP's
            # FP64 pipe busy all the time (152 x 4 x 0.5 lanes per clock at 2.07 GHz)
            cb = counters("batched")
            full_pipe = 152 * 4 * 0.5 * 2.07e9 / cb["fp64_thread_ops_per_cell_update"] if cb else None
            ex["batched_vs_plain"] = {**pv, "batched_value": value,
                                      "batched_over_plain_auto": value / pv["plain_auto"]["value"],
                                      "batched_over_plain_stages": value / pv["plain_stages"]["value"],
                                      "rate_at_full_fp64_pipe": full_pipe,
                                      "ratio_at_full_fp64_pipe": full_pipe / pv["plain_auto"]["value"] if cb else None,
                                      "how": "all 4096 problems through weno_theta_step one at a time, 20 RK steps "
                                             "each; cell-updates/s over the summed CUDA-event times of the calls"}
            del ws, src, u, u0
            torch.cuda.empty_cache()
            ex["single_problem"] = single_problem_measure(B, dev)
            ex["euler2d"] = euler2d_measure(B, dev)
            ex["adjoint"] = adjoint_measure(B, dev)
            ex["problems"] = problems_measure(B, dev)
            line.update(ex)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_profile_case(name):
    """Small cases of the dominant kernels for ncu captures (a few launches, a few GB at most)."""
    import torch

    from paper_1504_00731_gb300 import binding as B
    from paper_1504_00731_gb300 import build as BLD

    BLD.build_library()
    dev = torch.device("cuda", 0)
    if name == "batched-512":
        # 512 problems of the batched workload (6.9 M cells, 165 MB per state, above L2), with the
        # tile the autotuner picks on the whole batch (127 cells, six items per thread): two calls
        # of one RK step, three stage launches each (the second call's are the ones to capture)
        os.environ.setdefault("WT_BATCHED_TILE", "5127")
        b = W.euler_batch(512, seed=0)
        prob = B.problem(B.WT_FLUX_EULER1D, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
        segs = segments(B, b)
        total = int(b.u.shape[1])
        ws = B.alloc_workspace(B.workspace_bytes(prob, None, total, len(segs)), dev)
        u = torch.from_numpy(b.u).to(dev)
        B.weno_theta_step_batched(prob, segs, u, total, CFL, 1, ws)
        B.weno_theta_step_batched(prob, segs, u, total, CFL, 1, ws)
        print("cells", total)
    elif name == "stepblock-4096":
        U0, x, dx = W.euler_c2(4096, seed=0)
        prob = B.problem(B.WT_FLUX_EULER1D, bc=B.WT_BC_OUTFLOW, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
        g = B.grid_1d(4096, -5.0, 5.0)
        ws = B.alloc_workspace(B.workspace_bytes(prob, g), dev)
        u = torch.from_numpy(U0).to(dev)
        B.weno_theta_step(prob, g, u, CFL, ws, max_steps=200)
        print("cells", 4096)
    elif name == "2d-1024":
        U, dx, dy = W.euler2d_vortices(1024, 1024, seed=0)
        prob = B.problem(B.WT_FLUX_EULER2D, bc=B.WT_BC_PERIODIC, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
        g = B.grid_2d(1024, 1024)
        ws = B.alloc_workspace(B.workspace_bytes(prob, g), dev)
        u = torch.from_numpy(U).to(dev)
        B.weno_theta_step(prob, g, u, 0.45, ws, max_steps=1)
        print("cells", 1024 * 1024)
    elif name == "adjoint-64":
        # 64 problems of the adjoint workload, 8 steps with checkpoints every 4
        U0, dx = W.adjoint_batch(64, 16384)
        prob = B.problem(B.WT_FLUX_EULER1D, bc=B.WT_BC_OUTFLOW, mode=B.WT_MODE_FAST, alpha_R=W.ALPHA_R_SEEDED)
        g = B.grid_1d(16384, -5.0, 5.0)
        ws = B.alloc_workspace(B.adjoint_workspace_bytes(prob, g, 64, 8, 4), dev)
        u = torch.from_numpy(U0).to(dev)
        gT, g0, uT = torch.zeros_like(u), torch.empty_like(u), torch.empty_like(u)
        gT[:, 0, :] = 1e-3
        B.weno_theta_adjoint(prob, g, 64, u, CFL, 8, 4, gT, g0, ws, uT=uT)
        u = g0
        print("cells", 64 * 16384)
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    print("ok", bool(torch.isfinite(u).all()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the single-problem, 2D, adjoint and per-problem "
                                                              "measurements")
    ap.add_argument("--profile-case", default=None, help="run one small case for an ncu capture and exit")
    ap.add_argument("--cpu-baseline-only", action="store_true", help="print the oracle's CPU baseline and exit")
    args = ap.parse_args()
    if args.cpu_baseline_only:
        print(json.dumps(cpu_baseline_here()), flush=True)
    elif args.profile_case:
        run_profile_case(args.profile_case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
