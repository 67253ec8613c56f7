#!/usr/bin/env python3
"""Throughput of the GB300 finite-volume shallow-water step.

Workload (default): the 40M-triangle Thacker-type paraboloid basin -- the
paper's Sec. 3 benchmark generator on a 4472 x 4472 jittered grid at
dx = 0.04 m (178.9 m domain), cells emitted in scattered order and
Hilbert-renumbered by the library, FP32, CFL 0.9, H_threshold 1e-5 m.
A step is one full SSP-RK(2,2) step (both stages, the CFL reduction and the
epilogue) over all cells; the metric is cell-updates per second (one cell
advanced one full step).

One JSON line on rank 0:
  value        device-timed cell-updates/s over the K timed steps (inputs
               resident in HBM; the working set is ~5 GB, far above L2)
  e2e          the same metric through the public C ABI with host buffers:
               each step uploads the state from pinned host memory
               (vg_set_state_f32 for the FP32 solver, vg_set_state for FP64),
               advances one step and reads the state back (vg_get_state_f32 /
               vg_get_state); the FP32 solver also reports the FP64 host
               interface (f64_host)
  roofline     the dominant kernel's algorithmic bytes per launch over its
               CUDA-event duration, against the measured HBM copy bandwidth
               (MEASURED_PEAKS.json; without it the 6800 GB/s fallback,
               named in peak_kind)
  cpu_baseline the FP64 CPU oracle timed on this host on a bounded sample
               of the same workload

--impl reference times the oracle alone (the slow reference arm).
Multi-GPU (torchrun): independent replicas, one per GPU (the method's time
step couples every cell, so one problem is not split); value sums all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FV cell-updates/s & HBM GB/s vs ~8 TB/s; batched & adjoint vs plain forward"
UNIT = "cell-updates/s"

# Algorithmic bytes per cell and launch (compact-mesh minimum: state, bed,
# neighbour ids, vertex ids, centroid, shared vertex coordinates; each array
# touched once): stage 1 reads w^n, bed, mesh and writes R0; stage 2 also
# reads w^n and R0 and writes w^{n+1}.
ALGO_BYTES = {32: {"stage1": 64, "stage2": 76}, 64: {"stage1": 104, "stage2": 128}}
# The unfused RK stages (rk_unfused = 1) replace stage 2 by: update 1 (reads w^n,
# R0 and the bed, writes w1), the residual of w1 (stage 1's bytes) and update 2
# (reads w^n, w1, R(w1) and the bed, writes w^{n+1}).
UNFUSED_BYTES = {32: {"rk_update1": 40, "residual_w1": 64, "rk_update2": 52},
                 64: {"rk_update1": 80, "residual_w1": 104, "rk_update2": 104}}

# FP64 is bound by GB300's FP64 units, not HBM.  Algorithmic FP64 operations per
# cell per full step (add, sub, mul, div, sqrt on state-dependent values; the
# geometry is precomputed), counted in the oracle's own arithmetic by
# `python -m oracle.count_ops` on a 180,000-cell sample of each generator; the
# two stages run the same residual, so each stage is taken as half.
FP64_FLOPS_PER_CELL_STEP = {"thacker": 508.73, "flat": 690.68, "coast": 638.69}
# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA thread-operations
# per cycle per SM (ncu: sm__sass_thread_inst_executed_op_dfma_pred_on peak) x 2
# flops x 2.07 GHz maximum SM clock = 1.26 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

WORKLOADS = {
    "thacker_paraboloid_40m": dict(n=4472),
    "thacker_paraboloid_10m": dict(n=2236),
    "thacker_paraboloid_4m": dict(n=1414),
    "thacker_paraboloid_1m": dict(n=707),
    # all-wet control: the same grid over a flat 10 m bed with a Gaussian hump of
    # the free surface (no dry cells, so no wet/dry divergence)
    "flat_basin_allwet_40m": dict(n=4472, kind="flat"),
    "flat_basin_allwet_4m": dict(n=1414, kind="flat"),
    # ocean-to-coast basin (5.0M triangles graded 20:1, dry land, N-wave source)
    "coast_basin_5m": dict(n=None, kind="coast", hthr=1e-3),
}


def workload_hthr(name: str) -> float:
    return WORKLOADS[name].get("hthr", 1e-5)


def _sample_desc(name: str, n: int) -> str:
    if WORKLOADS[name].get("kind") == "coast":
        return f"coast basin of about {2 * n * n} triangles"
    return f"n={n}, dx=0.04 m"


def workload_inputs(name: str, n):
    """Mesh and initial state of a workload's generator on an n x n grid at dx = 0.04 m
    (coast basin: about 2 n^2 triangles of the same generator; n = None: 5.0M)."""
    from paper_2002_04889_gb300 import inputs as I
    if WORKLOADS[name].get("kind") == "coast":
        m = I.coast_mesh() if n is None else I.coast_mesh_with_cells(2 * n * n, seed=0)
        return m, I.coast_initial_state(m)
    if WORKLOADS[name].get("kind") == "flat":
        half = 0.5 * n * 0.04
        m = I.flat_basin_mesh(n, half, 10.0, shuffle_cells=True)
        return m, I.gaussian_hump_state(m, 0.0, 1.0, 0.0, 0.0, 0.1 * half)
    m = I.thacker_large_mesh(n=n)
    return m, I.thacker_initial_state(m)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job cell-updates/s of independent replicas: every rank advances its own
    cells_per_rank cells by `steps` steps; the job takes the slowest rank's time."""
    return cells_per_rank * steps * world / (ms_max * 1e-3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.skip = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: begin the timed region once it
            # samples, so that a short region is still covered
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.skip = len(self.lines)
        except (OSError, FileNotFoundError):
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples taken before the timed region began are left out, unless there
        # is no other
        lines = self.lines[self.skip:] or self.lines
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def code_digest(texts) -> str:
    """sha1 (first 12 hex) of source texts with // comments and whitespace
    removed, so that an edit of comments alone keeps the digest."""
    h = hashlib.sha1()
    for t in texts:
        code = re.sub(r"//[^\n]*", "", t)
        h.update("".join(code.split()).encode())
    return h.hexdigest()[:12]


def kernel_source_sha() -> str:
    texts = []
    for f in ("step_kernels.cuh", "step_f32.cu", "step_f64.cu", "step_f64_fast.cu"):
        with open(os.path.join(ROOT, "paper_2002_04889_gb300", "csrc", f)) as fh:
            texts.append(fh.read())
    return code_digest(texts)


def profiled_traffic(workload: str, precision: int, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"stage_kernels_{workload}_fp{precision}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_source_sha():
        return None
    m = re.search(rf"traffic_bytes_per_launch\s+{kernel}:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


def make_workload(name: str):
    return workload_inputs(name, WORKLOADS[name]["n"])


def cpu_baseline(budget_s: float = 15.0, n: int = 1414, workload: str = "thacker_paraboloid_40m",
                 single_budget_s: float = 5.0):
    """The FP64 oracle on a bounded sample of the workload: the same generator at the
    same dx on an n x n grid (2 n^2 triangles), as many steps as fit in budget_s, on
    all host cores (OpenMP); then the single-threaded oracle on the same sample for
    single_budget_s (reported beside it)."""
    import oracle as O
    m, s = workload_inputs(workload, n)
    om = O.OracleMesh.from_mesh(m)
    prm = O.params(h_threshold=workload_hthr(workload), cfl=0.9)
    cores = O.max_threads()

    def timed(budget):
        st = (s.H, s.Hu, s.Hv, 0.0)
        steps, t0 = 0, time.perf_counter()
        while True:
            r = om.run(prm, st, 1)
            st = (r["H"], r["Hu"], r["Hv"], r["t"])
            steps += 1
            el = time.perf_counter() - t0
            if el >= budget or steps >= 200:
                return steps, el

    steps, el = timed(budget_s)
    O.set_threads(1)
    try:
        steps1, el1 = timed(single_budget_s)
    finally:
        O.set_threads(cores)
    return {"value": m.nc * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps on a {m.nc}-triangle sample of the same "
                      f"generator ({_sample_desc(workload, n)}), {el:.1f} s",
            "single_thread": {"value": m.nc * steps1 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"the same sample, {steps1} steps, {el1:.1f} s"}}


def batched_leg(torch, stream, steps: int, n_scen: int = 32, renumber: str = "hilbert"):
    """Config 4: 8 coast basins of 50k..2M triangles x n_scen scenarios (uplift
    amplitude U[1,5] m, orientation U[0,180) deg), FP32, all advanced together to a
    common end time t_end with per-scenario time steps (one persistent launch per
    stage, graph replay, autotuned block size and CTAs per SM), against a loop of
    single-scenario solves (one context per mesh, each scenario set and advanced
    to t_end in turn) on the same GPU.  t_end is `steps` CFL steps of the fastest
    scenario.  Throughput counts each scenario's own steps (a scenario that reached
    t_end stops counting); every scenario's final state is compared with its
    single-context run, bit for bit."""
    import numpy as np
    from paper_2002_04889_gb300 import inputs as I
    from paper_2002_04889_gb300 import volna
    t0 = time.perf_counter()
    meshes = [I.coast_mesh_with_cells(n, seed=k) for k, n in enumerate(I.ensemble_meshes())]
    srcs = [I.ensemble_sources(k, n_scen) for k in range(len(meshes))]
    b = volna.Batch(32, device=torch.cuda.current_device(), stream=stream)
    b.set_params(h_threshold=1e-3, cfl=0.9)
    ids = [b.add_mesh(m, n_scen, renumber=renumber) for m in meshes]
    states = [[I.coast_initial_state(m, amplitude=amp, angle_deg=ang) for amp, ang in src]
              for m, src in zip(meshes, srcs)]

    def reset():
        for mid in ids:
            for j in range(n_scen):
                s0 = states[mid][j]
                b.set_state(mid, j, s0.H, s0.Hu, s0.Hv, 0.0)

    reset()
    setup = time.perf_counter() - t0
    tuned = b.autotune(3)
    reset()                               # the tuner restored the state; restart all at t = 0
    cells = b.info()["cells"]
    b.step(1)                             # t_end: `steps` steps of the fastest scenario
    dt1 = max(b.get_state(mid, j)[3] for mid in ids for j in range(n_scen))
    t_end = steps * dt1
    reset()
    b.run(t_end)                          # warm-up over the same run
    reset()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    batch_steps = b.run(t_end)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_batch = ev0.elapsed_time(ev1)
    # loop of single-scenario solves to the same t_end, each compared with its scenario
    t_loop = 0.0
    updates = 0
    same = True
    n_cmp = 0
    for mid, m in enumerate(meshes):
        sv = volna.Solver(32, device=torch.cuda.current_device(), stream=stream)
        sv.set_params(h_threshold=1e-3, cfl=0.9, block_cells=tuned[0])
        sv.upload_mesh(m, renumber=renumber)
        for j in range(n_scen):
            s0 = states[mid][j]
            sv.set_state(s0.H, s0.Hu, s0.Hv, 0.0)
            sv.step(2)                    # warm-up
            sv.set_state(s0.H, s0.Hu, s0.Hv, 0.0)
            torch.cuda.synchronize()
            ev0.record(stream)
            sv.advance_to(t_end)
            ev1.record(stream)
            torch.cuda.synchronize()
            t_loop += ev0.elapsed_time(ev1)
            H, Hu, Hv, t_s = sv.get_state()
            steps_s = int(sv.diagnostics()["steps"])
            bH, bHu, bHv, bt, bsteps = b.get_state(mid, j)
            updates += m.nc * int(bsteps)
            same = same and bsteps == steps_s and bt == t_s and all(
                np.array_equal(x, y) for x, y in zip((H, Hu, Hv), (bH, bHu, bHv)))
            n_cmp += 1
        sv.close()
    b.close()
    return {"workload": f"coast basins {I.ensemble_meshes()} triangles x {n_scen} scenarios, FP32, to a common "
                        f"t_end with per-scenario dt",
            "cells": cells, "t_end": t_end, "batched_steps": batch_steps,
            "cell_updates": updates, "autotuned": {"block_cells": tuned[0], "ctas_per_sm": tuned[2]},
            "value": updates / (ms_batch * 1e-3), "unit": UNIT,
            "loop_of_singles": updates / (t_loop * 1e-3),
            "speedup_vs_loop": t_loop / ms_batch, "scenarios_compared": n_cmp,
            "bitwise_equal_to_singles": bool(same), "setup_s": round(setup, 1)}


def adjoint_leg(torch, stream, steps: int, n: int = 707, slots: int = 16):
    """Config 5 mesh (Thacker basin, n x n squares, 2 n^2 triangles), FP64: the cost of
    the gradient of a 16-gauge misfit (forward with checkpoints every C steps, C the
    library's memory-balanced default, + reverse sweep recomputing each segment
    once) against the plain forward run of the same steps."""
    import numpy as np
    from paper_2002_04889_gb300 import inputs as I
    from paper_2002_04889_gb300 import volna
    m = I.thacker_mesh(n=n, half_width=1.0)
    s = I.thacker_initial_state(m)
    lat = np.array([[x, y] for x in np.linspace(-0.6, 0.6, 4) for y in np.linspace(-0.6, 0.6, 4)])
    dt = 0.8 * 0.9 * 0.1 * (2.0 / n)
    sv = volna.Solver(64, device=torch.cuda.current_device(), stream=stream)
    sv.set_params(h_threshold=1e-5, dt_fixed=dt)
    sv.upload_mesh(m)
    sv.set_gauges(lat)
    sv.set_state(s.H, s.Hu, s.Hv)
    sv.step(3)
    sv.set_state(s.H, s.Hu, s.Hv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sv.step(steps)                        # the literal FP64 build, which the adjoint reverses
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    sv.set_params(fp64_literal=0)         # the contracted build, for context
    sv.set_state(s.H, s.Hu, s.Hv)
    sv.step(3)
    sv.set_state(s.H, s.Hu, s.Hv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sv.step(steps)
    torch.cuda.synchronize()
    t_fwd_fast = time.perf_counter() - t0
    sv.set_params(h_threshold=1e-5, fp64_literal=1)
    sv.set_state(s.H, s.Hu, s.Hv)
    t0 = time.perf_counter()
    _, eta = sv.adj_forward(steps, dt)
    t1 = time.perf_counter()
    sv.adj_backward(np.full_like(eta, 1e-3), m.nv)
    t2 = time.perf_counter()
    # binomial checkpointing with `slots` state slots (0: skipped): far less
    # memory, more recomputation
    t3 = t4 = 0.0
    if slots > 0:
        sv.set_state(s.H, s.Hu, s.Hv)
        t3 = time.perf_counter()
        _, eta = sv.adj_forward_binomial(steps, dt, slots)
        sv.adj_backward(np.full_like(eta, 1e-3), m.nv)
        t4 = time.perf_counter()
    sv.close()
    # per cell and recorded step: state, R0, face values of both stages, one bit
    # of dry-fix branch and two of reconstruction flags; per checkpoint: the state
    rec = 24 + 24 + 144 + 3 / 8
    C = max(1, round(math.sqrt(steps * 24 / rec)))     # the library's default segment length
    return {"workload": f"Thacker basin {m.nc} triangles, FP64, {steps} steps, 16 gauges",
            "forward_s": round(t_fwd, 4), "forward_contracted_s": round(t_fwd_fast, 4),
            "adj_forward_s": round(t1 - t0, 4),
            "adj_backward_s": round(t2 - t1, 4), "cost_vs_forward": round((t2 - t0) / t_fwd, 3),
            "forward_value": m.nc * steps / t_fwd, "unit": UNIT,
            "segment_steps": C,
            "scratch_bytes_per_cell": round(math.ceil(steps / C) * 24 + C * rec),
            "binomial": None if slots <= 0 else {"slots": slots, "cost_vs_forward": round((t4 - t3) / t_fwd, 3),
                                                 "scratch_bytes_per_cell": (slots + 3) * 24 + rec}}


def roofline_of(prof, nc: int, precision: int, workload: str, step_ms: float):
    """Roofline of the dominant stage kernel from the per-kernel CUDA-event profile:
    HBM (FP32: algorithmic bytes per launch over its duration) or, for FP64, the
    FP64 units (algorithmic flops per launch over its duration)."""
    peak, peak_kind = measured_peaks()
    per_kernel = {k: (n, tot) for k, (n, tot) in prof.items() if n > 0}
    dom = max(("stage1", "stage2"), key=lambda k: per_kernel.get(k, (0, 0.0))[1])
    n_l, tot = per_kernel[dom]
    avg_ms = tot / n_l
    algo = ALGO_BYTES[precision][dom] * nc
    achieved = algo / (avg_ms * 1e-3) / 1e9
    traffic = profiled_traffic(workload, precision, dom)
    kernel_ms = {k: round(tot_ / max(n_, 1), 4) for k, (n_, tot_) in per_kernel.items()}
    per_cell = dict(ALGO_BYTES[precision], **UNFUSED_BYTES[precision])
    unfused = "rk_update1" in per_kernel
    step_bytes = sum(per_cell[k] for k in (("stage1", "rk_update1", "residual_w1", "rk_update2") if unfused
                                           else ("stage1", "stage2"))) * nc
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom,
                "algo_bytes_per_launch": algo, "peak_kind": f"{peak_kind} hbm_gbs",
                "kernel_avg_ms": kernel_ms,
                "step_algo_gbs": round(step_bytes / (step_ms * 1e-3) / 1e9, 1)}
    if unfused:
        # every kernel of the unfused step against the same peak
        roofline["per_kernel_gbs"] = {k: round(per_cell[k] * nc / (kernel_ms[k] * 1e-3) / 1e9, 1)
                                      for k in ("stage1", "rk_update1", "residual_w1", "rk_update2")
                                      if kernel_ms.get(k)}
    if precision == 64:
        kind = WORKLOADS[workload].get("kind", "thacker")
        flops = 0.5 * FP64_FLOPS_PER_CELL_STEP[kind] * nc
        tflops = flops / (avg_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                    "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                    "kernel": dom, "algo_flops_per_launch": flops,
                    "peak_kind": "derived: 152 SMs x 4 FP64 flop/cycle x 2.07 GHz",
                    "kernel_avg_ms": kernel_ms, "hbm_frac": round(achieved / peak, 4)}
    return roofline


def workload_leg(torch, stream, workload: str, precision: int, steps: int, warmup: int = 3, inputs=None,
                 renumber: str = "hilbert", variants=None):
    """One workload at one precision: device-timed cell-updates/s over `steps` steps
    (CUDA events on the solver's stream) and the dominant kernel's roofline.
    variants: {name: params} timed in turn on the same context from the same
    initial state (FP64: the literal and the contracted build); the first is the
    leg's own line, the others go under "variants"."""
    from paper_2002_04889_gb300 import volna
    mesh, st0 = inputs if inputs is not None else make_workload(workload)
    variants = variants or {"default": {}}
    sv = volna.Solver(precision=precision, device=torch.cuda.current_device(), stream=stream)
    out = None
    try:
        sv.set_params(h_threshold=workload_hthr(workload), cfl=0.9)
        sv.upload_mesh(mesh, renumber=renumber)
        for name, prm in variants.items():
            if prm:
                sv.set_params(**prm)
            sv.set_state(st0.H, st0.Hu, st0.Hv, 0.0)
            sv.step(warmup)
            sv.profile(True)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            sv.step(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            prof = sv.get_profile()
            sv.profile(False)
            d = sv.diagnostics()
            line = {"workload": workload, "cells": mesh.nc, "dtype": "f32" if precision == 32 else "f64",
                    "steps": steps, "value": mesh.nc * steps / (ms * 1e-3), "unit": UNIT,
                    "ms_per_step": ms / steps, "neg_count": d["neg_count"],
                    "roofline": roofline_of(prof, mesh.nc, precision, workload, ms / steps)}
            if out is None:
                out = line
                if len(variants) > 1:
                    out["variant"] = name
                    out["variants"] = {}
            else:
                out["variants"][name] = line
    finally:
        sv.close()
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    n = 707
    m, s = workload_inputs(args.workload, n)
    om = O.OracleMesh.from_mesh(m)
    prm = O.params(h_threshold=workload_hthr(args.workload), cfl=0.9)
    st = (s.H, s.Hu, s.Hv, 0.0)
    for _ in range(args.warmup):
        r = om.run(prm, st, 1)
        st = (r["H"], r["Hu"], r["Hv"], r["t"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = om.run(prm, st, 1)
        st = (r["H"], r["Hu"], r["Hv"], r["t"])
    el = time.perf_counter() - t0
    value = m.nc * args.steps / el
    sample = (f"FP64 CPU oracle, each step one SSP-RK(2,2) step on a {m.nc}-triangle sample of the "
              f"workload's generator ({_sample_desc(args.workload, n)})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "sample_cells": m.nc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="thacker_paraboloid_40m", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--renumber", default="hilbert", choices=["none", "morton", "rcm", "hilbert"])
    ap.add_argument("--fp64-build", default="literal", choices=["literal", "contracted"],
                    help="FP64 stage kernels of the main leg: literal (bit for bit the oracle's arithmetic, the "
                         "library default) or contracted (fused multiply-adds, fewer divisions)")
    ap.add_argument("--rk-unfused", type=int, default=0, choices=[0, 1],
                    help="1 runs the main leg with the RK stage updates as kernels of their own "
                         "(for profiling them; the default line is the fused step)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--batched-steps", type=int, default=20, help="0 skips the batched-ensemble leg")
    ap.add_argument("--batched-scenarios", type=int, default=32,
                    help="scenarios per mesh of the batched leg (32: the ensemble configuration)")
    ap.add_argument("--adjoint-steps", type=int, default=2000, help="0 skips the adjoint-cost leg")
    ap.add_argument("--adjoint-binomial-slots", type=int, default=16, help="0 skips the binomial run")
    ap.add_argument("--config-legs", type=int, default=1,
                    help="0 skips the other configurations (the other precision on the same mesh, the "
                         "all-wet control, and the 5M coast basin in FP32 and FP64)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    ws, rank, local = dist_env()
    import numpy as np
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2002_04889_gb300 import volna

    t_setup = time.perf_counter()
    mesh, st0 = make_workload(args.workload)
    stream = torch.cuda.Stream()
    sv = volna.Solver(precision=args.precision, device=torch.cuda.current_device(), stream=stream)
    sv.set_params(h_threshold=workload_hthr(args.workload), cfl=0.9,
                  fp64_literal=0 if args.fp64_build == "contracted" else 1, rk_unfused=args.rk_unfused)
    sv.upload_mesh(mesh, renumber=args.renumber)
    sv.set_state(st0.H, st0.Hu, st0.Hv, 0.0)
    nc = mesh.nc
    dev_gb = sv.device_bytes() / 1e9
    log(f"[bench] rank {rank}: {nc} cells ready in {time.perf_counter() - t_setup:.1f} s, "
        f"{dev_gb:.2f} GB on device")

    sv.step(args.warmup)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---- timed region: K steps, per-kernel CUDA events on the solver's stream
    sv.profile(True)
    d0 = sv.diagnostics()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        sv.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    prof = sv.get_profile()
    sv.profile(False)
    d1 = sv.diagnostics()
    launches = int(d1["launches"] - d0["launches"]) - 2   # minus the diagnostics' own 2
    ms = max_over_ranks(ms, "cuda")
    value = replica_throughput(nc, args.steps, ms, ws)

    # ---- roofline of the dominant kernel
    roofline = roofline_of(prof, nc, args.precision, args.workload, ms / args.steps)

    # ---- end to end through the C ABI with pinned host buffers
    def end_to_end(host_dtype, steps):
        """Seconds (max over ranks) for `steps` rounds of: state in from pinned host
        arrays of host_dtype, one step, state out to pinned host arrays."""
        fp32 = host_dtype == np.float32
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=host_dtype)).pin_memory().numpy()
        H, Hu, Hv, t_cur = sv.get_state()
        H, Hu, Hv = pin(H), pin(Hu), pin(Hv)
        tdt = torch.float32 if fp32 else torch.float64
        oH, oHu, oHv = (torch.empty(nc, dtype=tdt).pin_memory().numpy() for _ in range(3))
        set_fn = volna.vg_set_state_f32 if fp32 else volna.vg_set_state
        get_fn = volna.vg_get_state_f32 if fp32 else volna.vg_get_state
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            set_fn(sv.ctx, H, Hu, Hv, t_cur)
            sv.step(1)
            _, _, _, t_cur = get_fn(sv.ctx, nc, out=(oH, oHu, oHv))
            H, oH = oH, H
            Hu, oHu = oHu, Hu
            Hv, oHv = oHv, Hv
        torch.cuda.synchronize()
        return max_over_ranks(time.perf_counter() - t0, "cuda")

    e2e = None
    if args.e2e_steps > 0:
        # host arrays in the arithmetic's own precision (FP32 state <-> FP32 host
        # arrays loses nothing); the FP64 host interface is reported beside it
        host = np.float32 if args.precision == 32 else np.float64
        esz = np.dtype(host).itemsize
        el = end_to_end(host, args.e2e_steps)
        e2e = {"value": replica_throughput(nc, args.e2e_steps, el * 1e3, ws), "unit": UNIT,
               "h2d_bytes_per_step": 3 * esz * nc, "d2h_bytes_per_step": 3 * esz * nc,
               "steps": args.e2e_steps, "host_dtype": np.dtype(host).name}
        if args.precision == 32:
            el64 = end_to_end(np.float64, args.e2e_steps)
            e2e["f64_host"] = {"value": replica_throughput(nc, args.e2e_steps, el64 * 1e3, ws),
                               "h2d_bytes_per_step": 24 * nc, "d2h_bytes_per_step": 24 * nc}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_budget, workload=args.workload)
    sv.close()
    batched = adjoint = None
    configs = None
    if rank == 0 and args.config_legs > 0 and args.workload == "thacker_paraboloid_40m":
        # the other precision on the same 40M mesh (FP64: at most 20 timed steps,
        # ~90 ms each), the all-wet control (the 40M grid over a flat 10 m bed: no
        # dry cell, every cell reconstructs), then the 5M-triangle coast basin in
        # FP32 and FP64
        configs = {}
        other = 64 if args.precision == 32 else 32
        legs = [(f"thacker_paraboloid_40m_fp{other}", "thacker_paraboloid_40m", other, (mesh, st0)),
                ("flat_basin_allwet_40m_fp32", "flat_basin_allwet_40m", 32, None),
                ("thacker_paraboloid_40m_fp32_rk_unfused", "thacker_paraboloid_40m", 32, (mesh, st0)),
                ("coast_basin_5m_fp32", "coast_basin_5m", 32, None),
                ("coast_basin_5m_fp64", "coast_basin_5m", 64, None)]
        coast = None
        for key, wl, prec, inp in legs:
            try:
                if wl == "coast_basin_5m":
                    coast = coast if coast is not None else make_workload(wl)
                    inp = coast
                n_steps = min(args.steps, 20) if prec == 64 else args.steps
                # FP64: the literal build (bit for bit the oracle's arithmetic, the
                # default) and the contracted build (fp64_literal = 0)
                var = {"literal": {}, "contracted": {"fp64_literal": 0}} if prec == 64 else None
                if key.endswith("_rk_unfused"):
                    # the RK stage updates as kernels of their own (w1 and R(w1)
                    # through HBM), against the fused headline step
                    var = {"rk_unfused": {"rk_unfused": 1}}
                configs[key] = workload_leg(torch, stream, wl, prec, n_steps, inputs=inp,
                                            renumber=args.renumber, variants=var)
            except Exception as e:         # reported, not fatal: the headline is the forward step
                configs[key] = {"error": str(e)[:300]}
        del coast
    if rank == 0 and args.batched_steps > 0:
        try:
            batched = batched_leg(torch, stream, args.batched_steps, n_scen=args.batched_scenarios,
                                  renumber=args.renumber)
        except Exception as e:             # reported, not fatal: the headline is the forward step
            batched = {"error": str(e)[:300]}
    if rank == 0 and args.adjoint_steps > 0:
        try:
            adjoint = adjoint_leg(torch, stream, args.adjoint_steps, slots=args.adjoint_binomial_slots)
        except Exception as e:
            adjoint = {"error": str(e)[:300]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "cells": nc, "renumber": args.renumber,
                           **({"fp64_build": args.fp64_build} if args.precision == 64 else {}),
                           **({"rk_unfused": 1} if args.rk_unfused else {}),
                           "block_cells": 256, "cfl": 0.9, "h_threshold": workload_hthr(args.workload),
                           "l2": "inputs larger than L2 (%.1f GB resident)" % dev_gb,
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(),
                "neg_count": d1["neg_count"], "t_sim": d1["t"],
                "configs": configs, "batched": batched, "adjoint": adjoint}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
