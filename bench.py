#!/usr/bin/env python3
"""Throughput of the GB300 finite-volume shallow-water step.

Workload (default): the 40M-triangle Thacker-type paraboloid basin -- the
paper's Sec. 3 benchmark generator on a 4472 x 4472 jittered grid at
dx = 0.04 m (178.9 m domain), cells emitted in scattered order and
Morton-renumbered by the library, FP32, CFL 0.9, H_threshold 1e-5 m.
A step is one full SSP-RK(2,2) step (both stages, the CFL reduction and the
epilogue) over all cells; the metric is cell-updates per second (one cell
advanced one full step).

One JSON line on rank 0:
  value        device-timed cell-updates/s over the K timed steps (inputs
               resident in HBM; the working set is ~5 GB, far above L2)
  e2e          the same metric through the public C ABI with host buffers:
               each step uploads the state from pinned host memory
               (vg_set_state), advances one step and reads the state back
               (vg_get_state)
  roofline     the dominant kernel's algorithmic bytes per launch over its
               CUDA-event duration, against the measured HBM copy bandwidth
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

WORKLOADS = {
    "thacker_paraboloid_40m": dict(n=4472),
    "thacker_paraboloid_10m": dict(n=2236),
    "thacker_paraboloid_4m": dict(n=1414),
    "thacker_paraboloid_1m": dict(n=707),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        for ln in self.lines:
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


def kernel_source_sha() -> str:
    h = hashlib.sha1()
    for f in ("step_kernels.cuh", "step_f32.cu", "step_f64.cu"):
        with open(os.path.join(ROOT, "paper_2002_04889_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


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
    from paper_2002_04889_gb300 import inputs as I
    m = I.thacker_large_mesh(n=WORKLOADS[name]["n"])
    s = I.thacker_initial_state(m)
    return m, s


def cpu_baseline(budget_s: float = 15.0, n: int = 1414):
    """The FP64 oracle on a bounded sample of the workload: the same generator at the
    same dx on an n x n grid (2 n^2 triangles), as many steps as fit in budget_s."""
    import oracle as O
    from paper_2002_04889_gb300 import inputs as I
    m = I.thacker_large_mesh(n=n)
    s = I.thacker_initial_state(m)
    om = O.OracleMesh.from_mesh(m)
    prm = O.params(h_threshold=1e-5, cfl=0.9)
    st = (s.H, s.Hu, s.Hv, 0.0)
    steps, t0 = 0, time.perf_counter()
    while True:
        r = om.run(prm, st, 1)
        st = (r["H"], r["Hu"], r["Hv"], r["t"])
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 200:
            break
    return {"value": m.nc * steps / el, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps on a {m.nc}-triangle sample of the same "
                      f"generator (n={n}, dx=0.04 m), {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2002_04889_gb300 import inputs as I
    n = 707
    m = I.thacker_large_mesh(n=n)
    s = I.thacker_initial_state(m)
    om = O.OracleMesh.from_mesh(m)
    prm = O.params(h_threshold=1e-5, cfl=0.9)
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
              f"workload's generator (n={n}, dx=0.04 m)")
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
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="thacker_paraboloid_40m", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
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
    sv.set_params(h_threshold=1e-5, cfl=0.9)
    sv.upload_mesh(mesh, renumber="morton")
    sv.set_state(st0.H, st0.Hu, st0.Hv, 0.0)
    nc = mesh.nc
    log(f"[bench] rank {rank}: {nc} cells ready in {time.perf_counter() - t_setup:.1f} s, "
        f"{sv.device_bytes() / 1e9:.2f} GB on device")

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
    if ws > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = nc * args.steps * ws / (ms * 1e-3)

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    per_kernel = {k: (n, tot) for k, (n, tot) in prof.items() if n > 0}
    dom = max(("stage1", "stage2"), key=lambda k: per_kernel.get(k, (0, 0.0))[1])
    n_l, tot = per_kernel[dom]
    avg_ms = tot / n_l
    algo = ALGO_BYTES[args.precision][dom] * nc
    achieved = algo / (avg_ms * 1e-3) / 1e9
    traffic = profiled_traffic(args.workload, args.precision, dom)
    kernel_ms = {k: round(tot_ / max(n_, 1), 4) for k, (n_, tot_) in per_kernel.items()}
    step_bytes = (ALGO_BYTES[args.precision]["stage1"] + ALGO_BYTES[args.precision]["stage2"]) * nc
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom,
                "algo_bytes_per_launch": algo, "peak_kind": f"{peak_kind} hbm_gbs",
                "kernel_avg_ms": kernel_ms,
                "step_algo_gbs": round(step_bytes / (ms * 1e-3 / args.steps) / 1e9, 1)}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        H, Hu, Hv, t_cur = sv.get_state()
        H, Hu, Hv = pin(H), pin(Hu), pin(Hv)
        oH, oHu, oHv = (torch.empty(nc, dtype=torch.float64).pin_memory().numpy() for _ in range(3))
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            volna.vg_set_state(sv.ctx, H, Hu, Hv, t_cur)
            sv.step(1)
            _, _, _, t_cur = volna.vg_get_state(sv.ctx, nc, out=(oH, oHu, oHv))
            H, oH = oH, H
            Hu, oHu = oHu, Hu
            Hv, oHv = oHv, Hv
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([el], device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": nc * args.e2e_steps * ws / el, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * nc, "d2h_bytes_per_step": 3 * 8 * nc,
               "steps": args.e2e_steps}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_budget)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
                "config": {"workload": args.workload, "cells": nc, "renumber": "morton",
                           "block_cells": 256, "cfl": 0.9, "h_threshold": 1e-5,
                           "l2": "inputs larger than L2 (%.1f GB resident)" % (sv.device_bytes() / 1e9),
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(),
                "neg_count": d1["neg_count"], "t_sim": d1["t"]}
        print(json.dumps(line), flush=True)
    sv.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
