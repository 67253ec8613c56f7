"""Algorithmic FP64 operation counts per cell per step for the benchmark's
workloads, from the oracle compiled with an operation-counting scalar
(oracle/op_count.hpp).  TEST INFRASTRUCTURE: bench.py's FP64 roofline uses the
numbers this script prints (one adaptive SSP-RK(2,2) step from the initial state
of a 180,000-cell sample of each workload's generator; the coast basin's
threshold is 1e-3 m).

    python -m oracle.count_ops
"""
from __future__ import annotations

import oracle as O
from paper_2002_04889_gb300 import inputs as I


def counts(kind: str, n: int = 300) -> dict:
    half = 0.5 * n * 0.04
    hthr = 1e-5
    if kind == "flat":
        m = I.flat_basin_mesh(n, half, 10.0, shuffle_cells=True)
        s = I.gaussian_hump_state(m, 0.0, 1.0, 0.0, 0.0, 0.1 * half)
    elif kind == "coast":
        m = I.coast_mesh_with_cells(2 * n * n, seed=0)
        s = I.coast_initial_state(m)
        hthr = 1e-3
    else:
        m = I.thacker_large_mesh(n=n)
        s = I.thacker_initial_state(m)
    c = O.count_step_ops(m, (s.H, s.Hu, s.Hv), h_threshold=hthr, cfl=0.9)
    flops = c["add"] + c["sub"] + c["mul"] + c["div"] + c["sqrt"]
    per = {k: c[k] / m.nc for k in ("add", "sub", "mul", "div", "sqrt", "minmax")}
    per["flops"] = flops / m.nc
    return per


if __name__ == "__main__":
    for kind in ("thacker", "flat", "coast"):
        per = counts(kind)
        print(kind, " ".join(f"{k}={v:.2f}" for k, v in per.items()))
