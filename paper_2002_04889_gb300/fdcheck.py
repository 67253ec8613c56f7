"""Gradient check of the hand-written adjoint against central finite differences
of the FP64 forward run (the adjoint configuration: Thacker's basin of Sec. 3 on
n x n squares of [-1, 1]^2, a 16-gauge misfit, a fixed time step).

J = 1/2 sum_{n,g} (eta_g(t_n) - eta_g^target(t_n))^2 over 16 gauges on a 4 x 4
lattice in |x|, |y| <= 0.6 and every step; the target run has a seeded 0.01 m
Gaussian uplift of the free surface and a seeded +-1 % perturbation of the
vertex depths.  The time step is 0.8 times the CFL step (CFL 0.9) of the
initial state, shared by the target run, the finite differences and the
adjoint so that the gauge times coincide.  The initial state carries a small
smooth momentum in the deep water (1e-3 sin 3x, 1e-3 cos 2y): a momentum field
that is identically zero puts every cell's limiter on its D = 0 branch, whose
directional derivative is positively homogeneous but not linear, so a central
difference (the mean of the two one-sided slopes) would not measure the
adjoint's derivative there.  Directions: seeded normal vectors in
the initial depth (wet cells) and in the vertex depths.  For each direction the
adjoint's directional derivative <grad J, d> is compared with
(J(x + eps d) - J(x - eps d)) / (2 eps) at a main step and, for the first few
directions, over a sweep of steps.  J is piecewise smooth, and its kinks are
dense: Zhou's wave speeds (Sec. 2.2) take the min / max of two arguments that
are nearly equal wherever the flow is smooth, the limiter's active face and
the stencil's extremes switch, and a 1M-cell, 2000-step run evaluates billions
of such choices, so a step of 1e-6 crosses many kinks and the difference
quotient departs from the derivative of the branch taken by percents; it
approaches it as the step shrinks, until round-off takes over (the plateau).
The main step is therefore 1e-8.

``python -m paper_2002_04889_gb300.fdcheck`` runs it at full size (1M triangles,
2000 steps, 32 directions) on cuda:0 and prints one JSON object.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import inputs
from .volna import Solver

LATTICE = np.array([[x, y] for x in np.linspace(-0.6, 0.6, 4) for y in np.linspace(-0.6, 0.6, 4)])


def _cfl_dt(mesh, state, device):
    with Solver(64, device=device) as sv:
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.upload_mesh(mesh)
        sv.set_state(state.H, state.Hu, state.Hv, 0.0)
        sv.step(1)
        return 0.8 * sv.diagnostics()["last_dt"]


def fd_check(n: int = 707, n_steps: int = 2000, n_dirs: int = 32, eps: float = 1e-8,
             eps_sweep=(1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 1e-10), sweep_dirs: int = 4, seed: int = 0,
             device: int = 0) -> dict:
    mesh = inputs.thacker_mesh(n=n, half_width=1.0)
    s0 = inputs.thacker_initial_state(mesh)
    p = mesh.cell_points()
    deep = s0.H > 2e-2
    s = inputs.State(s0.H, s0.Hu + 1e-3 * np.sin(3.0 * p[:, 0]) * deep,
                     s0.Hv + 1e-3 * np.cos(2.0 * p[:, 1]) * deep, 0.0)
    dt = _cfl_dt(mesh, s, device)
    rng = np.random.default_rng(seed)
    bump = 0.01 * np.exp(-((p[:, 0] - 0.2) ** 2 + (p[:, 1] + 0.1) ** 2) / 0.05)
    wet = s.H > 2e-2
    depth_t = mesh.depth * (1.0 + 0.01 * (2.0 * rng.random(mesh.nv) - 1.0))

    sv = Solver(64, device=device)
    # the literal FP64 form: the finite differences run the program the adjoint reverses
    sv.set_params(h_threshold=1e-5, dt_fixed=dt, fp64_literal=1)
    sv.upload_mesh(mesh)
    sv.set_gauges(LATTICE)

    def records(H0, depth):
        sv.set_depth(depth)
        sv.set_state(H0, s.Hu, s.Hv, 0.0)
        sv.step(n_steps)
        _, eta = sv.gauges()
        return eta

    t0 = time.perf_counter()
    eta_t = records(s.H + bump * wet, depth_t)
    J = lambda H0, depth: 0.5 * float(np.sum((records(H0, depth) - eta_t) ** 2))
    # the gradient at (H0, depth) = (s.H, mesh.depth)
    sv.set_depth(mesh.depth)
    sv.set_state(s.H, s.Hu, s.Hv, 0.0)
    _, eta = sv.adj_forward(n_steps, dt)
    g = sv.adj_backward(eta - eta_t, mesh.nv)
    t_adj = time.perf_counter() - t0
    dirs = []
    for k in range(n_dirs):
        kind = "H0" if k < n_dirs // 2 else "depth"
        d = rng.standard_normal(mesh.nc) * wet if kind == "H0" else rng.standard_normal(mesh.nv)
        gd = float(np.dot(g[kind], d))

        def f(e):
            if kind == "H0":
                return J(s.H + e * d, mesh.depth)
            return J(s.H, mesh.depth + e * d)

        steps = list(eps_sweep) if (k % (n_dirs // 2)) < sweep_dirs // 2 else [eps]
        fds = {e: (f(e) - f(-e)) / (2.0 * e) for e in steps}
        errs = {e: abs(gd - fd) / max(abs(fd), 1e-300) for e, fd in fds.items()}
        best = min(errs, key=errs.get)
        dirs.append({"kind": kind, "adjoint": gd, "fd": fds, "rel_err": errs, "best_eps": best,
                     "best_rel_err": errs[best]})
    sv.close()
    main = [d["rel_err"][eps] for d in dirs if eps in d["rel_err"]]
    return {"mesh_cells": mesh.nc, "n_steps": n_steps, "dt": dt, "gauges": len(LATTICE), "eps": eps,
            "directions": dirs, "median_rel_err_at_eps": float(np.median(main)),
            "max_rel_err_at_eps": float(np.max(main)),
            "max_best_rel_err": float(max(d["best_rel_err"] for d in dirs)),
            "adjoint_s": round(t_adj, 2), "total_s": round(time.perf_counter() - t0, 1)}


def _jsonable(x):
    if isinstance(x, dict):
        return {str(k): _jsonable(v) for k, v in x.items()}
    if isinstance(x, list):
        return [_jsonable(v) for v in x]
    if isinstance(x, float) and not math.isfinite(x):
        return str(x)
    return x


if __name__ == "__main__":
    print(json.dumps(_jsonable(fd_check())))
