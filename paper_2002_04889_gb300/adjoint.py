"""torch.autograd bridge of the discrete adjoint (vg_adj_forward / vg_adj_backward).

``gauge_records(solver, H0, Hu0, Hv0, depth_v, n_steps, dt)`` runs the FP64 solver
with the fixed time step dt, or with the CFL time step of every step for dt = 0
(differentiated through as well), and returns the gauge records
eta[n_steps + 1, G] as a differentiable function of the initial state and the
per-vertex bathymetry.
Its backward is the hand-written CUDA adjoint with sqrt(N) checkpointing; the
tensors only cross the C ABI (argument marshalling).
"""
from __future__ import annotations

import numpy as np
import torch

from . import volna


class GaugeRecords(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H0, Hu0, Hv0, depth_v, solver, n_steps, dt, checkpoint_every):
        if solver.precision != 64:
            raise ValueError("the adjoint runs in FP64 solvers")
        to_np = lambda x: x.detach().to(torch.float64).cpu().numpy()
        solver.set_depth(to_np(depth_v))
        solver.set_state(to_np(H0), to_np(Hu0), to_np(Hv0), 0.0)
        _, eta = solver.adj_forward(int(n_steps), float(dt), int(checkpoint_every))
        ctx.solver = solver
        ctx.nv = depth_v.numel()
        ctx.device = H0.device
        return torch.as_tensor(eta, dtype=torch.float64, device=H0.device)

    @staticmethod
    def backward(ctx, g_eta):
        g = ctx.solver.adj_backward(g_eta.detach().to(torch.float64).cpu().numpy(), ctx.nv)
        t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=ctx.device)
        return t(g["H0"]), t(g["Hu0"]), t(g["Hv0"]), t(g["depth"]), None, None, None, None


def gauge_records(solver, H0, Hu0, Hv0, depth_v, n_steps: int, dt: float, checkpoint_every: int = 0):
    return GaugeRecords.apply(H0, Hu0, Hv0, depth_v, solver, n_steps, dt, checkpoint_every)


def cell_bed(tri: torch.Tensor, depth_v: torch.Tensor) -> torch.Tensor:
    """Cell bed z = -(mean of the three vertex depths), differentiable (user-side
    initial-condition algebra; the solver computes the same map internally)."""
    return -(depth_v[tri[:, 0]] + depth_v[tri[:, 1]] + depth_v[tri[:, 2]]) / 3.0
