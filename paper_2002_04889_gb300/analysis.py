"""Accuracy studies of Sec. 3 and Sec. 4, driven by the GPU solver (FP64).

* ``thacker_convergence``: the convergence study of Sec. 3 -- Thacker's basin on
  several grids, the centre gauge's error max over t in [0, t_fin] (the paper's
  "Linf norm at 10 s" read as the sup-norm of the centre-gauge error curve up to
  10 s) and the domain L1 / Linf errors of eta over the wet interior at t_fin,
  with the observed orders between successive grids.
* ``decompose`` / ``thacker_decomposition``: the error decomposition of Sec. 4.
  With the error at a gauge written as E(t) ~ C1(t) h^2 + C2(t) h^3 + C3(t) h^4
  (leading dissipation, leading dispersion, secondary dissipation), three runs
  on grids h, h/2, h/4 give a 3 x 3 linear system per time whose solution the
  paper prints in closed form.

Time step: the paper's dt = 0.45 dx (Sec. 3, "CFL = 0.45" in Sec. 4) is taken as
a cap on the step of the CFL rule, not as the step itself: on these triangles the
rule's CFL-1 step is about 0.06 dx, and a fixed step breaks down through the thin
films of the moving shoreline well below 0.45 dx.  The grids' gauge records sit at
different times, so the finer grids' records are interpolated linearly to the
coarsest grid's record times (the interpolation error, O(dt^2), is orders of
magnitude below the errors studied).

Errors are taken against Thacker's closed form at the centroid of the cell that
holds the gauge: a gauge reads its cell's eta (piecewise constant), and the offset
between the centroid and the gauge point is a sampling error whose constant
depends on where the centroid falls on each grid, not an error of the scheme.

``python -m paper_2002_04889_gb300.analysis`` runs both studies on cuda:0 and
prints one JSON object.
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import inputs
from .volna import Solver


def decompose(E1, E2, E3, h: float):
    """C1, C2, C3 from the errors on grids h, h/2, h/4 (Sec. 4 closed forms)."""
    E1, E2, E3 = (np.asarray(e, dtype=np.float64) for e in (E1, E2, E3))
    C1 = (E1 - 24.0 * E2 + 128.0 * E3) / (3.0 * h * h)
    C2 = -2.0 * (E1 - 20.0 * E2 + 64.0 * E3) / h ** 3
    C3 = 8.0 * (E1 - 12.0 * E2 + 32.0 * E3) / (3.0 * h ** 4)
    return C1, C2, C3


def thacker_run(n: int, t_fin: float, half_width: float = 2.0, gauge=(0.0, 0.0), cfl: float = 0.9,
                dt_max_over_dx: float = 0.45, device: int = 0) -> dict:
    """Thacker's basin (Sec. 3) on n x n squares of [-half_width, half_width]^2, FP64,
    CFL step capped at dt_max_over_dx * dx, to t_fin.  Returns the gauge records
    (t, eta, with the initial record), the closed form at the gauge cell's
    centroid at those times, and the interior (r < 0.5) L1 / Linf errors of eta at
    t_fin."""
    mesh = inputs.thacker_mesh(n=n, half_width=half_width)
    s = inputs.thacker_initial_state(mesh)
    dx = 2.0 * half_width / n
    with Solver(64, device=device) as sv:
        sv.set_params(h_threshold=1e-5, cfl=cfl, dt_max=dt_max_over_dx * dx)
        sv.upload_mesh(mesh)
        cell = int(sv.set_gauges(np.array([gauge], dtype=np.float64))[0])
        sv.set_state(s.H, s.Hu, s.Hv, 0.0)
        sv.advance_to(t_fin)
        t, eta = sv.gauges()
        H, _, _, t_end = sv.get_state()
        steps = sv.diagnostics()["steps"]
    p = mesh.cell_points()
    xc, yc = p[cell]
    exact = np.array([float(inputs.thacker_free_surface(xc, yc, tt)) for tt in t])
    z = -mesh.vertex_mean(mesh.depth)
    err = np.abs(H + z - inputs.thacker_free_surface(p[:, 0], p[:, 1], t_end))
    inner = p[:, 0] ** 2 + p[:, 1] ** 2 < 0.25
    return dict(n=n, dx=dx, cells=mesh.nc, steps=int(steps), t=t, eta=eta[:, 0], exact=exact,
                gauge_err=np.abs(eta[:, 0] - exact), l1=float(err[inner].mean()), linf=float(err[inner].max()))


def thacker_convergence(dxs=(0.048, 0.024, 0.012, 0.006), t_fin: float = 10.0, **kw) -> dict:
    """The convergence study of Sec. 3 on grids dx (n = 4 / dx squares per side)."""
    runs = [thacker_run(int(round(4.0 / dx)), t_fin, **kw) for dx in dxs]
    cen = [float(r["gauge_err"].max()) for r in runs]
    l1 = [r["l1"] for r in runs]
    linf = [r["linf"] for r in runs]
    order = lambda e: [math.log(e[k] / e[k + 1]) / math.log(runs[k]["dx"] / runs[k + 1]["dx"])
                       for k in range(len(e) - 1)]
    return dict(t_fin=t_fin, dx=[r["dx"] for r in runs], cells=[r["cells"] for r in runs],
                steps=[r["steps"] for r in runs], centre_gauge_linf=cen, centre_gauge_order=order(cen),
                interior_l1=l1, interior_l1_order=order(l1), interior_linf=linf,
                interior_linf_order=order(linf))


def thacker_decomposition(n_coarse: int = 167, t_fin: float = 10.0, half_width: float = 2.0, gauge=(0.0, 0.0),
                          **kw) -> dict:
    """Thacker's basin on n, 2n, 4n squares per side (h = 2 half_width / n), the
    gauge's error E_k(t) on the coarse grid's record times, and C1..C3(t).
    Returns dict(h, t, E[3, T], C1, C2, C3, eta[3, T], exact[3, T])."""
    runs = [thacker_run(n_coarse * 2 ** k, t_fin, half_width=half_width, gauge=gauge, **kw) for k in range(3)]
    t = runs[0]["t"]
    t = t[t <= min(r["t"][-1] for r in runs)]
    eta = np.stack([np.interp(t, r["t"], r["eta"]) for r in runs])
    exact = np.stack([np.interp(t, r["t"], r["exact"]) for r in runs])
    E = np.abs(eta - exact)
    h = 2.0 * half_width / n_coarse
    C1, C2, C3 = decompose(E[0], E[1], E[2], h)
    return dict(h=h, t=t, eta=eta, exact=exact, E=E, C1=C1, C2=C2, C3=C3)


def decomposition_summary(r: dict) -> dict:
    """Time averages of |E_j| and of |C_k h_j^(k+1)| on each grid j (which term
    dominates where)."""
    out = {"h": r["h"]}
    for j in range(3):
        hj = r["h"] / 2 ** j
        terms = [np.abs(r["C1"]) * hj ** 2, np.abs(r["C2"]) * hj ** 3, np.abs(r["C3"]) * hj ** 4]
        out[f"grid_{j}"] = {"h": hj, "mean_abs_E": float(r["E"][j].mean()),
                            "mean_abs_C1h2": float(terms[0].mean()), "mean_abs_C2h3": float(terms[1].mean()),
                            "mean_abs_C3h4": float(terms[2].mean())}
    return out


if __name__ == "__main__":
    conv = thacker_convergence()
    dec = thacker_decomposition()
    print(json.dumps({"convergence": conv, "decomposition": decomposition_summary(dec)}))
