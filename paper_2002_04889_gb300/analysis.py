"""Error decomposition of Sec. 4, driven by the GPU solver.

With the error at a gauge written as E(t) ~ C1(t) h^2 + C2(t) h^3 + C3(t) h^4
(leading dissipation, leading dispersion, secondary dissipation), three runs on
grids h, h/2, h/4 give a 3 x 3 linear system per time whose solution the paper
prints in closed form.  ``decompose`` evaluates those closed forms;
``thacker_decomposition`` runs Thacker's basin (Sec. 3: fixed dt proportional
to dx, centre gauge) on the three grids and returns E_k(t) and C1..C3(t).  The
paper's dt = 0.45 dx is stated for its own Courant convention; on these
triangles the CFL bound |K| / (3 l a) is about dx / 6 for a ~1 m/s wave, so the
default here is dt = 0.1 dx (0.6 of that bound).
"""
from __future__ import annotations

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


def thacker_decomposition(n_coarse: int = 168, t_fin: float = 10.0, dt_over_dx: float = 0.1,
                          half_width: float = 2.0, gauge=(0.0, 0.0), device: int = 0) -> dict:
    """Thacker's basin on n, 2n, 4n squares per side (h = 2 half_width / n), FP64,
    dt = dt_over_dx * dx, the gauge recorded at common times (every 1, 2, 4 steps).
    Returns dict(h, t, eta[3, T], exact[T], E[3, T], C1, C2, C3)."""
    runs = []
    for k in range(3):
        n = n_coarse * 2 ** k
        mesh = inputs.thacker_mesh(n=n, half_width=half_width)
        s = inputs.thacker_initial_state(mesh)
        dx = 2.0 * half_width / n
        dt = dt_over_dx * dx
        n_steps = int(round(t_fin / dt))
        with Solver(64, device=device) as sv:
            sv.set_params(h_threshold=1e-5, dt_fixed=dt, gauge_every=2 ** k)
            sv.upload_mesh(mesh)
            sv.set_gauges(np.array([gauge], dtype=np.float64))
            sv.set_state(s.H, s.Hu, s.Hv, 0.0)
            sv.step(n_steps)
            t, eta = sv.gauges()
        runs.append((t, eta[:, 0]))
    T = min(len(r[0]) for r in runs)
    t = runs[0][0][:T]
    eta = np.stack([r[1][:T] for r in runs])
    exact = np.array([float(inputs.thacker_free_surface(gauge[0], gauge[1], tt)) for tt in t])
    E = np.abs(eta - exact[None, :])
    h = 2.0 * half_width / n_coarse
    C1, C2, C3 = decompose(E[0], E[1], E[2], h)
    return dict(h=h, t=t, eta=eta, exact=exact, E=E, C1=C1, C2=C2, C3=C3)
