"""Closed-form solutions used as pins for the oracle.  TEST INFRASTRUCTURE.

* Thacker's periodic paraboloid basin (Sec. 3): the free surface and velocity
  in closed form.  Readings of the printed formula: the function the paper
  calls h(r, t) is the free surface eta plus -z(r), i.e. the water depth; the
  velocities are written in the printed text about (L/2, L/2), the corner of a
  [0, L] domain, while the paper's domain is [-L/2, L/2]^2, so they are taken
  about the origin: u = omega A sin(omega t) x / (2 (1 - A cos(omega t))).
* Ritter's dam break over a dry bed (textbook special case that exercises the
  dry-bed wave speeds): h = (2 c0 - x/t)^2 / (9 g) on -c0 t <= x <= 2 c0 t.
* The error decomposition of Sec. 4: the printed closed forms for C1, C2, C3.
"""
from __future__ import annotations

import math

import numpy as np


def thacker_constants(h0=0.1, alpha=1.0, r0=0.8, g=9.81):
    omega = math.sqrt(8.0 * g * h0) / alpha
    A = (alpha * alpha - r0 * r0) / (alpha * alpha + r0 * r0)
    return omega, A


def thacker_eta(x, y, t, h0=0.1, alpha=1.0, r0=0.8, g=9.81):
    """Free-surface elevation eta(r, t) of Sec. 3 (before clipping by the bed)."""
    omega, A = thacker_constants(h0, alpha, r0, g)
    r2 = np.asarray(x) ** 2 + np.asarray(y) ** 2
    c = 1.0 - A * math.cos(omega * t)
    return h0 * (math.sqrt(1.0 - A * A) / c - 1.0 - (r2 / alpha ** 2) * ((1.0 - A * A) / c ** 2 - 1.0))


def thacker_bed(x, y, h0=0.1, alpha=1.0):
    """Bed z(r) = -h0 (1 - r^2 / alpha^2) (Sec. 3)."""
    r2 = np.asarray(x) ** 2 + np.asarray(y) ** 2
    return -h0 * (1.0 - r2 / alpha ** 2)


def thacker_depth(x, y, t, **kw):
    """Water depth max(0, eta - z)."""
    kb = {k: kw[k] for k in ("h0", "alpha") if k in kw}
    return np.maximum(0.0, thacker_eta(x, y, t, **kw) - thacker_bed(x, y, **kb))


def thacker_velocity(x, y, t, h0=0.1, alpha=1.0, r0=0.8, g=9.81):
    omega, A = thacker_constants(h0, alpha, r0, g)
    c = 1.0 - A * math.cos(omega * t)
    f = omega * A * math.sin(omega * t) / (2.0 * c)
    return f * np.asarray(x), f * np.asarray(y)


def ritter_depth(x, t, h_left, g=9.81):
    """Depth of Ritter's dry-bed dam break at time t > 0 (dam at x = 0)."""
    c0 = math.sqrt(g * h_left)
    x = np.asarray(x, dtype=np.float64)
    xi = x / t
    h = np.where(xi <= -c0, h_left, np.where(xi >= 2.0 * c0, 0.0, (2.0 * c0 - xi) ** 2 / (9.0 * g)))
    return h


def error_decomposition(E1, E2, E3, h):
    """C1, C2, C3 of Sec. 4 from the errors on grids h, h/2, h/4 (printed closed forms)."""
    E1, E2, E3 = (np.asarray(e, dtype=np.float64) for e in (E1, E2, E3))
    C1 = (E1 - 24.0 * E2 + 128.0 * E3) / (3.0 * h ** 2)
    C2 = -2.0 * (E1 - 20.0 * E2 + 64.0 * E3) / h ** 3
    C3 = 8.0 * (E1 - 12.0 * E2 + 32.0 * E3) / (3.0 * h ** 4)
    return C1, C2, C3
