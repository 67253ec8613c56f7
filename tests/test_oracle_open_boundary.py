"""Pins of the oracle's open (transmissive) boundary, a reading (the paper keeps
walls, Sec. 2.5, and defers other conditions to Dutykh et al. 2011): ghost =
the cell's own state.  Pinned by the physical flux (closed form), uniform flow
through a channel, still water, and a wave that leaves the domain."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I

G = 9.81


def test_open_face_flux_is_the_physical_flux():
    rng = np.random.default_rng(5)
    for _ in range(50):
        H = rng.uniform(0.1, 3.0)
        u, v = rng.normal(size=2)
        th = rng.uniform(0, 2 * math.pi)
        n = (math.cos(th), math.sin(th))
        Phi, PL, PR, a = O.face_flux(G, 1e-6, (H, H * u, H * v), rng.normal(), None, 0.0, n, wall="open")
        un, ut = u * n[0] + v * n[1], -u * n[1] + v * n[0]
        F = np.array([H * un, H * un * un + 0.5 * G * H * H, H * un * ut])
        ref = np.array([F[0], F[1] * n[0] - F[2] * n[1], F[1] * n[1] + F[2] * n[0]])
        np.testing.assert_allclose(Phi, ref, rtol=1e-13, atol=1e-13)
        assert abs(PL) <= 1e-13 * G * H * H            # H* = H_f up to the rounding of (H + z) - z
        assert a == pytest.approx(abs(un) + math.sqrt(G * H), rel=1e-13)


def _strip(nx=60, length=6.0, width_cells=3):
    m = I.strip_mesh(nx, length, width_cells=width_cells)
    return m, I.boundary_edges(m, lambda mid: np.abs(np.abs(mid[:, 0]) - 0.5 * length) < 1e-9)


@pytest.mark.parametrize("u", [0.3, 4.0])        # subcritical and supercritical
def test_uniform_flow_through_open_channel(u):
    m, ends = _strip()
    om = O.OracleMesh.from_mesh(m)
    om.set_open(ends)
    z = om.get("z")
    H = 1.0 - z                                         # flat free surface at 1
    Hu = H * u
    r = om.run(O.params(h_threshold=1e-6, cfl=0.9), (H, Hu, np.zeros(m.nc), 0.0), 200)
    np.testing.assert_allclose(r["H"], H, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Hu"], Hu, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Hv"], 0.0, rtol=0, atol=1e-12)


def test_still_water_with_all_boundaries_open():
    m = I.flat_basin_mesh(20, 1.0, 2.0)
    om = O.OracleMesh.from_mesh(m)
    om.set_open(I.boundary_edges(m))
    s = I.lake_at_rest_state(m, 0.0)
    r = om.run(O.params(h_threshold=1e-6), (s.H, s.Hu, s.Hv, 0.0), 200)
    np.testing.assert_allclose(r["H"], s.H, rtol=0, atol=1e-12)
    assert np.max(np.abs(r["Hu"])) <= 1e-12 and np.max(np.abs(r["Hv"])) <= 1e-12


def test_wave_leaves_through_open_ends_and_reflects_from_walls():
    """A Gaussian hump (0.05 m) in a 1 m deep, 12 m long channel splits into two
    pulses that reach the ends after about 2 s.  At t = 6 s, with open ends the
    channel is nearly still and holds almost none of the excess water; with walls
    the pulses are back."""
    m, ends = _strip(nx=120, length=12.0)
    p = m.cell_points()
    H = 1.0 + 0.05 * np.exp(-(p[:, 0] / 0.5) ** 2)
    st = (H, np.zeros(m.nc), np.zeros(m.nc), 0.0)
    prm = O.params(h_threshold=1e-6, cfl=0.9, t_end=6.0)
    om = O.OracleMesh.from_mesh(m)
    om.set_open(ends)
    r_open = om.run(prm, st, 5000)
    walls = O.OracleMesh.from_mesh(m).run(prm, st, 5000)
    assert r_open["t"] == pytest.approx(6.0) and walls["t"] == pytest.approx(6.0)
    assert np.max(np.abs(r_open["H"] - 1.0)) <= 0.001     # 4 % of one outgoing pulse
    assert np.max(np.abs(walls["H"] - 1.0)) >= 0.01
    area = om.get("area")
    excess0 = np.sum(area * (H - 1.0))
    assert abs(np.sum(area * (r_open["H"] - 1.0))) <= 0.1 * excess0
    assert np.sum(area * walls["H"]) == pytest.approx(np.sum(area * H), rel=1e-13)
