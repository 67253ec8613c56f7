"""Pins of the oracle's absorbing boundary, a reading (the paper keeps walls,
Sec. 2.5, and defers other conditions to Dutykh et al. 2011): the characteristic
ghost of a sea at rest (eta = 0) beyond the boundary.  Pinned by the ghost state
solved independently from the Riemann invariants, still water, a wave that
leaves with far less reflection than through the open (zero-gradient) boundary,
and a raised basin that drains to the outer level."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I

G = 9.81


def test_absorbing_face_flux_is_the_flux_to_the_characteristic_ghost():
    """For random face states on random beds the absorbing flux equals the interior
    flux between the face state and the ghost built here from the Riemann
    invariants: u_n + 2c carried out from the face state, u_n - 2c = -2 c_0 brought
    in from the sea at rest (c_0 = sqrt(g max(0, -z))), tangential velocity kept."""
    rng = np.random.default_rng(17)
    n_checked = 0
    for _ in range(200):
        z = -rng.uniform(0.0, 50.0) if rng.uniform() < 0.9 else rng.uniform(0.0, 2.0)
        H = rng.uniform(0.05, 60.0)
        u, v = rng.normal(scale=3.0, size=2)
        th = rng.uniform(0, 2 * math.pi)
        n = (math.cos(th), math.sin(th))
        un, ut = u * n[0] + v * n[1], -u * n[1] + v * n[0]
        c, c0 = math.sqrt(G * H), math.sqrt(G * max(0.0, -z))
        Rp, Rm = un + 2.0 * c, -2.0 * c0
        ung, cg = 0.5 * (Rp + Rm), max(0.0, 0.25 * (Rp - Rm))
        Hg = cg * cg / G
        if Hg <= 1e-3:
            continue                                   # the interior path zeroes thin-film velocities
        ug, vg = ung * n[0] - ut * n[1], ung * n[1] + ut * n[0]
        Phi, PL, _, a = O.face_flux(G, 1e-6, (H, H * u, H * v), z, None, 0.0, n, wall="absorbing")
        ref, PLr, _, ar = O.face_flux(G, 1e-6, (H, H * u, H * v), z, (Hg, Hg * ug, Hg * vg), z, n)
        scale = max(1.0, float(np.max(np.abs(ref))))
        np.testing.assert_allclose(Phi, ref, rtol=0, atol=1e-11 * scale)
        assert PL == pytest.approx(PLr, abs=1e-11 * G * H * H)
        assert a == pytest.approx(ar, rel=1e-12)
        n_checked += 1
    assert n_checked > 150


def test_absorbing_ghost_at_rest_is_the_face_state():
    for z in (-0.5, -4.0, -4000.0):
        H = -z
        Phi, PL, _, a = O.face_flux(G, 1e-6, (H, 0.0, 0.0), z, None, 0.0, (0.6, 0.8), wall="absorbing")
        np.testing.assert_allclose(Phi, [0.0, 0.5 * G * H * H * 0.6, 0.5 * G * H * H * 0.8], rtol=1e-14, atol=0)
        assert a == pytest.approx(math.sqrt(G * H), rel=1e-14)


def test_still_water_with_all_boundaries_absorbing():
    m = I.flat_basin_mesh(20, 1.0, 2.0)
    om = O.OracleMesh.from_mesh(m)
    e = I.boundary_edges(m)
    om.set_boundary(e, [3] * len(e))
    s = I.lake_at_rest_state(m, 0.0)
    r = om.run(O.params(h_threshold=1e-6), (s.H, s.Hu, s.Hv, 0.0), 200)
    np.testing.assert_allclose(r["H"], s.H, rtol=0, atol=1e-12)
    assert np.max(np.abs(r["Hu"])) <= 1e-12 and np.max(np.abs(r["Hv"])) <= 1e-12


def _channel():
    m = I.strip_mesh(120, 12.0, width_cells=3)
    m.depth[:] = 1.0                                   # bed at -1 m: the sea at rest is eta = 0
    ends = I.boundary_edges(m, lambda mid: np.abs(np.abs(mid[:, 0]) - 6.0) < 1e-9)
    return m, ends


def test_wave_leaves_through_absorbing_ends_with_little_reflection():
    """The Gaussian hump (0.05 m on 1 m of water) of the open-boundary pin: at
    t = 6 s, when both pulses have reached the ends, absorbing ends leave far
    less behind than open ends (which reflect a few per cent of each pulse)."""
    m, ends = _channel()
    p = m.cell_points()
    H = 1.0 + 0.05 * np.exp(-(p[:, 0] / 0.5) ** 2)
    st = (H, np.zeros(m.nc), np.zeros(m.nc), 0.0)
    prm = O.params(h_threshold=1e-6, cfl=0.9, t_end=6.0)
    out = {}
    for kind in (2, 3):
        om = O.OracleMesh.from_mesh(m)
        om.set_boundary(ends, [kind] * len(ends))
        out[kind] = om.run(prm, st, 5000)
        assert out[kind]["t"] == pytest.approx(6.0)
    area = O.OracleMesh.from_mesh(m).get("area")
    dev = {k: float(np.max(np.abs(r["H"] - 1.0))) for k, r in out.items()}
    assert dev[3] <= 5e-5 and dev[3] <= 0.1 * dev[2]
    excess0 = np.sum(area * (H - 1.0))
    assert abs(np.sum(area * (out[3]["H"] - 1.0))) <= 1e-3 * excess0


def test_raised_basin_drains_to_the_outer_level():
    """Still water standing 2 cm above the outer sea level with absorbing
    boundaries flows out: the mean level falls to the outer level eta = 0 (after
    a small overshoot of the outflow) and the flow dies out."""
    m = I.flat_basin_mesh(16, 1.0, 1.0)
    om = O.OracleMesh.from_mesh(m)
    e = I.boundary_edges(m)
    om.set_boundary(e, [3] * len(e))
    s = I.lake_at_rest_state(m, 0.02)
    area = om.get("area")
    z = om.get("z")
    st = (s.H, s.Hu, s.Hv, 0.0)
    levels, speeds = [], []
    for _ in range(12):
        r = om.run(O.params(h_threshold=1e-6, cfl=0.9), st, 50)
        st = (r["H"], r["Hu"], r["Hv"], r["t"])
        levels.append(float(np.sum(area * (r["H"] + z)) / np.sum(area)))
        speeds.append(float(np.max(np.abs(r["Hu"]))))
    assert levels[0] < 0.015 and max(abs(x) for x in levels) < 0.02
    assert abs(levels[-1]) < 2e-4 and speeds[-1] < 0.05 * speeds[0]
