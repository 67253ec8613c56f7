"""Pins of the oracle's moving bed (time-dependent bathymetry of Sec. 2.1, read
as a kinematic rupture applied between steps with H unchanged).

Each pin compares against something the oracle does not compute through
vo_bed_at: a mesh built directly on the final (or initial) depths, exact
conservation of mass, the lake-at-rest invariant, and the linearity of the
rise ramp.
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I


def _motion(m, amp=0.02, width=0.4, v=2.0, start=0.0):
    up, on = I.radial_rupture(m.xy, amp, 0.1, -0.05, width, v, start)
    return up, on


def test_bed_before_onset_and_after_rise_match_static_meshes():
    m = I.thacker_mesh(n=24)
    up, on = _motion(m, start=1.0)
    om = O.OracleMesh.from_mesh(m)
    z0 = om.get("z").copy()
    rise = 0.25
    z_before = om.bed_at(m.depth, up, on, rise, 0.999)
    np.testing.assert_array_equal(z_before, z0)
    z_after = om.bed_at(m.depth, up, on, rise, on.max() + rise + 1.0)
    final = O.OracleMesh(m.xy, m.tri, m.depth - up)
    np.testing.assert_array_equal(z_after, final.get("z"))


def test_bed_ramp_is_linear_in_time():
    """With one onset for all vertices, the bed halfway through the rise is the
    mean of the initial and final beds."""
    m = I.thacker_mesh(n=16)
    up = _motion(m)[0]
    on = np.full(m.nv, 0.5)
    om = O.OracleMesh.from_mesh(m)
    z0 = om.get("z").copy()
    z1 = O.OracleMesh(m.xy, m.tri, m.depth - up).get("z")
    zh = om.bed_at(m.depth, up, on, 0.2, 0.6)
    np.testing.assert_allclose(zh, 0.5 * (z0 + z1), rtol=0, atol=1e-15)


def test_instantaneous_uplift_equals_static_run_on_uplifted_bed():
    """rise = 0 and onset 0: the bed at the start time is already the final one,
    so the run is the static run on depth0 - uplift, bit for bit."""
    m = I.thacker_mesh(n=20)
    s = I.thacker_initial_state(m)
    up, _ = _motion(m)
    on = np.zeros(m.nv)
    prm = O.params(h_threshold=1e-5, cfl=0.9)
    a = O.OracleMesh.from_mesh(m).run(prm, (s.H, s.Hu, s.Hv, 0.0), 30, bed_motion=(m.depth, up, on, 0.0))
    b = O.OracleMesh(m.xy, m.tri, m.depth - up).run(prm, (s.H, s.Hu, s.Hv, 0.0), 30)
    for f in ("H", "Hu", "Hv"):
        np.testing.assert_array_equal(a[f], b[f])
    np.testing.assert_array_equal(a["dts"], b["dts"])


def test_moving_bed_conserves_mass():
    m = I.thacker_mesh(n=32)
    s = I.thacker_initial_state(m)
    up, on = _motion(m, amp=0.03)
    om = O.OracleMesh.from_mesh(m)
    M0 = om.mass(s.H)
    prm = O.params(h_threshold=1e-5, cfl=0.9)
    r = om.run(prm, (s.H, s.Hu, s.Hv, 0.0), 200, bed_motion=(m.depth, up, on, 0.1))
    assert r["neg_count"] == 0
    assert abs(om.mass(r["H"]) - M0) / M0 <= 1e-13
    # the bed did move under the water: the flow differs from a static run
    st = O.OracleMesh.from_mesh(m).run(prm, (s.H, s.Hu, s.Hv, 0.0), 200)
    assert np.max(np.abs(r["H"] - st["H"])) > 1e-4


def test_uniform_uplift_keeps_lake_at_rest():
    """The whole bowl rises uniformly under still water with dry margins: H is
    unchanged, the wet free surface rises with the bed, nothing moves."""
    m = I.thacker_mesh(n=24)
    s = I.lake_at_rest_state(m, 0.02)
    om = O.OracleMesh.from_mesh(m)
    up = np.full(m.nv, 0.05)
    on = np.zeros(m.nv)
    prm = O.params(h_threshold=1e-5, cfl=0.9)
    r = om.run(prm, (s.H, s.Hu, s.Hv, 0.0), 100, bed_motion=(m.depth, up, on, 0.5))
    assert r["t"] > 0.5                                   # the rise is complete
    assert np.max(np.abs(r["Hu"])) <= 1e-12 and np.max(np.abs(r["Hv"])) <= 1e-12
    np.testing.assert_allclose(r["H"], s.H, rtol=0, atol=1e-13)
    wet = s.H > 0
    eta = r["H"] + om.get("z")
    np.testing.assert_allclose(eta[wet], 0.02 + 0.05, rtol=0, atol=1e-13)
