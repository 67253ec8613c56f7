"""Pins of the oracle's discrete adjoint (tape AD of the oracle's arithmetic)
against finite differences of the oracle's forward run (FP64).

J is piecewise smooth: the min/max of the wave speeds (Sec. 2.2) and of the
Barth-Jespersen limiter (Sec. 2.4) switch, and near-equal neighbour states put
such kinks close together, so the step is small (1e-9).  The adjoint must match
the central difference; if a kink still lies inside the step (MUSCL only), it
must lie between the two one-sided differences.
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I


def _setup(n=12, n_steps=15):
    m = I.thacker_mesh(n=n, half_width=1.2)
    s = I.thacker_initial_state(m)
    om = O.OracleMesh.from_mesh(m)
    gauges = np.array([[0.0, 0.0], [0.3, 0.1], [-0.2, 0.25], [0.1, -0.4]])
    cells = om.locate(gauges)
    dx = 2.4 / n
    dt = 0.1 * dx
    rng = np.random.default_rng(5)
    w = rng.normal(size=(n_steps + 1, len(cells)))
    # momentum only where the water is deep (velocities stay moderate), and in both
    # components: an identically zero field sits on the limiter's D = 0 branch, where
    # the directional derivative exists but is not linear in the direction
    deep = s.H > 2e-2
    p = m.cell_points()
    st = (s.H, s.Hu + 1e-3 * np.sin(3 * p[:, 0]) * deep, s.Hv + 1e-3 * np.cos(2 * p[:, 1]) * deep)
    return m, st, cells, dt, n_steps, w


def _J(m, state, depth, cells, dt, n_steps, w, order=2):
    om = O.OracleMesh(m.xy, m.tri, depth)
    r = om.run(O.params(dt_fixed=dt, order=order), (state[0], state[1], state[2], 0.0), n_steps,
               gauge_cells=cells)
    z = om.get("z")
    eta0 = state[0][cells] + z[cells]
    return float(np.sum(w[0] * eta0) + np.sum(w[1:] * r["gauges"]))


@pytest.mark.parametrize("order", [1, 2])
def test_oracle_adjoint_matches_forward_and_finite_differences(order):
    m, st, cells, dt, n_steps, w = _setup()
    ad = O.ad_gauge_gradient(m, st, dt, n_steps, cells, w, h_threshold=1e-5, order=order)
    J0 = _J(m, st, m.depth, cells, dt, n_steps, w, order)
    assert ad["J"] == pytest.approx(J0, rel=1e-13, abs=1e-15)      # the taped run is the oracle's run
    rng = np.random.default_rng(7)
    wet = st[0] > 1e-3
    eps = 1e-9             # kinks (Zhou speeds, limiter, face-depth threshold) are dense: a small step stays on one piece
    n_central = 0
    for kind in ("H", "Hu", "Hv", "depth"):
        for _ in range(4):
            if kind == "depth":
                d = rng.normal(size=m.nv)
                grad_dot = float(np.dot(ad["ddepth"], d))
            else:
                d = rng.normal(size=m.nc) * wet
                grad_dot = float(np.dot(ad["d" + kind + "0"], d))

            def shifted(e):
                if kind == "depth":
                    return _J(m, st, m.depth + e * d, cells, dt, n_steps, w, order)
                k = ("H", "Hu", "Hv").index(kind)
                stt = [a.copy() for a in st]
                stt[k] = stt[k] + e * d
                return _J(m, stt, m.depth, cells, dt, n_steps, w, order)
            jp, jm = shifted(eps), shifted(-eps)
            fd = (jp - jm) / (2 * eps)
            tol = 2e-6 * max(1.0, abs(fd))
            if abs(grad_dot - fd) <= tol:
                n_central += 1
                continue
            assert order == 2, (kind, grad_dot, fd)
            fwd, bwd = (jp - J0) / eps, (J0 - jm) / eps
            lo, hi = min(fwd, bwd) - tol, max(fwd, bwd) + tol
            assert lo <= grad_dot <= hi, (kind, grad_dot, fwd, bwd)
    assert n_central >= 12


def _J_cfl(m, state, depth, cells, n_steps, w, cfl=0.9):
    om = O.OracleMesh(m.xy, m.tri, depth)
    r = om.run(O.params(cfl=cfl), (state[0], state[1], state[2], 0.0), n_steps, gauge_cells=cells)
    z = om.get("z")
    eta0 = state[0][cells] + z[cells]
    return float(np.sum(w[0] * eta0) + np.sum(w[1:] * r["gauges"])), r["dts"]


def test_oracle_adjoint_through_the_cfl_time_step():
    """With the adaptive CFL step (Sec. 2.3 rule) every step's dt depends on the
    state through the minimum over cells; the taped adjoint differentiates
    through it and matches central differences of the adaptive forward run."""
    m, st, cells, _, n_steps, w = _setup()
    ad = O.ad_gauge_gradient(m, st, None, n_steps, cells, w, h_threshold=1e-5, cfl=0.9)
    J0, dts = _J_cfl(m, st, m.depth, cells, n_steps, w)
    assert ad["J"] == pytest.approx(J0, rel=1e-13, abs=1e-15)
    np.testing.assert_array_equal(ad["dts"], dts)
    assert np.ptp(dts) > 0                         # the step does change from step to step
    rng = np.random.default_rng(11)
    wet = st[0] > 1e-3
    eps = 1e-8
    n_ok = 0
    for kind in ("H", "Hu", "depth"):
        for _ in range(4):
            if kind == "depth":
                d = rng.normal(size=m.nv)
                gd = float(np.dot(ad["ddepth"], d))
                f = lambda e: _J_cfl(m, st, m.depth + e * d, cells, n_steps, w)[0]
            else:
                d = rng.normal(size=m.nc) * wet
                gd = float(np.dot(ad["d" + kind + "0"], d))
                k = ("H", "Hu").index(kind)

                def f(e, k=k, d=d):
                    stt = [a.copy() for a in st]
                    stt[k] = stt[k] + e * d
                    return _J_cfl(m, stt, m.depth, cells, n_steps, w)[0]
            jp, jm = f(eps), f(-eps)
            fd = (jp - jm) / (2 * eps)
            if abs(gd - fd) <= 2e-6 * max(1.0, abs(fd)):
                n_ok += 1
            else:
                fwd, bwd = (jp - J0) / eps, (J0 - jm) / eps
                assert min(fwd, bwd) - 2e-6 <= gd <= max(fwd, bwd) + 2e-6, (kind, gd, fwd, bwd)
    assert n_ok >= 9


def _J_bed(m, state, cells, n_steps, w, motion, depth=None):
    om = O.OracleMesh(m.xy, m.tri, m.depth if depth is None else depth)
    up, on, rise = motion
    d0 = m.depth if depth is None else depth
    z0 = om.bed_at(d0, up, on, rise, 0.0)
    eta0 = state[0][cells] + z0[cells]
    r = om.run(O.params(cfl=0.9), (state[0], state[1], state[2], 0.0), n_steps, gauge_cells=cells,
               bed_motion=(d0, up, on, rise))
    return float(np.sum(w[0] * eta0) + np.sum(w[1:] * r["gauges"]))


def test_oracle_adjoint_with_a_moving_bed():
    """Moving bed (a Gaussian uplift spreading from a point, rising over 0.05 s)
    under adaptive steps: the taped gradients with respect to the uplift and the
    onset times (the rupture history) match central differences."""
    m, st, cells, _, n_steps, w = _setup()
    up, on = I.radial_rupture(m.xy, 0.01, 0.1, -0.05, 0.4, 2.0, 0.0)
    motion = (up, on, 0.05)
    ad = O.ad_gauge_gradient(m, st, None, n_steps, cells, w, h_threshold=1e-5, cfl=0.9, bed_motion=motion)
    J0 = _J_bed(m, st, cells, n_steps, w, motion)
    assert ad["J"] == pytest.approx(J0, rel=1e-13, abs=1e-15)
    rng = np.random.default_rng(13)
    eps = 1e-8
    n_ok = 0
    for kind in ("uplift", "onset", "depth"):
        for _ in range(4):
            d = rng.normal(size=m.nv)
            if kind == "uplift":
                d = d * (up > 1e-4)
                gd = float(np.dot(ad["duplift"], d))
                f = lambda e, d=d: _J_bed(m, st, cells, n_steps, w, (up + e * d, on, 0.05))
            elif kind == "onset":
                d = d * 0.01
                gd = float(np.dot(ad["donset"], d))
                f = lambda e, d=d: _J_bed(m, st, cells, n_steps, w, (up, on + e * d, 0.05))
            else:
                gd = float(np.dot(ad["ddepth"], d))
                f = lambda e, d=d: _J_bed(m, st, cells, n_steps, w, motion, depth=m.depth + e * d)
            jp, jm = f(eps), f(-eps)
            fd = (jp - jm) / (2 * eps)
            if abs(gd - fd) <= 2e-6 * max(1.0, abs(fd)):
                n_ok += 1
            else:
                fwd, bwd = (jp - J0) / eps, (J0 - jm) / eps
                assert min(fwd, bwd) - 2e-6 <= gd <= max(fwd, bwd) + 2e-6, (kind, gd, fwd, bwd)
    assert n_ok >= 9
    assert np.max(np.abs(ad["donset"])) > 0 and np.max(np.abs(ad["duplift"])) > 0


@pytest.mark.parametrize("absorbing", [False, True])
def test_oracle_adjoint_with_open_boundaries(absorbing):
    """Open (transmissive) boundary faces on two sides of a 0.1 m basin whose hump
    drifts out through them, CFL steps: the taped gradients match central
    differences of the open-boundary run.  absorbing: the x side takes the
    characteristic ghost of a sea at rest instead (its c_0 = sqrt(g h) brings the
    bed into the ghost), the y side stays open."""
    m0 = I.flat_basin_mesh(12, 1.2, 0.1)
    # a gentle slope and curvature: on a perfectly flat bed every face is a tie of
    # max(z_L, z_R), where the depth derivative does not exist
    m = I.Mesh(m0.xy, m0.tri, 0.1 + 0.02 * m0.xy[:, 0] + 0.01 * m0.xy[:, 1] ** 2, name="sloped", meta=m0.meta)
    s = I.gaussian_hump_state(m, 0.0, 0.02, 0.6, -0.4, 0.5)
    p = m.cell_points()
    st = (s.H, 0.05 * s.H * (1.0 + 0.3 * np.sin(2 * p[:, 1])), -0.03 * s.H)
    om0 = O.OracleMesh.from_mesh(m)
    cells = om0.locate(np.array([[0.0, 0.0], [0.8, -0.8], [0.9, 0.3], [-0.5, -0.9]]))
    n_steps = 15
    w = np.random.default_rng(5).normal(size=(n_steps + 1, len(cells)))
    edges = np.concatenate([I.boundary_edges(m, lambda mid: mid[:, 0] > 1.19),
                            I.boundary_edges(m, lambda mid: mid[:, 1] < -1.19)])
    assert len(edges) > 5
    n_x = len(I.boundary_edges(m, lambda mid: mid[:, 0] > 1.19))
    kinds = np.array([3 if absorbing and e < n_x else 2 for e in range(len(edges))], dtype=np.int32)
    ad = O.ad_gauge_gradient(m, st, None, n_steps, cells, w, h_threshold=1e-5, cfl=0.9, open_edges=edges,
                             boundary_kinds=kinds)

    def J(state, depth):
        om = O.OracleMesh(m.xy, m.tri, depth)
        om.set_boundary(edges, kinds)
        r = om.run(O.params(cfl=0.9), (state[0], state[1], state[2], 0.0), n_steps, gauge_cells=cells)
        z = om.get("z")
        return float(np.sum(w[0] * (state[0][cells] + z[cells])) + np.sum(w[1:] * r["gauges"]))

    J0 = J(st, m.depth)
    assert ad["J"] == pytest.approx(J0, rel=1e-13, abs=1e-15)
    closed = O.ad_gauge_gradient(m, st, None, n_steps, cells, w, h_threshold=1e-5, cfl=0.9)
    assert np.linalg.norm(closed["dH0"] - ad["dH0"]) > 1e-6 * np.linalg.norm(ad["dH0"])
    if absorbing:
        opened = O.ad_gauge_gradient(m, st, None, n_steps, cells, w, h_threshold=1e-5, cfl=0.9, open_edges=edges)
        for k in ("dH0", "ddepth"):
            assert np.linalg.norm(opened[k] - ad[k]) > 1e-6 * np.linalg.norm(ad[k]), k
    # the state is nearly uniform, so limiter and wave-speed min/max kinks are dense:
    # central differences approach the adjoint as the step shrinks (the plateau)
    rng = np.random.default_rng(17)
    n_ok = 0
    for kind in ("H", "Hu", "depth"):
        for _ in range(3):
            if kind == "depth":
                d = rng.normal(size=m.nv) * 1e-2
                gd = float(np.dot(ad["ddepth"], d))
                f = lambda e, d=d: J(st, m.depth + e * d)
            else:
                d = rng.normal(size=m.nc)
                gd = float(np.dot(ad["d" + kind + "0"], d))
                k = ("H", "Hu", "Hv").index(kind)

                def f(e, k=k, d=d):
                    stt = [a.copy() for a in st]
                    stt[k] = stt[k] + e * d
                    return J(stt, m.depth)
            errs = [abs(gd - (f(eps) - f(-eps)) / (2 * eps)) / max(1e-12, abs(gd)) for eps in (1e-7, 1e-8, 1e-9)]
            n_ok += min(errs) <= 2e-4
    assert n_ok >= 8, n_ok
