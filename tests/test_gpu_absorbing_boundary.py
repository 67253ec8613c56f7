"""Absorbing boundary faces (vg_set_boundary with VG_BOUNDARY_ABSORBING) on the GPU
against the oracle's absorbing boundary (vo_set_boundary, pinned in
test_oracle_absorbing_boundary.py): the characteristic ghost of a sea at rest
(eta = 0) beyond the boundary."""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna
from gpu_helpers import FIELDS, rel_l2

pytestmark = pytest.mark.gpu


def _gpu(mesh, s, n, precision, edges, kinds, **prm):
    with volna.Solver(precision) as sv:
        sv.set_params(**prm)
        sv.upload_mesh(mesh)
        sv.set_boundary(edges, kinds)
        sv.set_state(s[0], s[1], s[2], 0.0)
        sv.step(n)
        H, Hu, Hv, t = sv.get_state()
        return dict(H=H, Hu=Hu, Hv=Hv, t=t, mass=sv.diagnostics()["mass"])


def _oracle(mesh, s, n, edges, kinds, **prm):
    om = O.OracleMesh.from_mesh(mesh)
    om.set_boundary(edges, [volna.BOUNDARY[k] if isinstance(k, str) else k for k in kinds])
    return om.run(O.params(**prm), (s[0], s[1], s[2], 0.0), n)


def _channel():
    m = I.strip_mesh(160, 12.0, width_cells=4)
    m.depth[:] = 1.0                                   # bed at -1 m: the sea at rest is eta = 0
    ends = I.boundary_edges(m, lambda mid: np.abs(np.abs(mid[:, 0]) - 6.0) < 1e-9)
    p = m.cell_points()
    H = 1.0 + 0.05 * np.exp(-((p[:, 0] - 2.0) / 0.5) ** 2)
    return m, ends, (H, np.zeros(m.nc), np.zeros(m.nc))


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_wave_meeting_absorbing_ends_matches_oracle(precision, tol):
    """A hump at rest (5 cm on 1 m of water, off centre) in a 12 m channel with
    absorbing ends, 600 steps (about 1.5 s): the right-going pulse is crossing
    the end.  Against the oracle; Hv (rounding noise about zero) against the
    scale of Hu."""
    m, ends, s = _channel()
    prm = dict(h_threshold=1e-6, cfl=0.9)
    kinds = ["absorbing"] * len(ends)
    g = _gpu(m, s, 600, precision, ends, kinds, **prm)
    r = _oracle(m, s, 600, ends, kinds, **prm)
    for f in ("H", "Hu"):
        assert rel_l2(g[f], r[f]) <= tol, f
    assert np.max(np.abs(g["Hv"] - r["Hv"])) <= tol * np.max(np.abs(r["Hu"]))


@pytest.mark.parametrize("precision", [64, 32])
def test_channel_returns_to_rest_through_absorbing_ends(precision):
    """After 1500 steps (about 3.8 s) both pulses have left: the water is back at
    the outer level to 1e-3 of the 5 cm hump and nearly still.  (A uniform current
    in the channel would not leave quietly: the sea beyond is at rest, and the
    condition stops it.)"""
    m, ends, s = _channel()
    g = _gpu(m, s, 1500, precision, ends, ["absorbing"] * len(ends), h_threshold=1e-6, cfl=0.9)
    assert np.max(np.abs(g["H"] - 1.0)) < 1e-3 and np.max(np.abs(g["Hu"])) < 1e-3


def test_coast_basin_absorbing_offshore_and_open_side():
    """Coast basin (6,500 triangles): the offshore arc r = 1000 km absorbing, one
    straight side open, the rest walls, FP64 against the oracle."""
    m = I.coast_mesh_with_cells(6500, seed=2)
    arc = I.boundary_edges(m, lambda mid: np.hypot(mid[:, 0], mid[:, 1]) > 0.999 * I.COAST_R_MAX)
    side = I.boundary_edges(m, lambda mid: np.abs(mid[:, 1]) < 1.0)
    assert len(arc) > 10 and len(side) > 10
    edges = np.concatenate([arc, side])
    kinds = ["absorbing"] * len(arc) + ["open"] * len(side)
    s0 = I.coast_initial_state(m)
    prm = dict(h_threshold=1e-3, cfl=0.9)
    g = _gpu(m, (s0.H, s0.Hu, s0.Hv), 60, 64, edges, kinds, **prm)
    r = _oracle(m, (s0.H, s0.Hu, s0.Hv), 60, edges, kinds, **prm)
    for f in FIELDS:
        assert rel_l2(g[f], r[f]) <= 1e-10, f


def test_batch_with_absorbing_boundary_equals_single():
    m, ends, s = _channel()
    kinds = ["absorbing"] * len(ends)
    with volna.Batch(32) as b:
        b.set_params(h_threshold=1e-6, cfl=0.9)
        mid = b.add_mesh(m, 2)
        b.set_boundary(mid, ends, kinds)
        s2 = (1.0 + 0.6 * (s[0] - 1.0), s[1], s[2])
        b.set_state(mid, 0, *s, 0.0)
        b.set_state(mid, 1, *s2, 0.0)
        b.step(120)
        for j, st in enumerate((s, s2)):
            H, Hu, Hv, _, _ = b.get_state(mid, j)
            ref = _gpu(m, st, 120, 32, ends, kinds, h_threshold=1e-6, cfl=0.9)
            for a, f in zip((H, Hu, Hv), FIELDS):
                np.testing.assert_array_equal(a, ref[f])


def test_unknown_kinds_are_rejected():
    m, ends, s = _channel()
    with volna.Solver(64) as sv:
        sv.upload_mesh(m)
        for bad in (0, 4, 7, -1):
            with pytest.raises(volna.VolnaError) as e:
                sv.set_boundary(ends, [bad] * len(ends))
            assert e.value.code == volna.VG_EINVAL


@pytest.mark.parametrize("dt", [2e-3, 0.0])
def test_adjoint_through_absorbing_ends_matches_oracle(dt):
    """A hump with a current toward the absorbing end of the channel, 60 steps
    (fixed dt, and the CFL step differentiated through its minimum): the GPU
    adjoint's gauge gradients (state and depth) equal the oracle's taped ones to
    1e-10; the absorbing ghost's bed term makes the depth gradient differ from the
    open boundary's."""
    m, ends, _ = _channel()
    p = m.cell_points()
    # the exponent is capped: a subnormal hump tail would make limiter ratios overflow
    hump = 0.05 * np.exp(-np.minimum(((p[:, 0] - 5.0) / 0.4) ** 2, 50.0))
    st = (1.0 + hump, 0.8 * hump + 0.01 * np.sin(3 * p[:, 0]),
          0.02 * hump * np.cos(5 * p[:, 1]) + 0.003 * np.sin(2 * p[:, 0] + 9 * p[:, 1]))
    gauges = np.array([[4.0, 0.0], [5.5, 0.05], [5.9, -0.05], [-5.9, 0.0]])
    cells = O.OracleMesh.from_mesh(m).locate(gauges)
    n_steps = 60
    W = np.random.default_rng(41).normal(size=(n_steps + 1, len(cells)))
    kinds = np.full(len(ends), volna.BOUNDARY["absorbing"], dtype=np.int32)
    out = {}
    for name, kk in (("absorbing", kinds), ("open", np.full(len(ends), volna.BOUNDARY["open"], dtype=np.int32))):
        with volna.Solver(64) as sv:
            sv.set_params(h_threshold=1e-5, cfl=0.9)
            sv.upload_mesh(m)
            sv.set_boundary(ends, kk)
            sv.set_gauges(gauges)
            sv.set_state(*st, 0.0)
            _, eta = sv.adj_forward(n_steps, dt)
            out[name] = (eta, sv.adj_backward(W, m.nv))
    eta, g = out["absorbing"]
    ad = O.ad_gauge_gradient(m, st, dt or None, n_steps, cells, W, h_threshold=1e-5, cfl=0.9, open_edges=ends,
                             boundary_kinds=kinds)
    np.testing.assert_allclose(eta, ad["eta"], rtol=0, atol=1e-13)
    for k_gpu, k_or in (("H0", "dH0"), ("Hu0", "dHu0"), ("Hv0", "dHv0"), ("depth", "ddepth")):
        err = np.linalg.norm(g[k_gpu] - ad[k_or]) / np.linalg.norm(ad[k_or])
        assert err <= 1e-10, (k_gpu, err)
    g_open = out["open"][1]
    assert np.linalg.norm(g_open["depth"] - g["depth"]) > 1e-3 * np.linalg.norm(g["depth"])
