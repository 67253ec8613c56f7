"""Open (transmissive) boundary faces (vg_set_open_boundary) on the GPU against
the oracle's open boundary (vo_set_open, pinned in test_oracle_open_boundary.py)."""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna
from gpu_helpers import FIELDS, rel_l2

pytestmark = pytest.mark.gpu


def _gpu(mesh, s, n, precision, edges, **prm):
    with volna.Solver(precision) as sv:
        sv.set_params(**prm)
        sv.upload_mesh(mesh)
        if edges is not None:
            sv.set_open_boundary(edges)
        sv.set_state(s[0], s[1], s[2], 0.0)
        sv.step(n)
        H, Hu, Hv, t = sv.get_state()
        return dict(H=H, Hu=Hu, Hv=Hv, t=t, mass=sv.diagnostics()["mass"])


def _oracle(mesh, s, n, edges, **prm):
    om = O.OracleMesh.from_mesh(mesh)
    om.set_open(edges)
    return om.run(O.params(**prm), (s[0], s[1], s[2], 0.0), n)


def _strip_wave():
    m = I.strip_mesh(160, 12.0, width_cells=4)
    ends = I.boundary_edges(m, lambda mid: np.abs(np.abs(mid[:, 0]) - 6.0) < 1e-9)
    p = m.cell_points()
    H = 1.0 + 0.05 * np.exp(-((p[:, 0] - 2.0) / 0.5) ** 2)
    return m, ends, (H, 0.3 * H, np.zeros(m.nc))


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_outgoing_wave_matches_oracle(precision, tol):
    """A hump drifting at 0.3 m/s in a 12 m channel, open at both ends, 1500
    steps (about 4 s): both pulses have reached the ends and left.  The flow is
    along the channel, so Hv (rounding noise about zero) is compared against the
    scale of Hu."""
    m, ends, s = _strip_wave()
    prm = dict(h_threshold=1e-6, cfl=0.9)
    g = _gpu(m, s, 1500, precision, ends, **prm)
    r = _oracle(m, s, 1500, ends, **prm)
    for f in ("H", "Hu"):
        assert rel_l2(g[f], r[f]) <= tol, f
    assert np.max(np.abs(g["Hv"] - r["Hv"])) <= tol * np.max(np.abs(r["Hu"]))
    area = O.OracleMesh.from_mesh(m).get("area")
    assert g["mass"] < np.sum(area * s[0]) - 1e-3          # water left through the ends


def test_coast_basin_open_offshore_fp64():
    """Coast basin (6,500 triangles): the offshore arc r = 1000 km open, the rest walls."""
    m = I.coast_mesh_with_cells(6500, seed=2)
    arc = I.boundary_edges(m, lambda mid: np.hypot(mid[:, 0], mid[:, 1]) > 0.999 * I.COAST_R_MAX)
    assert len(arc) > 10
    s0 = I.coast_initial_state(m)
    prm = dict(h_threshold=1e-3, cfl=0.9)
    g = _gpu(m, (s0.H, s0.Hu, s0.Hv), 60, 64, arc, **prm)
    r = _oracle(m, (s0.H, s0.Hu, s0.Hv), 60, arc, **prm)
    for f in FIELDS:
        assert rel_l2(g[f], r[f]) <= 1e-10, f


def test_batch_with_open_boundary_equals_single():
    m, ends, s = _strip_wave()
    with volna.Batch(32) as b:
        b.set_params(h_threshold=1e-6, cfl=0.9)
        mid = b.add_mesh(m, 2)
        b.set_open_boundary(mid, ends)
        b.set_state(mid, 0, *s, 0.0)
        b.set_state(mid, 1, s[0], -s[1], s[2], 0.0)
        b.step(120)
        for j, st in enumerate((s, (s[0], -s[1], s[2]))):
            H, Hu, Hv, _, _ = b.get_state(mid, j)
            ref = _gpu(m, st, 120, 32, ends, h_threshold=1e-6, cfl=0.9)
            for a, f in zip((H, Hu, Hv), FIELDS):
                np.testing.assert_array_equal(a, ref[f])


def test_reset_to_walls_and_invalid_edge():
    m, ends, s = _strip_wave()
    walls = _gpu(m, s, 50, 64, None, h_threshold=1e-6)
    with volna.Solver(64) as sv:
        sv.set_params(h_threshold=1e-6)
        sv.upload_mesh(m)
        sv.set_open_boundary(ends)
        with pytest.raises(volna.VolnaError) as e:
            sv.set_open_boundary([[0, 1 + m.nv // 2]])
        assert e.value.code == volna.VG_EINVAL
        sv.set_open_boundary([])               # every boundary face a wall again
        sv.set_state(*s, 0.0)
        sv.step(50)
        H, Hu, Hv, _ = sv.get_state()
    for a, f in zip((H, Hu, Hv), FIELDS):
        np.testing.assert_array_equal(a, walls[f])
