"""Moving bed (vg_set_bed_motion, the time-dependent depth of Sec. 2.1) on the
GPU against the oracle's moving bed (vo_bed_at, itself pinned in
test_oracle_moving_bed.py), through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna
from gpu_helpers import FIELDS, rel_l2

pytestmark = pytest.mark.gpu

GAUGES = np.array([[0.1, -0.05], [0.4, 0.2], [-0.3, 0.1]])


def _gpu(mesh, s, n, precision, motion, gauges=None, **prm):
    with volna.Solver(precision) as sv:
        sv.set_params(**prm)
        sv.upload_mesh(mesh)
        if motion is not None:
            sv.set_bed_motion(*motion)
        if gauges is not None:
            sv.set_gauges(gauges)
        sv.set_state(s.H, s.Hu, s.Hv, s.t)
        d0 = sv.diagnostics()
        sv.step(n)
        H, Hu, Hv, t = sv.get_state()
        out = dict(H=H, Hu=Hu, Hv=Hv, t=t, d0=d0, d1=sv.diagnostics())
        if gauges is not None:
            out["gt"], out["geta"] = sv.gauges()
        return out


def _oracle(mesh, s, n, motion, gauges=None, **prm):
    om = O.OracleMesh.from_mesh(mesh)
    cells = om.locate(gauges) if gauges is not None else None
    up, on, rise = motion
    return om.run(O.params(**prm), (s.H, s.Hu, s.Hv, s.t), n, gauge_cells=cells,
                  bed_motion=(mesh.depth, up, on, rise))


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 1e-4)])
def test_radial_rupture_matches_oracle(precision, tol):
    """Thacker basin (3,200 triangles) under a Gaussian uplift whose onset spreads
    from (0.1, -0.05) at 2 m/s with a 0.1 s rise; 60 adaptive steps."""
    m = I.thacker_mesh(n=40)
    s = I.thacker_initial_state(m)
    up, on = I.radial_rupture(m.xy, 0.02, 0.1, -0.05, 0.4, 2.0, 0.0)
    prm = dict(h_threshold=1e-5, cfl=0.9)
    g = _gpu(m, s, 60, precision, (up, on, 0.1), GAUGES, **prm)
    r = _oracle(m, s, 60, (up, on, 0.1), GAUGES, **prm)
    for f in FIELDS:
        assert rel_l2(g[f], r[f]) <= tol, f
    assert g["t"] == pytest.approx(r["t"], rel=1e-12 if precision == 64 else 1e-5)
    atol = 1e-12 if precision == 64 else 2e-5
    np.testing.assert_allclose(g["geta"][1:], r["gauges"], rtol=0, atol=atol)
    # the bed moved: the free surface differs from the static run at the gauges
    st = _gpu(m, s, 60, precision, None, GAUGES, **prm)
    assert np.max(np.abs(st["geta"] - g["geta"])) > 1e-3


def test_coast_rupture_matches_oracle_fp64():
    """Coast basin (6,500 triangles), N-wave source released along its axis."""
    m = I.coast_mesh_with_cells(6500, seed=1)
    s = I.coast_initial_state(m, amplitude=0.0)
    up, on = I.coast_rupture(m, v_rupture=2_000.0)
    prm = dict(h_threshold=1e-3, cfl=0.9)
    g = _gpu(m, s, 40, 64, (up, on, 20.0), **prm)
    r = _oracle(m, s, 40, (up, on, 20.0), **prm)
    for f in FIELDS:
        assert rel_l2(g[f], r[f]) <= 1e-10, f


@pytest.mark.parametrize("precision", [32, 64])
def test_instantaneous_uplift_equals_static_bed(precision):
    m = I.thacker_mesh(n=30)
    s = I.thacker_initial_state(m)
    up, _ = I.radial_rupture(m.xy, 0.02, 0.1, -0.05, 0.4, 2.0, 0.0)
    prm = dict(h_threshold=1e-5, cfl=0.9)
    a = _gpu(m, s, 25, precision, (up, np.zeros(m.nv), 0.0), **prm)
    mu = I.Mesh(m.xy, m.tri, m.depth - up, name="uplifted", meta=m.meta)
    b = _gpu(mu, s, 25, precision, None, **prm)
    for f in FIELDS:
        np.testing.assert_array_equal(a[f], b[f])


def test_mass_conserved_and_future_onset_is_inert():
    m = I.thacker_mesh(n=32)
    s = I.thacker_initial_state(m)
    up, on = I.radial_rupture(m.xy, 0.03, 0.1, -0.05, 0.4, 2.0, 0.0)
    prm = dict(h_threshold=1e-5, cfl=0.9)
    g = _gpu(m, s, 200, 64, (up, on, 0.1), **prm)
    assert g["d1"]["neg_count"] == 0
    assert abs(g["d1"]["mass"] - g["d0"]["mass"]) <= 1e-13 * g["d0"]["mass"]
    late = _gpu(m, s, 30, 64, (up, on + 1e6, 0.1), **prm)
    static = _gpu(m, s, 30, 64, None, **prm)
    for f in FIELDS:
        np.testing.assert_array_equal(late[f], static[f])


def test_remove_motion_and_guards():
    m = I.thacker_mesh(n=20)
    s = I.thacker_initial_state(m)
    up, on = I.radial_rupture(m.xy, 0.02, 0.1, -0.05, 0.4, 2.0, 0.0)
    with volna.Solver(64) as sv:
        sv.set_params(h_threshold=1e-5)
        sv.upload_mesh(m)
        sv.set_gauges(GAUGES)
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.set_bed_motion(up, on, 0.0)
        with pytest.raises(volna.VolnaError) as e:
            sv.set_depth(m.depth)
        assert e.value.code == volna.VG_ESTATE
        with pytest.raises(volna.VolnaError) as e:
            sv.set_bed_motion(up, on, -1.0)
        assert e.value.code == volna.VG_EINVAL
        M0 = sv.diagnostics()["mass"]
        sv.step(10)
        sv.set_bed_motion(None)               # static bed again, H kept
        assert abs(sv.diagnostics()["mass"] - M0) <= 1e-13 * M0
        sv.set_depth(m.depth)
        sv.step(5)
        assert np.isfinite(sv.get_state()[0]).all()


def test_pinned_state_io_follows_the_moving_bed():
    """FP32 with a moving bed: the in-place export of pinned host buffers (FP32 and
    FP64) forms H from the moved bed, as the staged export does, bit for bit; a
    state set from pinned buffers after the bed moved stores the same eta."""
    torch = pytest.importorskip("torch")
    m = I.thacker_mesh(n=40)
    s = I.thacker_initial_state(m)
    up, on = I.radial_rupture(m.xy, 0.02, 0.1, -0.05, 0.4, 2.0, 0.0)
    with volna.Solver(32) as sv:
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.upload_mesh(m)
        sv.set_bed_motion(up, on, 0.1)
        sv.set_state(s.H, s.Hu, s.Hv, s.t)
        sv.step(40)
        ref = sv.get_state()                                # staged (pageable) export
        for dt in (np.float32, np.float64):
            tdt = torch.float32 if dt == np.float32 else torch.float64
            out = tuple(torch.empty(m.nc, dtype=tdt).pin_memory().numpy() for _ in range(3))
            got = (volna.vg_get_state_f32 if dt == np.float32 else volna.vg_get_state)(sv.ctx, m.nc, out=out)
            for x, y in zip(got[:3], ref[:3]):
                np.testing.assert_array_equal(x, y.astype(dt))
        pin = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy() for x in ref[:3]]
        sv.set_state(*pin, ref[3])                           # in-place import over the moved bed
        again = sv.get_state()
        for x, y in zip(again[:3], ref[:3]):
            np.testing.assert_array_equal(x, y)
