"""Batched ensembles (vg_batch_*) against one context per scenario and the oracle.

The batch runs the same per-block arithmetic as a single context, so each
scenario's result must equal its own single-context run bit for bit (same
precision, same block size); FP64 scenarios also match the oracle within the
FP64 parity tolerance.
"""
import numpy as np
import pytest

from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna
from gpu_helpers import FIELDS, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _meshes():
    # three coast basins of uneven size (about 2.9k, 6.5k and 12k triangles)
    return [I.coast_mesh_with_cells(n, seed=k) for k, n in enumerate((3000, 6500, 12000))]


def _scenarios(mesh, k, n):
    out = []
    for amp, ang in I.ensemble_sources(k, n):
        s = I.coast_initial_state(mesh, amplitude=amp, angle_deg=ang)
        out.append(s)
    return out


def _single(mesh, s, precision, n_steps=None, t_end=None, **params):
    with volna.Solver(precision) as sv:
        sv.set_params(h_threshold=1e-3, cfl=0.9, **params)
        sv.upload_mesh(mesh)
        sv.set_state(s.H, s.Hu, s.Hv, 0.0)
        if t_end is not None:
            sv.advance_to(t_end)
        else:
            sv.step(n_steps)
        return sv.get_state()


@pytest.mark.parametrize("precision,literal", [(32, 1), (64, 1), (64, 0)])
def test_batch_equals_single_contexts(precision, literal):
    """Both FP64 builds (literal and contracted): a batch runs the build a single
    context of the same parameters runs."""
    meshes = _meshes()
    nscen = 3
    scen = [_scenarios(m, k, nscen) for k, m in enumerate(meshes)]
    with volna.Batch(precision) as b:
        b.set_params(h_threshold=1e-3, cfl=0.9, fp64_literal=literal)
        ids = [b.add_mesh(m, nscen) for m in meshes]
        for mid, ss in zip(ids, scen):
            for j, s in enumerate(ss):
                b.set_state(mid, j, s.H, s.Hu, s.Hv, 0.0)
        info = b.info()
        assert info["scenarios"] == 9 and info["cells"] == nscen * sum(m.nc for m in meshes)
        b.step(25)
        for mid, m, ss in zip(ids, meshes, scen):
            for j, s in enumerate(ss):
                H, Hu, Hv, t, steps = b.get_state(mid, j)
                ref = _single(m, s, precision, n_steps=25, fp64_literal=literal)
                assert steps == 25
                assert t == ref[3]
                for a, r in zip((H, Hu, Hv), ref[:3]):
                    np.testing.assert_array_equal(a, r)
    if precision == 64:
        m, s = meshes[0], scen[0][1]
        r = oracle_run(m, s, 25, h_threshold=1e-3, cfl=0.9)
        ref = _single(m, s, 64, n_steps=25, fp64_literal=literal)
        for f, g in zip(FIELDS, ref[:3]):
            assert rel_l2(g, r[f]) <= 1e-10


@pytest.mark.parametrize("precision", [32, 64])
def test_batch_run_to_common_end_time(precision):
    """Each scenario keeps its own dt and stops exactly at t_end; the batched
    kernels skip a scenario that reached t_end (its state carries over), and
    every scenario equals its single-context run to t_end bit for bit."""
    meshes = _meshes()[:2]
    scen = [_scenarios(m, k, 2) for k, m in enumerate(meshes)]
    t_end = 30.0
    with volna.Batch(precision) as b:
        b.set_params(h_threshold=1e-3, cfl=0.9)
        ids = [b.add_mesh(m, 2) for m in meshes]
        for mid, ss in zip(ids, scen):
            for j, s in enumerate(ss):
                b.set_state(mid, j, s.H, s.Hu, s.Hv, 0.0)
        taken = b.run(t_end, max_steps=100000)
        assert taken > 0
        steps = []
        for mid, m, ss in zip(ids, meshes, scen):
            for j, s in enumerate(ss):
                H, Hu, Hv, t, n = b.get_state(mid, j)
                assert t == pytest.approx(t_end, abs=1e-12)
                steps.append(n)
                ref = _single(m, s, precision, t_end=t_end)
                assert t == ref[3]
                for a, r in zip((H, Hu, Hv), ref[:3]):
                    np.testing.assert_array_equal(a, r)
        assert len(set(steps)) > 1          # uneven meshes take different numbers of steps


def test_batch_autotune_keeps_results():
    meshes = _meshes()[:2]
    scen = [_scenarios(m, k, 2) for k, m in enumerate(meshes)]
    with volna.Batch(32) as b:
        b.set_params(h_threshold=1e-3, cfl=0.9)
        ids = [b.add_mesh(m, 2) for m in meshes]
        for mid, ss in zip(ids, scen):
            for j, s in enumerate(ss):
                b.set_state(mid, j, s.H, s.Hu, s.Hv, 0.0)
        before = [b.get_state(mid, j) for mid in ids for j in range(2)]
        block, ms, ctas = b.autotune(3)
        assert block in (64, 128, 256) and ms > 0 and ctas >= 0
        after = [b.get_state(mid, j) for mid in ids for j in range(2)]
        for x, y in zip(before, after):               # the tuner restores the state
            for a, c in zip(x[:3], y[:3]):
                np.testing.assert_array_equal(a, c)
            assert x[3] == y[3] == 0.0
        b.step(10)
        for mid, m, ss in zip(ids, meshes, scen):
            for j, s in enumerate(ss):
                H, Hu, Hv, t, _ = b.get_state(mid, j)
                ref = _single(m, s, 32, n_steps=10)
                for a, r in zip((H, Hu, Hv), ref[:3]):
                    assert rel_l2(a, r) <= 1e-5


@pytest.mark.parametrize("precision,every", [(32, 1), (64, 3)])
def test_batch_gauges_equal_single_contexts(precision, every):
    """Gauge records of every scenario (t and eta, at set_state and after every
    `every` steps, 150 steps: more records than one device ring holds) equal
    those of a context of its own, bit for bit; a scenario that reached t_end
    records nothing more."""
    meshes = _meshes()[:2]
    scen = [_scenarios(m, k, 2) for k, m in enumerate(meshes)]
    pts = [I.coast_gauges(5) for _ in meshes]
    with volna.Batch(precision) as b:
        b.set_params(h_threshold=1e-3, cfl=0.9, gauge_every=every)
        ids = [b.add_mesh(m, 2) for m in meshes]
        b.set_gauges(ids[0], pts[0])
        for mid, ss in zip(ids, scen):
            for j, s in enumerate(ss):
                b.set_state(mid, j, s.H, s.Hu, s.Hv, 0.0)
        b.set_gauges(ids[1], pts[1])            # after the state: records from now on
        b.step(150)
        for mid, m, ss, p in zip(ids, meshes, scen, pts):
            for j, s in enumerate(ss):
                t, eta = b.gauges(mid, j)
                with volna.Solver(precision) as sv:
                    sv.set_params(h_threshold=1e-3, cfl=0.9, gauge_every=every)
                    sv.upload_mesh(m)
                    sv.set_gauges(p)
                    sv.set_state(s.H, s.Hu, s.Hv, 0.0)
                    sv.step(150)
                    t_ref, eta_ref = sv.gauges()
                assert len(t) == 1 + 150 // every
                np.testing.assert_array_equal(t, t_ref)
                np.testing.assert_array_equal(eta, eta_ref)
        # with t_end set, a scenario that reached it takes no step and records nothing
        t_now = b.get_state(ids[0], 0)[3]
        b.set_params(h_threshold=1e-3, cfl=0.9, gauge_every=every, t_end=t_now + 2.0)
        b.step(300)
        t, _ = b.gauges(ids[0], 0)
        assert t[-1] <= t_now + 2.0 + 1e-9
        assert np.all(np.diff(t) > 0)
