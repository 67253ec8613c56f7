"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 within 1e-10 relative L2 per field, FP32 within 1e-4 relative
L2 of the FP64 oracle per field (both after 100 steps on the Thacker basin).
FP64 runs the literal build by default (fp64_literal = 1: no multiply-add
contraction, every formula in the oracle's order), whose result equals the
oracle's bit for bit (tested); the contracted build (fp64_literal = 0) differs
by rounding only and is held to the 1e-10 tolerance.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna
from gpu_helpers import FIELDS, VertexAdjacency, gpu_run, oracle_run, patch_mesh, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def thacker():
    m = I.thacker_mesh(n=100)                  # 20,000 triangles, dx = 0.04 (Sec. 3 basin)
    return m, I.thacker_initial_state(m)


@pytest.fixture(scope="module")
def thacker_ref(thacker):
    m, s = thacker
    return oracle_run(m, s, 100, gauges=I.THACKER_GAUGES, h_threshold=1e-5, cfl=0.9)


@pytest.mark.parametrize("renumber", ["none", "morton", "rcm", "hilbert"])
def test_fp64_parity_thacker_100_steps(thacker, thacker_ref, renumber):
    m, s = thacker
    g = gpu_run(m, s, 100, precision=64, renumber=renumber, gauges=I.THACKER_GAUGES,
                h_threshold=1e-5, cfl=0.9)
    for f in FIELDS:
        err = rel_l2(g[f], thacker_ref[f])
        assert err <= TOL64, (f, err, np.abs(g[f] - thacker_ref[f]).max())
    assert g["t"] == pytest.approx(thacker_ref["t"], rel=1e-14)
    assert g["diag"]["neg_count"] == thacker_ref["neg_count"] == 0
    # gauges: record at t0 plus one per step, eta of the containing cell
    assert g["gauge_eta"].shape == (101, 3)
    np.testing.assert_allclose(g["gauge_eta"][1:], thacker_ref["gauges"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.diff(g["gauge_t"]), thacker_ref["dts"], rtol=1e-13)


@pytest.mark.parametrize("renumber", ["none", "morton", "hilbert"])
def test_fp64_equals_oracle_bit_for_bit(thacker, thacker_ref, renumber):
    """The literal FP64 build (fp64_literal = 1) evaluates every formula in the
    oracle's order without contraction, so 100 CFL steps of the Thacker basin
    (dry land: blocks that skip their zero fluxes) equal the oracle's result
    exactly, time steps included."""
    m, s = thacker
    g = gpu_run(m, s, 100, precision=64, renumber=renumber, gauges=I.THACKER_GAUGES,
                h_threshold=1e-5, cfl=0.9, fp64_literal=1)
    for f in FIELDS:
        np.testing.assert_array_equal(g[f], thacker_ref[f], err_msg=f)
    t, ts = 0.0, []
    for dt in thacker_ref["dts"]:          # t accumulated as both sides do: t = t + dt
        t = t + float(dt)
        ts.append(t)
    np.testing.assert_array_equal(g["gauge_t"][1:], np.array(ts))
    np.testing.assert_array_equal(g["gauge_eta"][1:], thacker_ref["gauges"])


def test_fp64_contracted_build_100_steps(thacker, thacker_ref):
    """The contracted FP64 build (fp64_literal = 0: fused multiply-adds, fewer
    divisions) within the FP64 tolerance of the oracle after 100 steps, gauges and
    time steps within round-off."""
    m, s = thacker
    g = gpu_run(m, s, 100, precision=64, renumber="hilbert", gauges=I.THACKER_GAUGES,
                h_threshold=1e-5, cfl=0.9, fp64_literal=0)
    errs = {f: rel_l2(g[f], thacker_ref[f]) for f in FIELDS}
    print("contracted FP64 relative L2 after 100 steps:", errs)
    for f in FIELDS:
        assert errs[f] <= TOL64, (f, errs[f])
    np.testing.assert_allclose(g["gauge_eta"][1:], thacker_ref["gauges"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.diff(g["gauge_t"]), thacker_ref["dts"], rtol=1e-12)


@pytest.mark.parametrize("renumber", ["morton", "hilbert"])
def test_fp32_parity_thacker_100_steps(thacker, thacker_ref, renumber):
    m, s = thacker
    g = gpu_run(m, s, 100, precision=32, renumber=renumber, h_threshold=1e-5, cfl=0.9)
    errs = {f: rel_l2(g[f], thacker_ref[f]) for f in FIELDS}
    print("FP32 relative L2 after 100 steps:", errs)
    for f in FIELDS:
        assert errs[f] <= TOL32, (f, errs[f])
    assert g["t"] == pytest.approx(thacker_ref["t"], rel=1e-4)


@pytest.mark.parametrize("n,block", [(7, 32), (23, 64), (37, 128), (50, 256), (61, 96), (70, 512)])
def test_ragged_tiles_fp64(n, block):
    """Meshes spanning several blocks with a ragged last block, several block sizes."""
    m = I.thacker_mesh(n=n, shuffle_cells=True)
    s = I.thacker_initial_state(m)
    assert m.nc % block != 0
    g = gpu_run(m, s, 20, precision=64, renumber="morton", h_threshold=1e-5, block_cells=block)
    r = oracle_run(m, s, 20, h_threshold=1e-5)
    for f in FIELDS:
        assert rel_l2(g[f], r[f]) <= TOL64, f


@pytest.mark.parametrize("precision", [32, 64])
def test_contexts_with_different_blocks_coexist(thacker, precision):
    """Two contexts in one process, the second configured with a smaller block
    (less shared memory per CTA): the first still steps, with the same result
    as a context on its own."""
    m, s = thacker
    big = volna.Solver(precision)
    big.set_params(h_threshold=1e-5, block_cells=256)
    big.upload_mesh(m)
    small = volna.Solver(precision)
    small.set_params(h_threshold=1e-5, block_cells=32)
    small.upload_mesh(m)
    for sv in (big, small):
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(3)
    a, b = big.get_state(), small.get_state()
    big.close()
    small.close()
    for i in range(3):
        np.testing.assert_allclose(a[i], b[i], rtol=0, atol=1e-5 if precision == 32 else 1e-13)


def test_coast_basin_fp64_fp32():
    """Synthetic ocean-to-coast basin (N-wave uplift, inundation, H_threshold 1e-3 m)."""
    m = I.coast_mesh(n_theta=40, n_xi=120)
    s = I.coast_initial_state(m)
    gauges = I.coast_gauges()
    r = oracle_run(m, s, 60, gauges=gauges, h_threshold=1e-3, cfl=0.9)
    g64 = gpu_run(m, s, 60, precision=64, gauges=gauges, h_threshold=1e-3, cfl=0.9)
    g32 = gpu_run(m, s, 60, precision=32, gauges=gauges, h_threshold=1e-3, cfl=0.9)
    for f in FIELDS:
        assert rel_l2(g64[f], r[f]) <= TOL64, f
        assert rel_l2(g32[f], r[f]) <= TOL32, (f, rel_l2(g32[f], r[f]))
    np.testing.assert_allclose(g64["gauge_eta"][1:], r["gauges"], atol=1e-9)


@pytest.mark.parametrize("order", [1, 2])
def test_fixed_dt_t_end_and_order(thacker, order):
    m, s = thacker
    kw = dict(h_threshold=1e-5, dt_fixed=0.45 * 0.04 * 0.1, t_end=0.05, order=order)
    g = gpu_run(m, s, 40, precision=64, **kw)
    r = oracle_run(m, s, 40, **kw)
    for f in FIELDS:
        assert rel_l2(g[f], r[f]) <= TOL64, f
    assert g["t"] == pytest.approx(0.05, abs=1e-15) and r["t"] == pytest.approx(0.05, abs=1e-15)
    assert g["diag"]["steps"] < 40          # steps after t_end do not move


def test_lake_at_rest_gpu():
    """Still water over emerging dry land stays still on the GPU (FP64 and FP32)."""
    m = I.thacker_mesh(n=60)
    s = I.lake_at_rest_state(m, 0.0)
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        g = gpu_run(m, s, 300, precision=prec, h_threshold=1e-5, dt_max=0.01)
        assert np.abs(g["Hu"]).max() <= tol and np.abs(g["Hv"]).max() <= tol
        wet = s.H > 0
        z = -m.vertex_mean(m.depth)
        assert np.abs((g["H"] + z)[wet] - (s.H + z)[wet]).max() <= tol * 10


def test_mass_conserved_gpu(thacker):
    m, s = thacker
    area = O.OracleMesh.from_mesh(m).get("area")
    M0 = float(np.sum(area * s.H))
    g = gpu_run(m, s, 500, precision=64, h_threshold=1e-5)
    assert abs(float(np.sum(area * g["H"])) - M0) / M0 < 1e-13
    assert g["diag"]["mass"] == pytest.approx(M0, rel=1e-13)
    assert g["diag"]["neg_count"] == 0


def test_single_and_two_triangles():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    for tri in (np.array([[0, 1, 2]]), np.array([[0, 1, 3], [0, 3, 2]])):
        m = I.Mesh(xy, tri.astype(np.int32), np.array([1.0, 1.2, 0.8, 1.1]))
        st = I.State(np.full(len(tri), 1.0) + 0.1 * np.arange(len(tri)), np.full(len(tri), 0.3),
                     np.full(len(tri), -0.2))
        g = gpu_run(m, st, 10, precision=64, h_threshold=1e-5)
        r = oracle_run(m, st, 10, h_threshold=1e-5)
        for f in FIELDS:
            assert rel_l2(g[f], r[f]) <= TOL64, f


def test_all_dry_does_not_move():
    m = I.thacker_mesh(n=10)
    z = np.zeros(m.nc)
    st = I.State(z.copy(), z.copy(), z.copy())
    g = gpu_run(m, st, 5, precision=64)
    assert g["t"] == 0.0 and g["diag"]["steps"] == 0
    assert np.all(g["H"] == 0.0)
    g = gpu_run(m, st, 5, precision=64, dt_max=0.01)
    assert g["t"] == pytest.approx(0.05) and g["diag"]["steps"] == 5


def test_invalid_inputs_rejected():
    m = I.thacker_mesh(n=8)
    s = I.thacker_initial_state(m)
    with volna.Solver(64) as sv:
        with pytest.raises(volna.VolnaError) as e:
            sv.step(1)
        assert e.value.code == volna.VG_ESTATE
        bad = m.tri.copy()
        bad[3, 1] = bad[3, 0]
        with pytest.raises(volna.VolnaError) as e:
            volna.vg_mesh_upload(sv.ctx, m.xy, bad, m.depth)
        assert e.value.code == volna.VG_EINVAL
        with pytest.raises(volna.VolnaError):
            volna.vg_mesh_upload(sv.ctx, m.xy, np.zeros((0, 3), np.int32), m.depth)
        sv.upload_mesh(m)
        H = s.H.copy()
        H[5] = -1.0
        with pytest.raises(volna.VolnaError) as e:
            sv.set_state(H, s.Hu, s.Hv)
        assert e.value.code == volna.VG_EINVAL
        H[5] = np.nan
        with pytest.raises(volna.VolnaError):
            sv.set_state(H, s.Hu, s.Hv)
        with pytest.raises(volna.VolnaError) as e:
            sv.set_gauges([[10.0, 10.0]])
        assert e.value.code == volna.VG_EINVAL
        with pytest.raises(volna.VolnaError):
            sv.set_params(order=3)
        with pytest.raises(volna.VolnaError):
            sv.set_params(block_cells=100)
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(2)


def test_device_state_roundtrip_torch():
    torch = pytest.importorskip("torch")
    m = I.thacker_mesh(n=30)
    s = I.thacker_initial_state(m)
    stream = torch.cuda.Stream()
    with volna.Solver(64, stream=stream) as sv:
        sv.upload_mesh(m)
        Hd = torch.tensor(s.H, device="cuda")
        sv.set_state(Hd, torch.tensor(s.Hu, device="cuda"), torch.tensor(s.Hv, device="cuda"))
        sv.step(3)
        out = sv.get_state_dev()
        H, Hu, Hv, _ = sv.get_state()
    np.testing.assert_array_equal(out[0].cpu().numpy(), H)
    np.testing.assert_array_equal(out[1].cpu().numpy(), Hu)
    r = oracle_run(m, s, 3, h_threshold=1e-5)
    assert rel_l2(H, r["H"]) <= TOL64


def test_advance_to_and_graph_replay_consistency(thacker):
    """Graph-replayed steps equal kernel-by-kernel (profiling) steps bit for bit."""
    m, s = thacker
    with volna.Solver(64) as a, volna.Solver(64) as b:
        for sv in (a, b):
            sv.upload_mesh(m)
            sv.set_state(s.H, s.Hu, s.Hv)
        b.profile(True)
        a.step(33)
        b.step(33)
        for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
            np.testing.assert_array_equal(x, y)
        prof = b.get_profile()
        assert prof["stage1"][0] == 33 and prof["stage2"][0] == 33
        a.advance_to(0.2)
        assert a.diagnostics()["t"] == pytest.approx(0.2, abs=1e-15)


@pytest.fixture(scope="module")
def big40m():
    """The 40M-triangle Thacker workload of the benchmark, its initial state, 48
    sampled cells (32 wet, 16 in the shoreline band) and the vertex adjacency."""
    m = I.thacker_large_mesh()
    s = I.thacker_initial_state(m)
    rng = np.random.default_rng(11)
    p = m.cell_points()
    r2 = (p[:, 0] ** 2 + p[:, 1] ** 2) / m.meta["alpha"] ** 2
    wet_pool = np.nonzero(s.H > 0)[0]
    shore_pool = np.nonzero((r2 > 0.75) & (r2 < 0.85))[0]
    samples = np.concatenate([rng.choice(wet_pool, 32, replace=False),
                              rng.choice(shore_pool, 16, replace=False)])
    return m, s, samples, VertexAdjacency(m.tri, m.nv)


@pytest.mark.slow
@pytest.mark.parametrize("precision", [32, 64])
def test_full_size_40m_sampled_10_steps(big40m, precision):
    """The 40M-triangle workload in the benchmark's launch configuration (Hilbert
    renumbering, 256-cell blocks, persistent CTAs walking many blocks) for 10
    steps of a fixed time step (0.8 of the initial CFL step, so that both sides
    take the same steps): each sampled cell against the oracle run on the cells
    within 40 vertex rings of it, which hold everything 10 steps can reach (a
    step reaches 4 face rings: two stages of a two-ring stencil)."""
    m, s, samples, adj = big40m
    n_steps = 10
    with volna.Solver(precision) as sv:
        sv.upload_mesh(m, renumber="hilbert")
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(1)
        dt = 0.8 * sv.diagnostics()["last_dt"]
        sv.set_params(h_threshold=1e-5, cfl=0.9, dt_fixed=dt)
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(n_steps)
        d = sv.diagnostics()
        H, Hu, Hv, t = sv.get_state()
    assert t == pytest.approx(n_steps * dt, rel=1e-12) and d["neg_count"] == 0
    tol = 1e-12 if precision == 64 else 1e-4
    worst = 0.0
    for k in samples:
        cells = adj.rings([k], 4 * n_steps)
        centre = int(np.searchsorted(cells, k))
        om = O.OracleMesh.from_mesh(patch_mesh(m, cells))
        r = om.run(O.params(h_threshold=1e-5, dt_fixed=dt), (s.H[cells], s.Hu[cells], s.Hv[cells], 0.0), n_steps)
        scale = max(float(np.abs(s.H[cells]).max()), 1e-3)
        for f, gv in (("H", H), ("Hu", Hu), ("Hv", Hv)):
            err = abs(gv[k] - r[f][centre]) / scale
            worst = max(worst, err)
            assert err <= tol, (k, f, gv[k], r[f][centre])
    print(f"40M, {n_steps} fixed steps, FP{precision}: largest sampled error / local depth scale {worst:.3e}")


@pytest.mark.slow
@pytest.mark.parametrize("precision", [32, 64])
def test_full_size_coast_5m_sampled_10_steps(precision):
    """The 5M-triangle ocean-to-coast basin of the benchmark (graded 20:1, dry land,
    N-wave uplift, H_threshold 1e-3 m) in its launch configuration for 10 fixed steps:
    sampled cells in the uplift, on the shoreline, in the open ocean and on dry
    land against the oracle on their 40-ring patches.  Errors are taken per field
    against that field's largest magnitude over the whole basin (the scale of the
    relative L2 tolerance; near the shore the momentum is round-off noise)."""
    m = I.coast_mesh()
    s = I.coast_initial_state(m)
    h = m.vertex_mean(m.depth)
    xi = np.abs(s.H - np.where(h > 0, h, 0.0))
    rng = np.random.default_rng(5)
    pools = [np.nonzero(xi > 0.5)[0],                            # in the uplift
             np.nonzero((s.H > 0) & (s.H < 5.0))[0],             # shoreline water
             np.nonzero(s.H > 1000.0)[0],                        # open ocean
             np.nonzero((s.H == 0) & (h > -5.0))[0]]             # dry land by the shore
    samples = np.concatenate([rng.choice(pl, 8, replace=False) for pl in pools])
    n_steps = 10
    with volna.Solver(precision) as sv:
        sv.upload_mesh(m, renumber="hilbert")
        sv.set_params(h_threshold=1e-3, cfl=0.9)
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(1)
        dt = 0.8 * sv.diagnostics()["last_dt"]
        sv.set_params(h_threshold=1e-3, cfl=0.9, dt_fixed=dt)
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(n_steps)
        H, Hu, Hv, t = sv.get_state()
    tol = 1e-12 if precision == 64 else 1e-4
    scales = {f: float(np.abs(v).max()) for f, v in (("H", H), ("Hu", Hu), ("Hv", Hv))}
    adj = VertexAdjacency(m.tri, m.nv)
    worst = 0.0
    for k in samples:
        cells = adj.rings([k], 4 * n_steps)
        centre = int(np.searchsorted(cells, k))
        om = O.OracleMesh.from_mesh(patch_mesh(m, cells))
        r = om.run(O.params(h_threshold=1e-3, dt_fixed=dt), (s.H[cells], s.Hu[cells], s.Hv[cells], 0.0), n_steps)
        for f, gv in (("H", H), ("Hu", Hu), ("Hv", Hv)):
            scale = scales[f]
            err = abs(gv[k] - r[f][centre]) / scale
            worst = max(worst, err)
            assert err <= tol, (k, f, gv[k], r[f][centre], scale)
    print(f"coast 5M, {n_steps} fixed steps, FP{precision}: largest sampled error / field scale {worst:.3e}")


@pytest.mark.slow
@pytest.mark.parametrize("precision", [32, 64])
def test_full_size_40m_sampled(big40m, precision):
    """The 40M-triangle workload in the benchmark's launch configuration (Hilbert
    renumbering, 256-cell blocks): one step on the GPU; 48 sampled cells checked
    against the oracle run on their 4-ring patches with the GPU's time step, the
    time step checked against the sampled CFL bounds, and mass conservation."""
    m, s, samples, adj = big40m
    with volna.Solver(precision) as sv:
        sv.upload_mesh(m, renumber="hilbert")
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.set_state(s.H, s.Hu, s.Hv)
        d0 = sv.diagnostics()
        sv.step(1)
        d1 = sv.diagnostics()
        H, Hu, Hv, t = sv.get_state()
    dt = d1["last_dt"]
    assert dt > 0 and t == pytest.approx(dt)
    assert abs(d1["mass"] - d0["mass"]) / d0["mass"] < (1e-13 if precision == 64 else 1e-5)
    tol = 1e-12 if precision == 64 else 1e-4
    for k in samples:
        cells = adj.rings([k], 4)
        pm = patch_mesh(m, cells)
        centre = int(np.searchsorted(cells, k))
        om = O.OracleMesh.from_mesh(pm)
        st = (s.H[cells], s.Hu[cells], s.Hv[cells], 0.0)
        _, am = om.residual(O.params(h_threshold=1e-5), *st[:3])
        area = om.get("area")
        if am[centre] > 0:      # the GPU's dt is the global minimum of these bounds
            assert dt <= 0.9 * area[centre] / (3.0 * am[centre]) * (1 + (1e-12 if precision == 64 else 1e-5))
        r = om.run(O.params(h_threshold=1e-5, dt_fixed=dt), st, 1)
        scale = max(float(np.abs(s.H[cells]).max()), 1e-3)
        for f, gv in (("H", H), ("Hu", Hu), ("Hv", Hv)):
            assert abs(gv[k] - r[f][centre]) <= tol * scale, (k, f, gv[k], r[f][centre])


@pytest.mark.parametrize("precision", [32, 64])
def test_pinned_host_buffers_are_used_in_place(thacker, precision):
    """vg_set_state / vg_get_state with pinned (page-locked, mapped) host buffers
    read and write them in place from the kernels (one thread per original
    cell); the result equals the staged copy of pageable buffers bit for bit."""
    torch = pytest.importorskip("torch")
    m, s = thacker
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()
    with volna.Solver(precision) as a, volna.Solver(precision) as b:
        for sv in (a, b):
            sv.set_params(h_threshold=1e-5)
            sv.upload_mesh(m)
        a.set_state(pin(s.H), pin(s.Hu), pin(s.Hv), 0.0)
        b.set_state(s.H, s.Hu, s.Hv, 0.0)
        a.step(7)
        b.step(7)
        outs = [torch.empty(m.nc, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
        _, _, _, ta = volna.vg_get_state(a.ctx, m.nc, out=tuple(outs))
        ref = b.get_state()
        for x, y in zip(outs, ref[:3]):
            np.testing.assert_array_equal(x, y)
        assert ta == ref[3]


@pytest.mark.parametrize("precision", [32, 64])
def test_fp32_host_interface(thacker, precision):
    """vg_set_state_f32 / vg_get_state_f32: FP32 host arrays (pinned: read and
    written in place; pageable: staged) store exactly the state that FP64 host
    arrays of the same values store, and the FP32 export is the FP32 rounding of
    the FP64 export, bit for bit."""
    torch = pytest.importorskip("torch")
    m, s = thacker
    f32 = [np.ascontiguousarray(x, dtype=np.float32) for x in (s.H, s.Hu, s.Hv)]
    pin = lambda a: torch.from_numpy(a.copy()).pin_memory().numpy()
    with volna.Solver(precision) as a, volna.Solver(precision) as b, volna.Solver(precision) as c:
        for sv in (a, b, c):
            sv.set_params(h_threshold=1e-5)
            sv.upload_mesh(m)
        volna.vg_set_state_f32(a.ctx, *[pin(x) for x in f32], 0.0)
        c.set_state(*f32, 0.0)                          # pageable FP32: staged
        b.set_state(*[x.astype(np.float64) for x in f32], 0.0)
        for sv in (a, b, c):
            sv.step(7)
        ref = b.get_state()
        outs = tuple(torch.empty(m.nc, dtype=torch.float32).pin_memory().numpy() for _ in range(3))
        got_pinned = volna.vg_get_state_f32(a.ctx, m.nc, out=outs)
        got_paged = c.get_state(np.float32)
        for got in (got_pinned, got_paged):
            for x, y in zip(got[:3], ref[:3]):
                assert x.dtype == np.float32
                np.testing.assert_array_equal(x, y.astype(np.float32))
            assert got[3] == ref[3]
        # pinned views off the 16-byte grid take the one-cell-per-thread path
        def pin_off(x):
            buf = torch.empty(x.size + 1, dtype=torch.from_numpy(x).dtype).pin_memory().numpy()
            buf[1:] = x
            return buf[1:]
        for dt in (np.float32, np.float64):
            src = [pin_off(x.astype(dt)) for x in f32]
            (volna.vg_set_state_f32 if dt == np.float32 else volna.vg_set_state)(a.ctx, *src, 0.0)
            a.step(7)
            out = tuple(pin_off(np.zeros(m.nc, dtype=dt)) for _ in range(3))
            got = (volna.vg_get_state_f32 if dt == np.float32 else volna.vg_get_state)(a.ctx, m.nc, out=out)
            for x, y in zip(got[:3], ref[:3]):
                np.testing.assert_array_equal(x, y.astype(dt))
        bad = f32[0].copy()
        bad[3] = -1.0
        with pytest.raises(volna.VolnaError):
            volna.vg_set_state_f32(a.ctx, bad, f32[1], f32[2], 0.0)
        with pytest.raises(ValueError):
            volna.vg_get_state_f32(a.ctx, m.nc, out=tuple(np.empty(m.nc) for _ in range(3)))


def test_fp32_host_interface_ragged_tail():
    """A cell count that is not a multiple of 4 (5202 triangles): the last cells
    after the 16-byte groups of the in-place import / export are still moved."""
    torch = pytest.importorskip("torch")
    m = I.thacker_mesh(n=51)
    s = I.thacker_initial_state(m)
    assert m.nc % 4 == 2
    f32 = [np.ascontiguousarray(x, dtype=np.float32) for x in (s.H, s.Hu, s.Hv)]
    pin = lambda a: torch.from_numpy(a.copy()).pin_memory().numpy()
    with volna.Solver(32) as a, volna.Solver(32) as b:
        for sv in (a, b):
            sv.set_params(h_threshold=1e-5)
            sv.upload_mesh(m)
        volna.vg_set_state_f32(a.ctx, *[pin(x) for x in f32], 0.0)
        b.set_state(*[x.astype(np.float64) for x in f32], 0.0)
        a.step(3)
        b.step(3)
        ref = b.get_state()
        out = tuple(torch.empty(m.nc, dtype=torch.float32).pin_memory().numpy() for _ in range(3))
        got = volna.vg_get_state_f32(a.ctx, m.nc, out=out)
        for x, y in zip(got[:3], ref[:3]):
            np.testing.assert_array_equal(x, y.astype(np.float32))
