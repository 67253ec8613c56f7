"""The hand-written CUDA adjoint (vg_adj_forward / vg_adj_backward) against
(1) the oracle's discrete adjoint -- tape AD of the oracle's own arithmetic, an
independent program -- and (2) central finite differences of the GPU forward
run, all in FP64 with a fixed time step.

Time step (reading of the adjoint set-up): the CFL step of the initial state
(CFL 0.9) times a 0.8 safety factor, shared by the target run, the finite
differences and the adjoint so that gauge times coincide.
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna

pytestmark = pytest.mark.gpu

LATTICE = np.array([[x, y] for x in np.linspace(-0.6, 0.6, 4) for y in np.linspace(-0.6, 0.6, 4)])


def _case(n, half_width=1.0):
    m = I.thacker_mesh(n=n, half_width=half_width)
    s = I.thacker_initial_state(m)
    p = m.cell_points()
    deep = s.H > 2e-2
    Hu = s.Hu + 1e-3 * np.sin(3 * p[:, 0]) * deep
    Hv = s.Hv + 1e-3 * np.cos(2 * p[:, 1]) * deep
    om = O.OracleMesh.from_mesh(m)
    _, am = om.residual(O.params(), s.H, Hu, Hv)
    dt = 0.8 * om.time_step(O.params(cfl=0.9), am, 0.0)
    return m, (s.H, Hu, Hv), dt, om.locate(LATTICE)


def _gpu_adjoint(m, st, dt, n_steps, W, every=0):
    with volna.Solver(64) as sv:
        sv.set_params(h_threshold=1e-5)
        sv.upload_mesh(m)
        sv.set_gauges(LATTICE)
        sv.set_state(*st, 0.0)
        _, eta = sv.adj_forward(n_steps, dt, every)
        g = sv.adj_backward(W, m.nv)
    return eta, g


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_adjoint_matches_oracle_tape_adjoint():
    """2,048-triangle basin, 20 steps, random weights on 16 gauges."""
    m, st, dt, cells = _case(32)
    n_steps = 20
    W = np.random.default_rng(3).normal(size=(n_steps + 1, len(cells)))
    eta, g = _gpu_adjoint(m, st, dt, n_steps, W)
    ad = O.ad_gauge_gradient(m, st, dt, n_steps, cells, W, h_threshold=1e-5)
    np.testing.assert_allclose(eta, ad["eta"], rtol=0, atol=1e-13)
    for k_gpu, k_or in (("H0", "dH0"), ("Hu0", "dHu0"), ("Hv0", "dHv0"), ("depth", "ddepth")):
        err = _rel(g[k_gpu], ad[k_or])
        assert err <= 1e-10, (k_gpu, err)


@pytest.mark.parametrize("every", [1, 3])
def test_checkpoint_interval_does_not_change_the_gradient(every):
    m, st, dt, cells = _case(24)
    n_steps = 11
    W = np.random.default_rng(4).normal(size=(n_steps + 1, len(cells)))
    _, g0 = _gpu_adjoint(m, st, dt, n_steps, W, every=0)
    _, g1 = _gpu_adjoint(m, st, dt, n_steps, W, every=every)
    for k in ("H0", "Hu0", "Hv0", "depth"):
        np.testing.assert_array_equal(g0[k], g1[k])


def _fd_agrees(f, x0_shift, gd, eps_list=(1e-6, 1e-7, 1e-8, 1e-9), rel=2e-4):
    """Central differences at several steps (the plateau): True if one of them
    matches the adjoint's directional derivative gd within rel.  The wave-speed
    min/max of Sec. 2.2 tie exactly for equal neighbour states, so near-ties are
    everywhere in smooth flow and a step can straddle some; the sweep looks for
    the plateau between that and round-off."""
    errs = []
    for eps in eps_list:
        fd = (f(eps) - f(-eps)) / (2 * eps)
        errs.append(abs(gd - fd) / max(abs(fd), 1e-14))
    return min(errs) <= rel, errs


def test_adjoint_vs_central_differences():
    """Misfit J = 1/2 sum (eta - eta_target)^2 over 16 gauges and 40 steps on a
    3,200-triangle basin; the target run has a seeded 0.01 m Gaussian uplift and
    a seeded +-1 % bathymetry perturbation.  8 seeded directions in the initial
    depth (wet cells) and in the vertex depths."""
    m, st, dt, cells = _case(40)
    n_steps = 40
    rng = np.random.default_rng(12)
    p = m.cell_points()
    bump = 0.01 * np.exp(-((p[:, 0] - 0.2) ** 2 + (p[:, 1] + 0.1) ** 2) / 0.05)
    wet = st[0] > 2e-2
    depth_t = m.depth * (1.0 + 0.01 * (2 * rng.random(m.nv) - 1))

    def run(H0, depth):
        sv = volna.Solver(64)
        sv.set_params(h_threshold=1e-5)
        sv.upload_mesh(m)
        sv.set_depth(depth)
        sv.set_gauges(LATTICE)
        sv.set_state(H0, st[1], st[2], 0.0)
        _, eta = sv.adj_forward(n_steps, dt)
        return sv, eta

    sv_t, eta_t = run(st[0] + bump * wet, depth_t)
    sv_t.close()

    def J(H0, depth):
        sv, eta = run(H0, depth)
        sv.close()
        return 0.5 * float(np.sum((eta - eta_t) ** 2))

    sv, eta = run(st[0], m.depth)
    g = sv.adj_backward(eta - eta_t, m.nv)
    sv.close()
    n_ok = 0
    for k in range(8):
        if k % 2 == 0:
            d = rng.normal(size=m.nc) * wet
            gd = float(np.dot(g["H0"], d))
            ok, errs = _fd_agrees(lambda e: J(st[0] + e * d, m.depth), None, gd)
        else:
            d = rng.normal(size=m.nv) * m.depth * 1e-2
            gd = float(np.dot(g["depth"], d))
            ok, errs = _fd_agrees(lambda e: J(st[0], m.depth + e * d), None, gd)
        n_ok += ok
    assert n_ok >= 7, n_ok


def test_autograd_uplift_and_bathymetry():
    """torch.autograd: in the wet cells H0 = eta_base + uplift - z(depth), elsewhere
    the base depth (a dry cell sits exactly on the kink of max(0, .), where no
    derivative exists); gradients of a gauge misfit with respect to the uplift
    field and the vertex depths agree with central differences of the whole
    pipeline."""
    torch = pytest.importorskip("torch")
    from paper_2002_04889_gb300.adjoint import cell_bed, gauge_records
    m, st, dt, cells = _case(24)
    n_steps = 20
    tri = torch.tensor(m.tri.astype(np.int64))
    z0 = -m.vertex_mean(m.depth)
    eta_base = torch.tensor(st[0] + z0)          # free surface of the base state
    wet = torch.tensor((st[0] > 2e-2).astype(np.float64))
    rng = np.random.default_rng(21)
    target = torch.tensor(rng.normal(size=(n_steps + 1, len(cells))) * 1e-3)
    sv = volna.Solver(64)
    sv.set_params(h_threshold=1e-5)
    sv.upload_mesh(m)
    sv.set_gauges(LATTICE)

    H_base = torch.tensor(st[0])

    def loss_of(uplift, depth):
        H0 = wet * (eta_base + uplift - cell_bed(tri, depth)) + (1.0 - wet) * H_base
        eta = gauge_records(sv, H0, torch.tensor(st[1]), torch.tensor(st[2]), depth, n_steps, dt)
        return 0.5 * torch.sum((eta - target) ** 2)

    up = torch.zeros(m.nc, dtype=torch.float64, requires_grad=True)
    dep = torch.tensor(m.depth, requires_grad=True)
    L = loss_of(up, dep)
    L.backward()
    for grad, which in ((up.grad, 0), (dep.grad, 1)):
        d = torch.tensor(rng.normal(size=grad.numel())) * (1.0 if which == 0 else 1e-2)
        gd = float(torch.dot(grad, d))
        with torch.no_grad():
            if which == 0:
                f = lambda e: float(loss_of(e * d, dep))
            else:
                f = lambda e: float(loss_of(up, dep + e * d))
            ok, errs = _fd_agrees(f, None, gd)
        assert ok, (which, gd, errs)
    sv.close()


def test_adjoint_through_cfl_time_steps_matches_oracle():
    """dt = 0: every step takes the CFL step of its state (Sec. 2.3 rule), and the
    adjoint differentiates through it.  Against the oracle's taped adjoint of the
    same adaptive run (2,048 triangles, 20 steps): the step sizes agree, the
    gradients to 1e-10; the gradient differs from the fixed-step one."""
    m, st, _, cells = _case(32)
    n_steps = 20
    W = np.random.default_rng(8).normal(size=(n_steps + 1, len(cells)))
    with volna.Solver(64) as sv:
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.upload_mesh(m)
        sv.set_gauges(LATTICE)
        sv.set_state(*st, 0.0)
        t, eta = sv.adj_forward(n_steps, 0.0)
        g = sv.adj_backward(W, m.nv)
    ad = O.ad_gauge_gradient(m, st, None, n_steps, cells, W, h_threshold=1e-5, cfl=0.9)
    np.testing.assert_allclose(np.diff(t), ad["dts"], rtol=1e-12, atol=0)
    assert np.ptp(ad["dts"]) > 0
    np.testing.assert_allclose(eta, ad["eta"], rtol=0, atol=1e-13)
    for k_gpu, k_or in (("H0", "dH0"), ("Hu0", "dHu0"), ("Hv0", "dHv0"), ("depth", "ddepth")):
        err = _rel(g[k_gpu], ad[k_or])
        assert err <= 1e-10, (k_gpu, err)
    fixed = O.ad_gauge_gradient(m, st, float(ad["dts"][0]), n_steps, cells, W, h_threshold=1e-5)
    assert _rel(fixed["dH0"], ad["dH0"]) > 1e-6


def test_adjoint_through_cfl_steps_vs_central_differences():
    """Misfit of 16 gauges over 30 adaptive steps on 3,200 triangles: the adjoint's
    directional derivatives agree with central differences of the GPU's own
    adaptive forward run (8 seeded directions, the plateau of steps)."""
    m, st, _, cells = _case(40)
    n_steps = 30
    rng = np.random.default_rng(19)
    wet = st[0] > 2e-2
    p = m.cell_points()
    bump = 0.01 * np.exp(-((p[:, 0] - 0.2) ** 2 + (p[:, 1] + 0.1) ** 2) / 0.05)

    def run(H0, depth):
        sv = volna.Solver(64)
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.upload_mesh(m)
        sv.set_depth(depth)
        sv.set_gauges(LATTICE)
        sv.set_state(H0, st[1], st[2], 0.0)
        _, eta = sv.adj_forward(n_steps, 0.0)
        return sv, eta

    sv_t, eta_t = run(st[0] + bump * wet, m.depth)
    sv_t.close()

    def J(H0, depth):
        sv, eta = run(H0, depth)
        sv.close()
        return 0.5 * float(np.sum((eta - eta_t) ** 2))

    sv, eta = run(st[0], m.depth)
    g = sv.adj_backward(eta - eta_t, m.nv)
    sv.close()
    n_ok = 0
    for k in range(8):
        if k % 2 == 0:
            d = rng.normal(size=m.nc) * wet
            gd = float(np.dot(g["H0"], d))
            ok, errs = _fd_agrees(lambda e: J(st[0] + e * d, m.depth), None, gd)
        else:
            d = rng.normal(size=m.nv) * m.depth * 1e-2
            gd = float(np.dot(g["depth"], d))
            ok, errs = _fd_agrees(lambda e: J(st[0], m.depth + e * d), None, gd)
        n_ok += ok
    assert n_ok >= 7, n_ok


@pytest.mark.parametrize("adaptive", [False, True])
def test_adjoint_with_moving_bed_matches_oracle(adaptive):
    """A Gaussian uplift spreading from (0.1, -0.05) at 2 m/s, rising over 0.05 s,
    under the basin (2,048 triangles, 20 steps, fixed or CFL steps): the GPU
    gradients with respect to the initial state, the depths, the uplift and the
    onset times equal the oracle's taped ones to 1e-10."""
    m, st, dt_fixed, cells = _case(32)
    n_steps = 20
    up, on = I.radial_rupture(m.xy, 0.01, 0.1, -0.05, 0.4, 2.0, 0.0)
    W = np.random.default_rng(23).normal(size=(n_steps + 1, len(cells)))
    dt = 0.0 if adaptive else dt_fixed
    with volna.Solver(64) as sv:
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.upload_mesh(m)
        sv.set_gauges(LATTICE)
        sv.set_bed_motion(up, on, 0.05)
        sv.set_state(*st, 0.0)
        _, eta = sv.adj_forward(n_steps, dt)
        g = sv.adj_backward(W, m.nv)
        gu, go = sv.adj_bed_gradient(m.nv)
    ad = O.ad_gauge_gradient(m, st, dt or None, n_steps, cells, W, h_threshold=1e-5, cfl=0.9,
                             bed_motion=(up, on, 0.05))
    np.testing.assert_allclose(eta, ad["eta"], rtol=0, atol=1e-13)
    pairs = (("H0", g["H0"], "dH0"), ("Hu0", g["Hu0"], "dHu0"), ("Hv0", g["Hv0"], "dHv0"),
             ("depth", g["depth"], "ddepth"), ("uplift", gu, "duplift"), ("onset", go, "donset"))
    for name, gg, k_or in pairs:
        err = _rel(gg, ad[k_or])
        assert err <= 1e-10, (name, err)
    assert np.max(np.abs(go)) > 0 and np.max(np.abs(gu)) > 0


@pytest.mark.parametrize("absorbing", [False, True])
def test_adjoint_with_open_boundaries_matches_oracle(absorbing):
    """Two sides of a 0.1 m basin open, a hump drifting out through them, CFL steps
    (3,200 triangles, 25 steps): the GPU gradients equal the oracle's taped ones
    (same open edges) to 1e-10.  absorbing: the x side takes the characteristic
    ghost of a sea at rest (whose c_0 brings the bed into the ghost), the y side
    stays open."""
    m0 = I.flat_basin_mesh(40, 1.0, 0.1)
    # a gentle slope and curvature: on a perfectly flat bed every face is a tie of
    # max(z_L, z_R), where the depth derivative does not exist
    m = I.Mesh(m0.xy, m0.tri, 0.1 + 0.02 * m0.xy[:, 0] + 0.01 * m0.xy[:, 1] ** 2, name="sloped", meta=m0.meta)
    s = I.gaussian_hump_state(m, 0.0, 0.02, 0.5, -0.3, 0.4)
    p = m.cell_points()
    st = (s.H, 0.05 * s.H * (1.0 + 0.3 * np.sin(2 * p[:, 1])), -0.03 * s.H)
    cells = O.OracleMesh.from_mesh(m).locate(LATTICE)
    n_steps = 25
    edges = np.concatenate([I.boundary_edges(m, lambda mid: mid[:, 0] > 0.999),
                            I.boundary_edges(m, lambda mid: mid[:, 1] < -0.999)])
    assert len(edges) > 10
    n_x = len(I.boundary_edges(m, lambda mid: mid[:, 0] > 0.999))
    kinds = np.array([3 if absorbing and e < n_x else 2 for e in range(len(edges))], dtype=np.int32)
    W = np.random.default_rng(29).normal(size=(n_steps + 1, len(cells)))
    with volna.Solver(64) as sv:
        sv.set_params(h_threshold=1e-5, cfl=0.9)
        sv.upload_mesh(m)
        sv.set_boundary(edges, kinds)
        sv.set_gauges(LATTICE)
        sv.set_state(*st, 0.0)
        _, eta = sv.adj_forward(n_steps, 0.0)
        g = sv.adj_backward(W, m.nv)
    ad = O.ad_gauge_gradient(m, st, None, n_steps, cells, W, h_threshold=1e-5, cfl=0.9, open_edges=edges,
                             boundary_kinds=kinds)
    np.testing.assert_allclose(eta, ad["eta"], rtol=0, atol=1e-13)
    for k_gpu, k_or in (("H0", "dH0"), ("Hu0", "dHu0"), ("Hv0", "dHv0"), ("depth", "ddepth")):
        err = _rel(g[k_gpu], ad[k_or])
        assert err <= 1e-10, (k_gpu, err)


@pytest.mark.parametrize("slots", [1, 2, 5])
@pytest.mark.parametrize("adaptive", [False, True])
def test_binomial_checkpointing_gives_the_same_gradient(slots, adaptive):
    """vg_adj_forward_binomial keeps only the first state and reverses 23 steps
    with a few state slots, recomputing along the binomial schedule: the gradient
    (with a moving bed, so the per-step times matter too) equals the sqrt(N)
    checkpointed one bit for bit."""
    m, st, dt_fixed, cells = _case(24)
    n_steps = 23
    up, on = I.radial_rupture(m.xy, 0.01, 0.1, -0.05, 0.4, 2.0, 0.0)
    W = np.random.default_rng(31).normal(size=(n_steps + 1, len(cells)))
    dt = 0.0 if adaptive else dt_fixed
    out = []
    for mode in ("sqrt", "binomial"):
        with volna.Solver(64) as sv:
            sv.set_params(h_threshold=1e-5, cfl=0.9)
            sv.upload_mesh(m)
            sv.set_gauges(LATTICE)
            sv.set_bed_motion(up, on, 0.05)
            sv.set_state(*st, 0.0)
            if mode == "sqrt":
                sv.adj_forward(n_steps, dt)
            else:
                sv.adj_forward_binomial(n_steps, dt, slots)
            g = sv.adj_backward(W, m.nv)
            g["uplift"], g["onset"] = sv.adj_bed_gradient(m.nv)
            out.append(g)
    for k in ("H0", "Hu0", "Hv0", "depth", "uplift", "onset"):
        np.testing.assert_array_equal(out[0][k], out[1][k])
