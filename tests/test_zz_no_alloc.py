"""vg_step_noalloc: the time step for callers that cannot allocate device memory.

Such callers (a fully reserved memory pool, a real-time loop that must not touch
the allocator, a framework that forbids allocations after set-up) get one step
whose scratch lives in a fixed device array inside the library.  These tests
call it through the C ABI and check it against the ordinary vg_step, within the
parity tolerances of the other GPU tests (FP64 1e-10, FP32 1e-4 relative L2),
on two calls in a row (the second call starts from the first call's output and
must not see stale scratch), and check that neither call takes device memory.
The file is named to run last.
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna

pytestmark = pytest.mark.gpu

TOL = {64: 1e-10, 32: 1e-4}


def _rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_matches_vg_step_on_two_calls(precision):
    torch = pytest.importorskip("torch")
    m = I.thacker_mesh(n=60, shuffle_cells=True)        # 7,200 triangles
    s = I.thacker_initial_state(m)
    with volna.Solver(precision) as ref:
        ref.upload_mesh(m)
        ref.set_state(s.H, s.Hu, s.Hv, 0.0)
        ref.step(1)
        r1 = ref.get_state()
        ref.step(1)
        r2 = ref.get_state()

    # the stored state form: (H, Hu, Hv) in FP64; (eta, Hu, Hv) in FP32 with eta =
    # H + z formed in FP64 and rounded once, z the cell bed (the oracle's vertex
    # mean in the same local vertex order, bit for bit the library's FP64 bed)
    z = O.OracleMesh.from_mesh(m).get("z")
    dtype = torch.float64 if precision == 64 else torch.float32
    with volna.Solver(precision) as sv:
        sv.upload_mesh(m)
        new_of_old = sv.permutation()
        w0 = np.zeros((3, m.nc))
        first = s.H if precision == 64 else s.H + z
        for row, v in enumerate((first, s.Hu, s.Hv)):
            w0[row, new_of_old] = v
        a = torch.tensor(w0, dtype=dtype, device="cuda")
        b = torch.empty_like(a)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dt1 = volna.vg_step_noalloc(sv.ctx, a.data_ptr(), b.data_ptr(), 0.0)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        dt2 = volna.vg_step_noalloc(sv.ctx, b.data_ptr(), a.data_ptr(), dt1)
        torch.cuda.synchronize()
        free2 = torch.cuda.mem_get_info()[0]
        out1 = b.double().cpu().numpy()[:, new_of_old]
        out2 = a.double().cpu().numpy()[:, new_of_old]
    # no device memory was taken by either call (the scratch was committed at set-up)
    assert free1 >= free0 and free2 >= free1, (free0, free1, free2)

    if precision == 32:
        # stored eta -> depth, as the state export forms it: dry where eta does not
        # exceed the FP32 bed, else eta - z in FP64
        z32 = z.astype(np.float32).astype(np.float64)
        for out in (out1, out2):
            out[0] = np.where(out[0] - z32 <= 0.0, 0.0, np.maximum(0.0, out[0] - z))
    for out, r in ((out1, r1), (out2, r2)):
        for row in range(3):
            assert _rel_l2(out[row], r[row]) <= TOL[precision], (precision, row)
    assert dt1 > 0 and dt2 > 0
    assert dt1 == pytest.approx(r1[3], rel=1e-14 if precision == 64 else 1e-6)
    assert dt1 + dt2 == pytest.approx(r2[3], rel=1e-14 if precision == 64 else 1e-6)


def test_noalloc_rejects_meshes_above_its_limit_and_moving_beds():
    torch = pytest.importorskip("torch")
    n = 363                                               # 2 * 363^2 = 263,538 > 262,144
    m = I.thacker_mesh(n=n)
    assert m.nc > volna.VG_NOALLOC_MAX_CELLS
    with volna.Solver(64) as sv:
        sv.upload_mesh(m)
        a = torch.zeros((3, m.nc), dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        with pytest.raises(volna.VolnaError) as e:
            volna.vg_step_noalloc(sv.ctx, a.data_ptr(), b.data_ptr(), 0.0)
        assert e.value.code == volna.VG_EINVAL
        assert "at most" in str(e.value)
    small = I.thacker_mesh(n=20)
    s = I.thacker_initial_state(small)
    with volna.Solver(64) as sv:
        sv.upload_mesh(small)
        sv.set_state(s.H, s.Hu, s.Hv, 0.0)
        sv.set_bed_motion(np.full(small.nv, 0.01), np.zeros(small.nv), 0.5)
        a = torch.zeros((3, small.nc), dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        with pytest.raises(volna.VolnaError) as e:
            volna.vg_step_noalloc(sv.ctx, a.data_ptr(), b.data_ptr(), 0.0)
        assert e.value.code == volna.VG_ESTATE
        sv.set_bed_motion(None)
        volna.vg_step_noalloc(sv.ctx, a.data_ptr(), b.data_ptr(), 0.0)
