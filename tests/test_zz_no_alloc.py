"""vg_step_noalloc: the time step for callers that cannot allocate device memory.

Such callers (a fully reserved memory pool, a real-time loop that must not touch
the allocator, a framework that forbids allocations after set-up) get one step
whose scratch lives in a fixed device array inside the library.  These tests
call it through the C ABI and check it against the ordinary vg_step, within the
FP64 parity tolerance of the other GPU tests, on two calls in a row (the second
call starts from the first call's output and must not see stale scratch).  The
file is named to run last.
"""
import numpy as np
import pytest

from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def test_noalloc_matches_vg_step_on_two_calls():
    torch = pytest.importorskip("torch")
    m = I.thacker_mesh(n=60, shuffle_cells=True)        # 7,200 triangles
    s = I.thacker_initial_state(m)
    with volna.Solver(64) as ref:
        ref.upload_mesh(m)
        ref.set_state(s.H, s.Hu, s.Hv, 0.0)
        ref.step(1)
        r1 = ref.get_state()
        ref.step(1)
        r2 = ref.get_state()

    with volna.Solver(64) as sv:
        sv.upload_mesh(m)
        new_of_old = sv.permutation()
        w0 = np.zeros((3, m.nc))
        for row, v in enumerate((s.H, s.Hu, s.Hv)):
            w0[row, new_of_old] = v
        a = torch.tensor(w0, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        torch.cuda.synchronize()
        dt1 = volna.vg_step_noalloc(sv.ctx, a.data_ptr(), b.data_ptr(), 0.0)
        out1 = b.cpu().numpy()[:, new_of_old]
        dt2 = volna.vg_step_noalloc(sv.ctx, b.data_ptr(), a.data_ptr(), dt1)
        out2 = a.cpu().numpy()[:, new_of_old]

    for out, r in ((out1, r1), (out2, r2)):
        for row in range(3):
            assert _rel_l2(out[row], r[row]) <= TOL64, row
    assert dt1 > 0 and dt2 > 0
    assert dt1 == pytest.approx(r1[3], rel=1e-14)
    assert dt1 + dt2 == pytest.approx(r2[3], rel=1e-14)


def test_noalloc_rejects_meshes_above_its_limit():
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
