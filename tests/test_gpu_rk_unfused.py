"""The unfused SSP-RK(2,2) stages (vg_params.rk_unfused = 1: update 1, the
residual of w1 and update 2 as kernels of their own, w1 and R(w1) through
device memory) against the fused stage-2 kernel: the same arithmetic cell by
cell (Sec. 2.3), so FP64 results are equal bit for bit, to each other and to
the oracle, and FP32 results agree to rounding."""
import numpy as np
import pytest

from paper_2002_04889_gb300 import inputs as I
from gpu_helpers import FIELDS, gpu_run, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def thacker():
    m = I.thacker_mesh(n=100)
    return m, I.thacker_initial_state(m)


def test_fp64_unfused_equals_fused_and_oracle(thacker):
    m, s = thacker
    kw = dict(precision=64, renumber="hilbert", gauges=I.THACKER_GAUGES, h_threshold=1e-5, cfl=0.9)
    fused = gpu_run(m, s, 100, **kw)
    unfused = gpu_run(m, s, 100, rk_unfused=1, **kw)
    ref = oracle_run(m, s, 100, gauges=I.THACKER_GAUGES, h_threshold=1e-5, cfl=0.9)
    for f in FIELDS:
        assert np.array_equal(unfused[f], fused[f]), f
        assert np.array_equal(unfused[f], ref[f]), f
    assert unfused["t"] == fused["t"]
    np.testing.assert_array_equal(unfused["gauge_eta"], fused["gauge_eta"])
    # two more launches per step: update 1, residual of w1, update 2 replace stage 2
    assert unfused["diag"]["launches"] - fused["diag"]["launches"] == 2 * 100


def test_fp32_unfused_matches_fused(thacker):
    m, s = thacker
    kw = dict(precision=32, renumber="hilbert", h_threshold=1e-5, cfl=0.9)
    fused = gpu_run(m, s, 100, **kw)
    unfused = gpu_run(m, s, 100, rk_unfused=1, **kw)
    errs = {f: rel_l2(unfused[f], fused[f]) for f in FIELDS}
    same = all(np.array_equal(unfused[f], fused[f]) for f in FIELDS)
    print("FP32 unfused vs fused, 100 steps, relative L2:", errs, "bitwise:", same)
    for f in FIELDS:
        assert errs[f] <= 1e-6, (f, errs[f])
    assert unfused["t"] == pytest.approx(fused["t"], rel=1e-6)


@pytest.mark.parametrize("precision", [64, 32])
def test_unfused_dry_fix_counts_and_t_end(precision):
    """Coast basin (inundation, dry fix of both updates): the negative-depth count
    and the state at t_end, where the finished steps copy the state unchanged."""
    m = I.coast_mesh(n_theta=40, n_xi=120)
    s = I.coast_initial_state(m)
    kw = dict(precision=precision, h_threshold=1e-3, cfl=0.9)
    fused = gpu_run(m, s, 60, **kw)
    t_end = 0.5 * fused["t"]
    fused_end = gpu_run(m, s, 60, t_end=t_end, **kw)
    unfused_end = gpu_run(m, s, 60, t_end=t_end, rk_unfused=1, **kw)
    assert unfused_end["t"] == fused_end["t"] == pytest.approx(t_end, rel=1e-12)
    assert unfused_end["diag"]["neg_count"] == fused_end["diag"]["neg_count"]
    for f in FIELDS:
        if precision == 64:
            assert np.array_equal(unfused_end[f], fused_end[f]), f
        else:
            assert rel_l2(unfused_end[f], fused_end[f]) <= 1e-6, f
