"""Failure detection without faulting the GPU: errors are provoked on the host
(bad inputs, absurd parameters) and come back as status codes."""
import numpy as np
import pytest

from paper_2002_04889_gb300 import inputs as I
from paper_2002_04889_gb300 import volna

pytestmark = pytest.mark.gpu


def test_non_finite_state_is_reported():
    """An absurd gravity overflows the fluxes; vg_step reports VG_ENONFINITE and
    the context stays usable."""
    m = I.thacker_mesh(n=12)
    s = I.thacker_initial_state(m)
    with volna.Solver(64) as sv:
        sv.upload_mesh(m)
        sv.set_params(g=1e300, dt_fixed=1.0)
        sv.set_state(s.H, s.Hu, s.Hv)
        with pytest.raises(volna.VolnaError) as e:
            sv.step(3)
        assert e.value.code == volna.VG_ENONFINITE
        sv.set_params(g=9.81)                    # recover: reset the state and go on
        sv.set_state(s.H, s.Hu, s.Hv)
        sv.step(3)
        assert np.isfinite(sv.get_state()[0]).all()


def test_strict_positivity_reports_negative_depth():
    """A dam break onto a dry bed, one step at ten times the CFL step: the cells
    behind the dam drain below zero.  By default they are counted (the same count
    as the oracle's) and emptied; with strict_positivity vg_step returns
    VG_ENEGDEPTH."""
    import oracle as O
    m = I.flat_basin_mesh(n=20, half_width=1.0, depth=0.0)
    s = I.dam_break_state(m, 0.5)
    om = O.OracleMesh.from_mesh(m)
    _, am = om.residual(O.params(), s.H, s.Hu, s.Hv)
    dt = 10.0 * om.time_step(O.params(), am, 0.0)
    ref = om.run(O.params(dt_fixed=dt), (s.H, s.Hu, s.Hv), 1)
    assert ref["neg_count"] > 0
    for strict in (0, 1):
        with volna.Solver(64) as sv:
            sv.upload_mesh(m)
            sv.set_params(dt_fixed=dt, strict_positivity=strict)
            sv.set_state(s.H, s.Hu, s.Hv)
            if strict:
                with pytest.raises(volna.VolnaError) as e:
                    sv.step(1)
                assert e.value.code == volna.VG_ENEGDEPTH
            else:
                sv.step(1)
                d = sv.diagnostics()
                assert d["neg_count"] == ref["neg_count"] and d["min_H"] >= 0.0
