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
    """A time step far above the CFL limit drains cells below zero; with
    strict_positivity the step fails with VG_ENEGDEPTH (otherwise it is counted)."""
    m = I.thacker_mesh(n=20)
    s = I.thacker_initial_state(m)
    with volna.Solver(64) as sv:
        sv.upload_mesh(m)
        sv.set_params(dt_fixed=0.1, strict_positivity=1)
        sv.set_state(s.H, s.Hu, s.Hv)
        with pytest.raises(volna.VolnaError) as e:
            sv.step(5)
        assert e.value.code in (volna.VG_ENEGDEPTH, volna.VG_ENONFINITE)
    with volna.Solver(64) as sv:
        sv.upload_mesh(m)
        sv.set_params(dt_fixed=0.1)
        sv.set_state(s.H, s.Hu, s.Hv)
        try:
            sv.step(2)
        except volna.VolnaError as e:
            assert e.code == volna.VG_ENONFINITE
        assert sv.diagnostics()["neg_count"] > 0
