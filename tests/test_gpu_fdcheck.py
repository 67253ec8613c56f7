"""The adjoint configuration's gradient check at reduced size: the hand-written
adjoint's directional derivatives of a 16-gauge misfit against central finite
differences of the FP64 forward run, 8 seeded directions (initial depth and
vertex depths), each with a sweep of steps: the misfit is piecewise smooth with
dense kinks (the min / max of Zhou's wave speeds tie wherever the flow is
smooth), so the difference quotient approaches the adjoint's derivative as the
step shrinks, until round-off.  The full-size check
(1M triangles, 2000 steps, 32 directions) is `python -m
paper_2002_04889_gb300.fdcheck`."""
import numpy as np
import pytest

from paper_2002_04889_gb300 import fdcheck

pytestmark = pytest.mark.gpu


def test_adjoint_gradient_against_finite_differences_reduced():
    r = fdcheck.fd_check(n=100, n_steps=200, n_dirs=8, eps=1e-8, eps_sweep=(1e-6, 1e-7, 1e-8, 1e-9),
                         sweep_dirs=8)
    for d in r["directions"]:
        print(d["kind"], d["adjoint"], d["best_eps"], d["best_rel_err"])
    assert all(abs(d["adjoint"]) > 0 for d in r["directions"])
    best = sorted(d["best_rel_err"] for d in r["directions"])
    # every direction agrees at the plateau of its steps
    assert best[-1] <= 2e-3, r
    assert best[len(best) // 2] <= 5e-4, r
