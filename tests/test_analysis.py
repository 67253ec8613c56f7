"""Sec. 4 error decomposition: the product's closed forms against the 3 x 3 system
they solve (CPU), and a small GPU run of Thacker's basin on three grids."""
import numpy as np
import pytest

from paper_2002_04889_gb300 import analysis


def test_decompose_solves_the_printed_system():
    rng = np.random.default_rng(11)
    for h in (0.024, 0.1):
        E = rng.normal(size=(3, 7)) * 1e-3
        C = analysis.decompose(E[0], E[1], E[2], h)
        for k in range(3):
            hk = h / 2 ** k
            np.testing.assert_allclose(C[0] * hk ** 2 + C[1] * hk ** 3 + C[2] * hk ** 4, E[k], rtol=1e-9,
                                       atol=1e-15)


@pytest.mark.gpu
def test_thacker_decomposition_small():
    r = analysis.thacker_decomposition(n_coarse=40, t_fin=1.0)
    assert r["E"].shape[0] == 3 and r["E"].shape[1] > 10
    h = r["h"]
    recon = r["C1"] * h ** 2 + r["C2"] * h ** 3 + r["C3"] * h ** 4
    np.testing.assert_allclose(recon, r["E"][0], rtol=1e-8, atol=1e-14)
    # the error shrinks under refinement (time-averaged, Sec. 3)
    m = r["E"].mean(axis=1)
    assert m[0] > m[1] > m[2]
