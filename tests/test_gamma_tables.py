"""The package's Dirac matrices (used to build Gamma for the CUDA path) equal the
oracle's independently written table."""

import numpy as np

from oracle import dirac
from paper_2212_04430_gb300 import gamma as pg


def test_gamma_tables_agree():
    for mu in range(4):
        assert np.array_equal(pg.gamma_mu(mu + 1), dirac.GAMMA[mu])
    assert np.array_equal(pg.gamma5(), dirac.GAMMA5)
    assert np.allclose(pg.gamma_matrix("g5g3"), dirac.gamma_product(["g5", "g3"]))
    assert np.allclose(pg.gamma_matrix("1"), np.eye(4))
