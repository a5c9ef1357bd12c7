"""Pins of the oracle's hopping parameter expansion (paper Sec. 3.1, the remark after
Eq. (sampled_single)): the truncation identity, closed forms of the exact low orders, the exact
low orders from displacement-p distance-(K-1) probing, and the variance reduction."""

import numpy as np
import pytest

from oracle import dirac as odirac
from oracle import estimators as oest
from oracle import hpe as ohpe
from oracle import philox
from oracle import probing as opr
from oracle import solve as osolve

import inputs

G3 = odirac.gamma_product(["g3"])


def test_truncation_identity_per_sample():
    """z^dag G Om (D+s)^-1 z = sum_{k<K} z^dag G Om (kappa H)^k z / A + remainder, for every z:
    the remainder of the expansion taken from the solver (a wrong kappa, order or A fails)."""
    dims = (2, 2, 4, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=91)
    m, s = 0.1, 0.3
    A = 4.0 + m + s
    solver = oest.make_dense_solver(u, m, dims)
    for K in (1, 2, 4):
        for p in (0, 1):
            z = philox.z4_noise(v, 5, 0, 0, K + 3 * p)
            full = oest.contract(u, z, solver(z, s), G3, p, dims)
            y = z / A
            low = 0j
            for _ in range(K):
                low += oest.contract(u, z, y, G3, p, dims)
                y = ohpe.apply_H(u, y, dims) / (2 * A)
            rem = ohpe.stochastic_part(u, solver, z, m, s, G3, p, K, dims)
            assert low + rem == pytest.approx(full, rel=1e-11, abs=1e-11), (K, p)


def test_exact_part_plus_remainder_is_the_trace():
    dims = (2, 2, 4, 2)
    u = inputs.gauge_field(dims, "smooth", seed=92, eps=0.5)
    m, s = 0.05, 0.4
    g = odirac.gamma_product(["g5", "g3"])
    for (p, K) in ((0, 4), (1, 4), (2, 3)):
        t = ohpe.exact_part_dense(u, m, s, g, p, K, dims)
        rem = np.trace(ohpe.remainder_matrix(u, m, s, g, p, K, dims))
        full = np.trace(osolve.dense_GammaOmega(u, g, p, dims) @ osolve.dense_inverse(u, m, s, dims))
        assert t + rem == pytest.approx(full, rel=1e-11), (p, K)


def test_closed_forms_of_the_low_orders():
    """Any gauge field: p = 1, K = 2 gives kappa 3V tr(G (1 + g_z)) / A (the one backward z hop);
    p = 2, K = 3 (Lz = 6) gives kappa^2 6V tr(G (1 + g_z)) / A ((1 + g_z)^2 = 2 (1 + g_z));
    p = 0, K = 4 (every extent >= 3) gives 3V tr(G) / A (no odd closed paths, and a
    back-tracking pair (1 - g)(1 + g) vanishes)."""
    dims = (2, 2, 6, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=93)
    m, s = 0.0, 0.5
    A = 4.0 + m + s
    kappa = 1.0 / (2 * A)
    for g in (G3, odirac.gamma_product(["g5", "g3"]), odirac.IDENT4):
        tr1 = np.trace(g @ (odirac.IDENT4 + odirac.GAMMA[2]))
        assert ohpe.exact_part_dense(u, m, s, g, 1, 2, dims) == pytest.approx(kappa * 3 * v * tr1 / A, abs=1e-10)
        assert ohpe.exact_part_dense(u, m, s, g, 2, 3, dims) == pytest.approx(kappa ** 2 * 6 * v * tr1 / A,
                                                                               abs=1e-10)
    dims4 = (4, 4, 4, 4)
    u4 = inputs.gauge_field(dims4, "haar", seed=94)
    col, nc = opr.greedy_coloring(dims4, 3, 0)
    for g in (odirac.IDENT4, G3):
        t = ohpe.exact_part_probed(u4, m, s, g, 0, 4, dims4, col, nc)
        assert t == pytest.approx(3 * 256 * np.trace(g) / A, abs=1e-9)


@pytest.mark.parametrize("p,K", [(0, 2), (0, 4), (1, 3), (1, 4), (2, 4)])
def test_probing_gives_the_exact_low_orders(p, K):
    """Displacement-p distance-(K-1) colours make the probed sum exact (Sec. 3.1); one distance
    less is not enough where the order K - 1 term links distinct sites."""
    dims = (2, 2, 6, 2)
    u = inputs.gauge_field(dims, "smooth", seed=95, eps=0.6)
    m, s = 0.1, 0.2
    g = odirac.gamma_product(["g5", "g3"])
    ref = ohpe.exact_part_dense(u, m, s, g, p, K, dims)
    col, nc = opr.greedy_coloring(dims, K - 1, p)
    assert ohpe.exact_part_probed(u, m, s, g, p, K, dims, col, nc) == pytest.approx(ref, rel=1e-11, abs=1e-11)
    if (p, K) == (0, 4):
        # Gamma = I: the spin traces of the third-order paths between distinct sites survive
        ref1 = ohpe.exact_part_dense(u, m, s, odirac.IDENT4, p, K, dims)
        col2, nc2 = opr.greedy_coloring(dims, K - 2, p)
        assert abs(ohpe.exact_part_probed(u, m, s, odirac.IDENT4, p, K, dims, col2, nc2) - ref1) > 1e-6


def test_expansion_reduces_the_variance():
    """For m + s > 0 the remainder's exact Z4 variance is far below that of the plain estimator."""
    dims = (2, 2, 4, 2)
    u = inputs.gauge_field(dims, "smooth", seed=96, eps=0.4)
    m, s = -0.2, 0.6
    plain = osolve.dense_GammaOmega(u, G3, 1, dims) @ osolve.dense_inverse(u, m, s, dims)
    rem = ohpe.remainder_matrix(u, m, s, G3, 1, 4, dims)
    assert oest.exact_z4_variance(rem) < 0.2 * oest.exact_z4_variance(plain)
