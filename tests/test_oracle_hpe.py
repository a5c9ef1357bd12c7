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


# ---- the generalised expansion (the Wilson-clover operator) ----------------------------------
from oracle import clover as oclover  # noqa: E402


def _cterm(u, dims, c_sw):
    return oclover.clover_term(u.reshape((4,) + odirac.lattice_shape(dims) + (3, 3)), c_sw)


def test_generalised_truncation_identity_per_sample():
    """With the clover term, z^dag G Om (D_sw+s)^-1 z = sum_{k<K} z^dag G Om K^k A^-1 z + remainder
    for every z, K = A(x)^-1 H / 2 and A(x) = 4 + m + s + C(x): the remainder from the solver, the
    low orders by direct site solves (a factor of A(x) on the wrong side, or the scalar A, fails)."""
    dims = (2, 2, 4, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=191)
    m, s = 0.1, 0.3
    ct = _cterm(u, dims, 1.2)
    blocks = ohpe.site_factor(ct, 4.0 + m + s, v)
    solver = oest.make_dense_solver(u, m, dims, -1, ct)
    for K in (1, 2, 4):
        for p in (0, 1):
            z = philox.z4_noise(v, 6, 0, 0, K + 3 * p)
            full = oest.contract(u, z, solver(z, s), G3, p, dims)
            y = np.linalg.solve(blocks, z.reshape(v, 12, 1))[..., 0].reshape(z.shape)
            low = 0j
            for _ in range(K):
                low += oest.contract(u, z, y, G3, p, dims)
                hy = ohpe.apply_H(u, y, dims) / 2
                y = np.linalg.solve(blocks, hy.reshape(v, 12, 1))[..., 0].reshape(z.shape)
            rem = ohpe.stochastic_part(u, solver, z, m, s, G3, p, K, dims, cterm=ct)
            assert low + rem == pytest.approx(full, rel=1e-11, abs=1e-11), (K, p)


def test_generalised_exact_part_plus_remainder_and_probing():
    """T_exact + Tr(remainder) = Tr(G Om (D_sw+s)^-1), and displacement-p distance-(K-1) probing gives
    T_exact exactly (A(x)^-1 is local to a site)."""
    dims = (2, 2, 6, 2)
    u = inputs.gauge_field(dims, "smooth", seed=192, eps=0.6)
    m, s = 0.05, 0.4
    ct = _cterm(u, dims, 1.0)
    g = odirac.gamma_product(["g5", "g3"])
    for (p, K) in ((0, 4), (1, 3), (2, 4)):
        t = ohpe.exact_part_dense(u, m, s, g, p, K, dims, cterm=ct)
        rem = np.trace(ohpe.remainder_matrix(u, m, s, g, p, K, dims, cterm=ct))
        full = np.trace(osolve.dense_GammaOmega(u, g, p, dims) @ osolve.dense_inverse(u, m, s, dims, -1, ct))
        assert t + rem == pytest.approx(full, rel=1e-11), (p, K)
        col, nc = opr.greedy_coloring(dims, K - 1, p)
        assert ohpe.exact_part_probed(u, m, s, g, p, K, dims, col, nc, cterm=ct) == pytest.approx(
            t, rel=1e-11, abs=1e-11), (p, K)


def test_generalised_order_zero_on_a_constant_abelian_field():
    """On a constant abelian field C(x) = c X (x) 1, X = i gamma_mu gamma_nu (X^2 = 1, tr X = 0),
    c = (c_sw / 2) sin B, so A^-1 = (a - c X) / (a^2 - c^2) at every site and the order-0 term is
    Tr(A^-1) = 12 V a / (a^2 - c^2) for Gamma = 1, p = 0."""
    dims = (4, 4, 2, 2)
    v = int(np.prod(dims))
    u, b = inputs.abelian_field(dims, n=1, mu=0, nu=1)
    c_sw, m, s = 1.5, 0.2, 0.3
    a = 4.0 + m + s
    c = 0.5 * c_sw * np.sin(b)
    col, nc = opr.greedy_coloring(dims, 0, 0)
    t = ohpe.exact_part_probed(u, m, s, odirac.IDENT4, 0, 1, dims, col, nc, cterm=_cterm(u, dims, c_sw))
    assert t == pytest.approx(12 * v * a / (a * a - c * c), rel=1e-12)
    assert abs(12 * v * a / (a * a - c * c) - 12 * v / a) > 1e-3  # the clover term matters here


def test_generalised_expansion_without_clover_is_the_classical_one():
    dims = (2, 2, 4, 2)
    u = inputs.gauge_field(dims, "smooth", seed=193, eps=0.5)
    m, s = 0.0, 0.5
    zero = _cterm(u, dims, 0.0)
    for (p, K) in ((0, 4), (1, 2)):
        assert ohpe.exact_part_dense(u, m, s, G3, p, K, dims, cterm=zero) == pytest.approx(
            ohpe.exact_part_dense(u, m, s, G3, p, K, dims), rel=1e-12, abs=1e-12)


def test_generalised_expansion_reduces_the_variance():
    dims = (2, 2, 4, 2)
    u = inputs.gauge_field(dims, "smooth", seed=194, eps=0.4)
    m, s = -0.2, 0.6
    ct = _cterm(u, dims, 1.0)
    plain = osolve.dense_GammaOmega(u, G3, 1, dims) @ osolve.dense_inverse(u, m, s, dims, -1, ct)
    rem = ohpe.remainder_matrix(u, m, s, G3, 1, 4, dims, cterm=ct)
    assert oest.exact_z4_variance(rem) < 0.2 * oest.exact_z4_variance(plain)
