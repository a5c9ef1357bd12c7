"""Pins of the oracle's probing colorings and probed / diluted noise (paper Sec. 2.1,
Eq. (probing_vectors), displacement-p probing, and Sec. 3.1 full spin-color dilution)."""

import itertools

import numpy as np
import pytest

from oracle import estimators as oest
from oracle import philox
from oracle import probing as opr
from oracle import solve as osolve

import inputs


def _torus_l1(dims, a, b):
    return sum(min((a[m] - b[m]) % dims[m], (b[m] - a[m]) % dims[m]) for m in range(4))


def _coords(dims, i):
    x0 = i % dims[0]
    i //= dims[0]
    x1 = i % dims[1]
    i //= dims[1]
    return (x0, x1, i % dims[2], i // dims[2])


@pytest.mark.parametrize("dims,k,p", [((4, 4, 4, 4), 1, 0), ((4, 4, 4, 4), 2, 0), ((4, 4, 6, 2), 1, 1),
                                      ((4, 2, 6, 4), 2, 2)])
def test_coloring_separates_every_conflicting_pair(dims, k, p):
    """Checked from coordinates, independently of the oracle's conflict sets: two sites whose
    hop distance is at most k (p = 0), or one of which lies within distance k of the other
    displaced by +-p along z, have different colors."""
    color, nc = opr.greedy_coloring(dims, k, p)
    v = int(np.prod(dims))
    assert color.min() == 0 and color.max() == nc - 1
    xs = [_coords(dims, i) for i in range(v)]
    for i in range(v):
        for j in range(i + 1, v):
            if p == 0:
                close = _torus_l1(dims, xs[i], xs[j]) <= k
            else:
                up = (xs[i][0], xs[i][1], (xs[i][2] + p) % dims[2], xs[i][3])
                dn = (xs[i][0], xs[i][1], (xs[i][2] - p) % dims[2], xs[i][3])
                close = _torus_l1(dims, up, xs[j]) <= k or _torus_l1(dims, dn, xs[j]) <= k
            if close:
                assert color[i] != color[j], (i, j)


def test_distance_one_coloring_is_the_checkerboard():
    """On an even torus the greedy distance-1 coloring in site order is the even/odd split."""
    dims = (4, 2, 4, 6)
    color, nc = opr.greedy_coloring(dims, 1, 0)
    assert nc == 2
    par = np.array([sum(_coords(dims, i)) % 2 for i in range(int(np.prod(dims)))])
    assert np.array_equal(color, par)


def test_pieces_partition_the_noise():
    """The pieces of a sample restrict one Z4 vector to disjoint supports that cover it."""
    dims = (2, 2, 2, 4)
    v = int(np.prod(dims))
    color, nc = opr.greedy_coloring(dims, 1, 0)
    z = philox.z4_noise(v, 77, 3, 1, 5)
    tot = np.zeros_like(z)
    for (j, a) in opr.pieces(nc, True):
        piece = opr.probed_noise(v, 77, 3, 1, 5, color, j, a)
        assert np.count_nonzero(piece) == np.count_nonzero(color == j)  # one component per site
        assert not np.any(tot[piece != 0])
        tot += piece
    assert np.array_equal(tot, z)


def test_exact_mean_and_variance_by_enumeration():
    """Brute force over all 4^6 Z4 vectors: the sum of the piece estimators has mean
    sum_i A_ii and the variance of the formula (pieces independent, off-diagonal squares)."""
    rng = np.random.default_rng(12)
    a = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    cls = [np.array([0, 2, 5]), np.array([1, 3]), np.array([4])]
    vals = []
    for ks in itertools.product(range(4), repeat=6):
        z = 1j ** np.array(ks)
        vals.append(sum(np.vdot(z[c], a[np.ix_(c, c)] @ z[c]) for c in cls))
    vals = np.array(vals)
    mean, var = opr.exact_mean_and_variance(a, cls)
    assert vals.mean() == pytest.approx(mean, rel=1e-12)
    assert np.mean(np.abs(vals - vals.mean()) ** 2) == pytest.approx(var, rel=1e-12)
    # one piece covering everything is plain Hutchinson
    m1, v1 = opr.exact_mean_and_variance(a, [np.arange(6)])
    assert m1 == pytest.approx(np.trace(a)) and v1 == pytest.approx(oest.exact_z4_variance(a))


def test_single_site_colors_with_dilution_give_the_exact_trace():
    """With every site its own color and full spin-color dilution every piece has one
    non-zero entry, so each level sample equals Tr(A_l) exactly (no noise)."""
    dims = (2, 2, 2, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=81)
    sig = [0.1, 0.5]
    gam = np.eye(4)
    colors = np.arange(v)
    solver = oest.make_dense_solver(u, -0.2, dims)
    got = opr.probed_level_samples(u, -0.2, sig, gam, 1, [2, 2], 5, 0, dims, colors, v, True,
                                   estimator=oest.DIFF, solver=solver)
    mats = oest.exact_level_matrices(u, -0.2, sig, gam, 1, dims, estimator=oest.DIFF)
    for lev in range(2):
        assert np.allclose(got[lev], np.trace(mats[lev]), rtol=1e-10, atol=1e-12), lev


@pytest.mark.parametrize("est", ["diff", "split_even"])
def test_probed_samples_match_the_dense_route(est):
    """The probed / diluted level sample equals sum_pieces z_piece^dag A_l z_piece with the
    dense level matrix (solves, contraction and levels checked against one dense product)."""
    dims = (2, 2, 4, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=82, eps=0.5)
    sig = [0.05, 0.4]
    gam = np.diag([1, 1, -1, -1]).astype(complex)
    color, nc = opr.greedy_coloring(dims, 1, 1)
    solver = oest.make_dense_solver(u, -0.25, dims)
    e = oest.ESTIMATORS[est]
    got = opr.probed_level_samples(u, -0.25, sig, gam, 1, [2, 1], 9, 4, dims, color, nc, True,
                                   estimator=e, solver=solver)
    mats = oest.exact_level_matrices(u, -0.25, sig, gam, 1, dims, estimator=e)
    for lev in range(2):
        for s in range(len(got[lev])):
            ref = 0j
            for (j, a) in opr.pieces(nc, True):
                z = opr.probed_noise(v, 9, 4, lev, s, color, j, a).ravel()
                ref += np.vdot(z, mats[lev] @ z)
            assert got[lev][s] == pytest.approx(ref, rel=1e-9, abs=1e-12), (lev, s)


def test_probing_removes_the_near_diagonal_variance():
    """On the lattice operator, distance-1 probing with dilution has a smaller exact variance
    than plain Z4 noise, and both estimators have expectation Tr(A)."""
    dims = (2, 2, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=83, eps=0.4)
    a = osolve.dense_inverse(u, -0.2, 0.3, dims, -1)
    color, nc = opr.greedy_coloring(dims, 1, 0)
    m_plain, v_plain = opr.exact_mean_and_variance(a, opr.classes(dims, None, 0, False))
    m_prob, v_prob = opr.exact_mean_and_variance(a, opr.classes(dims, color, nc, True))
    assert m_plain == pytest.approx(np.trace(a)) and m_prob == pytest.approx(np.trace(a))
    assert v_prob < 0.5 * v_plain


def test_probed_variance_sample_with_single_site_colours_is_exact():
    """Single-site colours and full dilution: every noise vector gives a_i = Tr(Gamma Omega_p A_i)
    and b_ij = Tr(A_i Gamma Omega_p A_j), A_i = (D + s_i)^-1 (the pieces are the unit vectors, and
    y^(i)^dag = e^dag A_i), so both sampled variances vanish."""
    dims = (2, 2, 2, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=84)
    s_hat = [0.1, 0.6]
    gam = np.diag([1, -1, 1, -1]).astype(complex)
    solver = oest.make_dense_solver(u, -0.2, dims)
    out = opr.probed_variance_sample(u, -0.2, s_hat, gam, [0, 1], 2, 3, 0, dims, np.arange(v), v, True,
                                     solver=solver)
    inv = [osolve.dense_inverse(u, -0.2, s, dims, -1) for s in s_hat]
    for pi, p in enumerate([0, 1]):
        g = osolve.dense_GammaOmega(u, gam, p, dims)
        for i in range(2):
            assert np.allclose(out["a"][:, pi, i], np.trace(g @ inv[i]), rtol=1e-10)
            for j in range(i, 2):
                assert np.allclose(out["b"][:, pi, i, j], np.trace(inv[i] @ g @ inv[j]), rtol=1e-10)
    scale = max(np.abs(out["a"]).max(), np.abs(out["b"]).max()) ** 2
    assert np.abs(out["VL"]).max() < 1e-12 * scale and np.abs(out["Vbar"]).max() < 1e-12 * scale


def test_probed_variance_sample_without_pieces_is_the_plain_algorithm():
    dims = (2, 2, 4, 2)
    u = inputs.gauge_field(dims, "smooth", seed=85, eps=0.5)
    solver = oest.make_dense_solver(u, -0.25, dims)
    gam = np.diag([1, 1, -1, -1]).astype(complex)
    a = opr.probed_variance_sample(u, -0.25, [0.05, 0.3], gam, [1], 3, 5, 1, dims, None, 0, False, solver=solver)
    b = oest.variance_sample(u, -0.25, [0.05, 0.3], gam, [1], 3, 5, 1, dims, -1, solver)
    for key in ("a", "b", "VL", "Vbar"):
        assert np.allclose(a[key], b[key], rtol=1e-13, atol=1e-13), key


def test_dilution_gives_the_adjoint_solution_without_a_solve():
    """Sec. 3.1: with full spin-colour dilution a piece z lives on one spin s, so gamma_5 z = eps z
    (eps = +1 for s < 2, -1 otherwise) and y = (D + s)^-dag z = gamma_5 (D + s)^-1 gamma_5 z equals
    eps gamma_5 x, x = (D + s)^-1 z: the identity the library's diluted variance sampling uses
    instead of a second solve, checked here against the adjoint solve taken as written."""
    dims = (2, 2, 4, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=86)
    solver = oest.make_dense_solver(u, -0.3, dims)
    color, nc = opr.greedy_coloring(dims, 1, 0)
    for comp in (0, 4, 7, 11):
        z = opr.probed_noise(v, 3, 0, 0, 1, color, 1, comp)
        eps = 1.0 if comp // 3 < 2 else -1.0
        y = oest.adjoint_solution(solver, z, 0.2)
        x = solver(z, 0.2)
        g5x = x * np.array([1, 1, -1, -1])[None, :, None]
        assert np.allclose(y, eps * g5x, rtol=1e-12, atol=1e-13), comp
