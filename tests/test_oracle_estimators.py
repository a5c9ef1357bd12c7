"""Pins of the oracle's noise and estimator layer.

Exact identities (telescoping, one-end trick, cyclic equality), the exact
Z4 mean and variance from dense inverses, and the published Philox
known-answer vectors.
"""

import os

import numpy as np
import pytest

import inputs
from oracle import dirac, estimators, philox, solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[:4], w[4:6], w[6:]))
    return rows


def _shift_sets():
    sets = {}
    with open(os.path.join(GOLDEN, "paper_shift_sets.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t = line.split()
                sets[t[0]] = [float(x) for x in t[1:]]
    return sets


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(*ctr, *key)
        assert [int(g) for g in got] == out


def test_z4_noise_statistics():
    """Each of {1, i, -1, -i} with frequency 1/4; distinct (site, level, sample) counters
    give uncorrelated entries."""
    v = 4096
    k = philox.z4_codes(v, seed=2024, job=0, level=0, sample=0).ravel()
    n = k.size
    for val in range(4):
        f = np.count_nonzero(k == val)
        assert abs(f - n / 4) < 5 * np.sqrt(n * 3 / 16)
    z0 = philox.z4_noise(v, 2024, 0, 0, 0).ravel()
    z1 = philox.z4_noise(v, 2024, 0, 1, 0).ravel()
    z2 = philox.z4_noise(v, 2024, 0, 0, 1).ravel()
    for other in (z1, z2):
        c = np.vdot(z0, other) / n
        assert abs(c) < 5 / np.sqrt(n)
    assert np.allclose(np.abs(z0), 1.0)
    g5 = philox.z4_noise(v, 2024, 0, 0, 0, gamma5=True)
    assert np.allclose(g5, dirac.spin_mul(dirac.GAMMA5, z0.reshape(v, 4, 3)))


def _small_setup(seed=81):
    dims = (2, 2, 2, 2)
    u = inputs.gauge_field(dims, "haar", seed=seed)
    return dims, u


@pytest.mark.parametrize("estimator", [estimators.DIFF, estimators.SPLIT_EVEN, estimators.PRODUCT])
def test_telescoping_sum_exact(estimator):
    """Eq. (tele_sum) / (tele_sum_prod_disp): the level traces add up to
    Tr(Gamma Omega_p (D + sigma_0)^-1) for any sigma_0."""
    dims, u = _small_setup()
    sig = _shift_sets()["optimal_g3_p4"]
    gam = dirac.GAMMA[2]
    for p in (0, 1):
        mats = estimators.exact_level_matrices(u, -0.4, sig, gam, p, dims, -1, estimator)
        total = sum(np.trace(a) for a in mats)
        ref = np.trace(solve.dense_GammaOmega(u, gam, p, dims) @ solve.dense_inverse(u, -0.4, sig[0], dims))
        assert abs(total - ref) < 1e-11 * max(1.0, abs(ref))


def test_one_end_trick_identity():
    """A^-1 (A - B) B^-1 = B^-1 - A^-1 with A - B = (s1 - s0) I (Sec. 2.2)."""
    dims, u = _small_setup()
    a = solve.dense_operator(u, -0.3, 0.4, dims)
    b = solve.dense_operator(u, -0.3, 0.1, dims)
    ai, bi = np.linalg.inv(a), np.linalg.inv(b)
    assert np.abs(ai @ (a - b) @ bi - (bi - ai)).max() < 1e-12
    assert np.abs((a - b) - 0.3 * np.eye(a.shape[0])).max() < 1e-14


def test_split_even_cyclic_equality():
    """Eq. (cyclic_commute): equal traces, different matrices."""
    dims, u = _small_setup(82)
    gam = solve.dense_GammaOmega(u, dirac.gamma_product(["g5", "g4"]), 0, dims)
    i0 = solve.dense_inverse(u, -0.3, 0.05, dims)
    i1 = solve.dense_inverse(u, -0.3, 0.25, dims)
    lhs = gam @ i0 @ i1
    rhs = i0 @ gam @ i1
    assert abs(np.trace(lhs) - np.trace(rhs)) < 1e-11
    assert np.abs(lhs - rhs).max() > 1e-3


def test_practical_variance_normalisation_by_hand():
    """Eq. (practical_variance) as printed divides by N (reading C6), not N - 1. Sample sets
    worked by hand: {1, i, -1, -i} has mean 0 and mean |c|^2 = 1, so 1 (N - 1 would give 4/3);
    {2, 4}: 10 - 9 = 1 (N - 1: 2); {1+i, 1-i, 3+i}: 14/3 - 26/9 = 16/9 (N - 1: 8/3). A column
    per sample set checks that levels are kept apart."""
    assert abs(estimators.practical_variance([1, 1j, -1, -1j]) - 1.0) < 1e-12
    assert abs(estimators.practical_variance([2.0, 4.0]) - 1.0) < 1e-12
    assert abs(estimators.practical_variance([1 + 1j, 1 - 1j, 3 + 1j]) - 16.0 / 9.0) < 1e-12
    cols = np.array([[1, 2.0], [1j, 4.0], [-1, 2.0], [-1j, 4.0]])
    assert np.allclose(estimators.practical_variance(cols), [1.0, 1.0], rtol=0, atol=1e-12)
    # a constant set has no variance, a single sample none either (up to the rounding of the
    # one-pass form)
    assert abs(estimators.practical_variance([3 - 2j] * 5)) < 1e-12
    assert abs(estimators.practical_variance([7.5])) < 1e-12


def _mc_check(samples, exact_mean, exact_var):
    c = np.asarray(samples)
    n = c.size
    mean = c.mean()
    var = estimators.practical_variance(c)
    se_mean = np.sqrt(var / n)
    d2 = np.abs(c - mean) ** 2
    se_var = d2.std() / np.sqrt(n)
    assert abs(mean - exact_mean) < 5 * se_mean + 1e-12, (mean, exact_mean, se_mean)
    assert abs(var - exact_var) < 5 * se_var + 1e-12, (var, exact_var, se_var)
    return var, se_var


def test_hutchinson_z4_mean_and_variance():
    """Eq. (test) is unbiased; its Z4 variance is ||A||_F^2 - sum |A_ii|^2, which
    Eq. (practical_variance) estimates. The printed factor 2 of Eq. (test_var) is
    far outside the statistical error for Z4 noise."""
    dims, u = _small_setup(83)
    v = int(np.prod(dims))
    a = solve.dense_GammaOmega(u, dirac.GAMMA[2], 1, dims) @ solve.dense_inverse(u, -0.4, 0.1, dims)
    ns = 20000
    zs = np.stack([philox.z4_noise(v, 7, 0, 0, s).ravel() for s in range(ns)])
    c = np.einsum("si,ij,sj->s", zs.conj(), a, zs)
    var, se = _mc_check(c, np.trace(a), estimators.exact_z4_variance(a))
    assert abs(var - estimators.exact_var_paper(a)) > 20 * se


@pytest.mark.parametrize("estimator", [estimators.DIFF, estimators.SPLIT_EVEN, estimators.PRODUCT])
def test_level_samples_match_exact_levels(estimator):
    """The oracle's per-level samples (Eq. (fs_trace_est)) have the exact dense level
    trace as mean and the exact Z4 variance of the level matrix as variance."""
    dims, u = _small_setup(84)
    sig = [0.0, 0.1, 0.5]
    gam = dirac.gamma_product(["g5", "g3"])
    p = 1
    solver = estimators.make_dense_solver(u, -0.2, dims)
    n = [3000, 3000, 3000]
    out = estimators.mlmc_level_trace(u, -0.2, sig, gam, p, n, 99, 3, dims, -1, estimator, solver)
    mats = estimators.exact_level_matrices(u, -0.2, sig, gam, p, dims, -1, estimator)
    for lev in range(3):
        _mc_check(out["samples"][lev], np.trace(mats[lev]), estimators.exact_z4_variance(mats[lev]))


def test_diff_equals_product_on_same_noise():
    """One-end trick: DIFF and PRODUCT samples agree value by value on the same noise."""
    dims, u = _small_setup(85)
    sig = [0.0, 0.05, 0.3]
    solver = estimators.make_dense_solver(u, -0.3, dims)
    kw = dict(dims=dims, bc_t=-1, solver=solver)
    d = estimators.level_samples(u, -0.3, sig, dirac.GAMMA[3], 2, [20, 20, 20], 5, 1, estimator=estimators.DIFF, **kw)
    q = estimators.level_samples(u, -0.3, sig, dirac.GAMMA[3], 2, [20, 20, 20], 5, 1, estimator=estimators.PRODUCT, **kw)
    for a, b in zip(d, q):
        assert np.abs(a - b).max() < 1e-10 * max(1.0, np.abs(a).max())


def test_adjoint_solution_solves_dagger_system():
    """y = gamma_5 (D+s)^-1 gamma_5 z solves (D+s)^dag y = z (Eq. (conj_shifted_linear_systems))."""
    dims, u = _small_setup(86)
    v = int(np.prod(dims))
    z = philox.z4_noise(v, 1, 0, 0, 0)
    solver = estimators.make_solver(u, -0.4, dims)
    y = estimators.adjoint_solution(solver, z, 0.15)
    d = solve.dense_operator(u, -0.4, 0.15, dims)
    assert np.abs(d.conj().T @ y.ravel() - z.ravel()).max() < 1e-10


def test_variance_sample_matches_exact():
    """Sec. 3.1 algorithm: a_i and b_ij have the exact traces and Z4 variances of
    Gamma Omega_p (D+s_i)^-1 and (D+s_i)^-1 Gamma Omega_p (D+s_j)^-1."""
    dims, u = _small_setup(87)
    s_hat = _shift_sets()["sampling"]
    gam = dirac.GAMMA[2]
    plist = [0, 2]
    solver = estimators.make_dense_solver(u, -0.3, dims)
    ns = 3000
    out = estimators.variance_sample(u, -0.3, s_hat, gam, plist, ns, 17, 0, dims, -1, solver)
    inv = [solve.dense_inverse(u, -0.3, s, dims) for s in s_hat]
    for pi, p in enumerate(plist):
        go = solve.dense_GammaOmega(u, gam, p, dims)
        for i in range(len(s_hat)):
            a = go @ inv[i]
            _mc_check(out["a"][:, pi, i], np.trace(a), estimators.exact_z4_variance(a))
            assert abs(out["VL"][pi, i] - estimators.practical_variance(out["a"][:, pi, i])) < 1e-12
            for j in range(i, len(s_hat)):
                b = inv[i] @ go @ inv[j]
                _mc_check(out["b"][:, pi, i, j], np.trace(b), estimators.exact_z4_variance(b))
                assert abs(out["Vl"][pi, i, j] - (s_hat[j] - s_hat[i]) ** 2 * out["Vbar"][pi, i, j]) < 1e-12
