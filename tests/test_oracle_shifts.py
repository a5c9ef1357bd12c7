"""Pins of the oracle's shift selection and sample allocation (paper Sec. 3.2, 3.3,
Eq. (ml_cost_shifts), Eq. (opt_shifts), Eq. (num_samples), Eq. (total_var))."""

import itertools
import math

import numpy as np
import pytest

from oracle import shifts as osh


# ---------------------------------------------------------------- PCHIP
def test_pchip_matches_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(3, 9))
        x = np.sort(rng.uniform(0, 2, n))
        x[0] = 0.0
        if trial % 2:
            y = np.cumsum(rng.uniform(-0.2, 2.0, n))          # mostly monotone
        else:
            y = rng.normal(size=n)                            # sign changes
        xq = np.linspace(-0.3, 2.3, 57)                       # includes extrapolation
        ref = interp.PchipInterpolator(x, y, extrapolate=True)(xq)
        got = osh.interpolate(x, y, xq)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), trial


def test_two_points_are_linear_and_nodes_are_reproduced():
    assert np.allclose(osh.interpolate([1.0, 3.0], [2.0, 6.0], [0.0, 2.0, 4.0]), [0.0, 4.0, 8.0])
    x = np.array([0.0, 0.05, 0.25, 0.5, 1.0])
    y = np.array([3.0, 1.0, 0.5, -1.0, -4.0])
    assert np.allclose(osh.interpolate(x, y, x), y, atol=1e-14)


# ---------------------------------------------------------------- manifolds
S_HAT = np.array([0.0, 0.05, 0.25, 0.5, 1.0])


def test_log_linear_manifold_is_recovered_exactly():
    """ln Vbar(a, b) = c0 + c1 a + c2 b is reproduced exactly by every stage (PCHIP is exact
    on linear data); c1 != c2 so a transposed argument fails."""
    c0, c1, c2 = 1.5, -7.0, -3.0
    vbar = np.exp(c0 + c1 * S_HAT[:, None] + c2 * S_HAT[None, :])
    vbar = np.triu(vbar)  # only j >= i is sampled
    s = osh.paper_evaluation_set(S_HAT)
    V = osh.interp_pair(S_HAT, vbar, s)
    for i in range(0, len(s), 7):
        for k in range(i + 1, len(s), 5):
            ref = (s[k] - s[i]) ** 2 * math.exp(c0 + c1 * s[i] + c2 * s[k])
            assert V[i, k] == pytest.approx(ref, rel=1e-10), (i, k)
    assert np.all(np.isnan(V[np.tril_indices(len(s))]))
    VL = osh.interp_single(S_HAT, np.exp(2.0 - 4.0 * S_HAT), s)
    assert np.allclose(VL, np.exp(2.0 - 4.0 * s), rtol=1e-12)


def test_sampled_points_are_reproduced():
    rng = np.random.default_rng(8)
    vbar = np.triu(np.exp(rng.normal(size=(5, 5))))
    VL_hat = np.exp(rng.normal(size=5))
    s = osh.paper_evaluation_set(S_HAT)
    V = osh.interp_pair(S_HAT, vbar, s)
    VL = osh.interp_single(S_HAT, VL_hat, s)
    pos = [int(np.where(s == x)[0][0]) for x in S_HAT]
    for a in range(5):
        assert VL[pos[a]] == pytest.approx(VL_hat[a], rel=1e-12)
        for b in range(a + 1, 5):
            ref = (S_HAT[b] - S_HAT[a]) ** 2 * vbar[a, b]
            assert V[pos[a], pos[b]] == pytest.approx(ref, rel=1e-10), (a, b)


def test_paper_evaluation_set():
    s = osh.paper_evaluation_set(S_HAT)
    assert s[0] == 0.0 and s[-1] == 1.0 and np.all(np.diff(s) > 0)
    assert set(S_HAT).issubset(set(s))
    assert np.isclose(s[1], 1e-5) and np.isclose(s[4], 1e-2) and np.isclose(s[5], 0.011)
    assert len(s) == 84  # 0, the 80 grid points (1.0 among them), and 0.05, 0.25, 0.5


def test_next_neighbour_cost():
    r = osh.iteration_cost(S_HAT, [50, 40, 30, 20, 10], [0.0, 0.01, 0.05, 0.06, 0.5, 0.7, 1.0])
    assert list(r) == [50, 40, 40, 30, 20, 10, 10]


# ---------------------------------------------------------------- selection
def _toy():
    """Evaluation set = sampling set (n = 4): no interpolation between nodes matters."""
    s_hat = np.array([0.0, 0.1, 0.3, 1.0])
    VL_hat = np.array([64.0, 16.0, 4.0, 1.0])
    vbar = np.triu(np.full((4, 4), 100.0))
    r_hat = np.array([4.0, 4.0, 2.0, 1.0])
    return s_hat, VL_hat, vbar, r_hat


def test_selection_hand_worked():
    """L = 1 at n = 4 by hand. Candidates sigma_1 in {0.1, 0.3, 1.0}:
    F = sqrt((r0 + r1)(s1 - 0)^2 100) + sqrt(r1 VL(s1)):
      0.1: sqrt(8 * 0.01 * 100) + sqrt(4 * 16) = 2.828.. + 8  = 10.83
      0.3: sqrt(6 * 0.09 * 100) + sqrt(2 * 4)  = 7.348.. + 2.828.. = 10.18
      1.0: sqrt(5 * 1.00 * 100) + sqrt(1 * 1)  = 22.36 + 1 = 23.36"""
    s_hat, VL_hat, vbar, r_hat = _toy()
    idx, F = osh.select_shifts(s_hat, VL_hat, vbar, r_hat, s_hat, 1)
    assert idx == [0, 2]
    assert F == pytest.approx(math.sqrt(6 * 0.09 * 100) + math.sqrt(8.0), rel=1e-12)


def test_selection_scale_invariance_and_brute_force_consistency():
    rng = np.random.default_rng(21)
    s_hat = S_HAT
    vbar = np.triu(np.exp(rng.normal(size=(5, 5)) - 3 * s_hat[None, :]))
    VL_hat = np.exp(1.0 - 5 * s_hat + rng.normal(scale=0.1, size=5))
    r_hat = np.array([80.0, 60.0, 40.0, 30.0, 20.0])
    s = np.unique(np.concatenate([s_hat, np.linspace(0.0, 1.0, 15)]))
    idx, F = osh.select_shifts(s_hat, VL_hat, vbar, r_hat, s, 3)
    idx2, F2 = osh.select_shifts(s_hat, 9.0 * VL_hat, 9.0 * vbar, r_hat, s, 3)
    idx3, F3 = osh.select_shifts(s_hat, VL_hat, vbar, 4.0 * r_hat, s, 3)
    assert idx == idx2 == idx3
    assert F2 == pytest.approx(3 * F, rel=1e-12) and F3 == pytest.approx(2 * F, rel=1e-12)
    # every other admissible choice costs at least as much
    VL = osh.interp_single(s_hat, VL_hat, s)
    Vl = osh.interp_pair(s_hat, vbar, s)
    r = osh.iteration_cost(s_hat, r_hat, s)
    for comb in itertools.combinations(range(1, len(s)), 3):
        V, C = osh.level_terms((0,) + comb, VL, Vl, r)
        if not np.any(np.isnan(V)):
            assert np.sum(np.sqrt(C * V)) >= F * (1 - 1e-12)


# ---------------------------------------------------------------- allocation
def test_sample_allocation_lagrange_optimum():
    V = np.array([5.0, 2.0, 0.7, 0.05])
    C = np.array([90.0, 70.0, 50.0, 20.0])
    eps2 = 1e-3
    N, mu, V_FS, C_FS = osh.sample_allocation(V, C, eps2)
    assert V_FS == pytest.approx(eps2, rel=1e-12)                       # Eq. (total_var) at the optimum
    assert C_FS == pytest.approx(np.sum(np.sqrt(V * C)) ** 2 / eps2, rel=1e-12)  # Eq. (ml_cost_shifts)
    # any other allocation with the same total variance costs more
    rng = np.random.default_rng(5)
    for _ in range(50):
        M = N * np.exp(rng.normal(scale=0.3, size=4))
        M *= np.sum(V / M) / eps2  # rescale onto V_FS = eps2
        assert np.sum(V / M) == pytest.approx(eps2, rel=1e-12)
        assert np.sum(M * C) > C_FS * (1 - 1e-12)
