"""Shift selection and sample allocation: the library (host code, no GPU) against the
oracle on the same sampled variances (paper Sec. 3.2-3.3).

Tolerances: interpolated variances relative 1e-11 (the same formulas in a different
evaluation order, then exp); the selected indices exactly (the argmin is unique on these
inputs; a near-tie within 1e-12 relative would be reported as such); F relative 1e-12."""

import numpy as np
import pytest

from oracle import shifts as osh

pkg = pytest.importorskip("paper_2212_04430_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


S_HAT = np.array([0.0, 0.05, 0.25, 0.5, 1.0])


def _sampled(seed, m=5):
    """Variances shaped like the paper's (Fig. boundary): Vbar falls steeply away from 0,
    then near-exponentially; V_L likewise; iteration counts fall with the shift."""
    rng = np.random.default_rng(seed)
    s_hat = S_HAT if m == 5 else np.concatenate([[0.0], np.sort(rng.uniform(0.01, 1.0, m - 1))])
    a, b = s_hat[:, None], s_hat[None, :]
    vbar = np.exp(4.0 - 6.0 * np.sqrt(a) - 3.0 * b + rng.normal(scale=0.2, size=(m, m)))
    vbar = np.triu(vbar)
    VL = np.exp(3.0 - 5.0 * s_hat + rng.normal(scale=0.2, size=m))
    iters = np.round(120.0 * np.exp(-1.5 * s_hat) + rng.integers(0, 5, m))
    return s_hat, VL, vbar, iters


def test_evaluation_grid():
    for s_hat in (S_HAT, np.array([0.005, 0.05, 0.25, 0.5, 1.0])):
        s = pkg.fs_eval_grid(s_hat)
        ref = osh.paper_evaluation_set(s_hat)
        assert len(s) == len(ref) and np.allclose(s, ref, rtol=1e-14, atol=0)
        assert s[0] == s_hat[0]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_interpolated_manifolds(seed):
    s_hat, VL_hat, vbar, _ = _sampled(seed)
    s = osh.paper_evaluation_set(s_hat)
    VL, Vl = pkg.fs_interp_variances(s_hat, VL_hat, vbar, s)
    assert np.allclose(VL, osh.interp_single(s_hat, VL_hat, s), rtol=1e-11, atol=0)
    ref = osh.interp_pair(s_hat, vbar, s)
    both = ~np.isnan(ref)
    assert np.array_equal(both, ~np.isnan(Vl))
    assert np.allclose(Vl[both], ref[both], rtol=1e-11, atol=0)


@pytest.mark.parametrize("seed,L,m,s0", [(0, 1, 5, 0.0), (1, 2, 5, 0.0), (2, 3, 5, 0.0), (3, 2, 4, 0.0),
                                         (4, 3, 6, 0.0), (5, 3, 5, 0.005)])
def test_selected_shifts_match_brute_force(seed, L, m, s0):
    s_hat, VL_hat, vbar, iters = _sampled(seed, m)
    s_hat = s_hat.copy()
    s_hat[0] = s0
    s = np.unique(np.concatenate([s_hat, np.linspace(0.0, 1.0, 21), [1e-3, 1e-2]]))
    s = s[s >= s0]
    got = pkg.fs_select_shifts(s_hat, VL_hat, vbar, iters, s, L)
    idx, F = osh.select_shifts(s_hat, VL_hat, vbar, iters, s, L)
    assert got["F"] == pytest.approx(F, rel=1e-12)
    assert got["idx"] == idx
    assert np.allclose(got["sigma"], s[idx])
    VL = osh.interp_single(s_hat, VL_hat, s)
    Vl = osh.interp_pair(s_hat, vbar, s)
    r = osh.iteration_cost(s_hat, iters, s)
    V, C = osh.level_terms(idx, VL, Vl, r)
    assert np.allclose(got["V"], V, rtol=1e-11) and np.array_equal(got["C"], C)


def test_paper_sized_selection_six_shifts():
    """n = 84 evaluation shifts, six shifts (seven levels) as in the paper's runs: the DP
    minimiser beats 2000 random admissible choices and every single-index move of itself."""
    s_hat, VL_hat, vbar, iters = _sampled(7)
    s = pkg.fs_eval_grid(s_hat)
    got = pkg.fs_select_shifts(s_hat, VL_hat, vbar, iters, s, 6)
    VL = osh.interp_single(s_hat, VL_hat, s)
    Vl = osh.interp_pair(s_hat, vbar, s)
    r = osh.iteration_cost(s_hat, iters, s)

    def F(ix):
        V, C = osh.level_terms(ix, VL, Vl, r)
        return np.inf if np.any(np.isnan(V)) else float(np.sum(np.sqrt(V * C)))

    best = got["idx"]
    assert F(best) == pytest.approx(got["F"], rel=1e-12)
    rng = np.random.default_rng(9)
    for _ in range(2000):
        ix = [0] + sorted(rng.choice(np.arange(1, len(s)), 6, replace=False).tolist())
        assert F(ix) >= got["F"] * (1 - 1e-12)
    for l in range(1, 7):
        for k in range(best[l - 1] + 1, best[l + 1] if l < 6 else len(s)):
            ix = list(best)
            ix[l] = k
            assert F(ix) >= got["F"] * (1 - 1e-12)


def test_sample_allocation_parity_and_errors():
    V = np.array([3.0, 1.2, 0.4, 0.02])
    C = np.array([200.0, 150.0, 90.0, 30.0])
    N, mu, vfs, cfs = pkg.fs_sample_allocation(V, C, 2e-4)
    N2, mu2, vfs2, cfs2 = osh.sample_allocation(V, C, 2e-4)
    assert np.allclose(N, N2, rtol=1e-13) and mu == pytest.approx(mu2, rel=1e-13)
    assert vfs == pytest.approx(vfs2, rel=1e-13) and cfs == pytest.approx(cfs2, rel=1e-13)
    with pytest.raises(pkg.FsError):
        pkg.fs_sample_allocation(V, C, 0.0)
    with pytest.raises(pkg.FsError):
        pkg.fs_sample_allocation(V, -C, 1e-3)
    s_hat, VL_hat, vbar, iters = _sampled(1)
    with pytest.raises(pkg.FsError):
        pkg.fs_select_shifts(s_hat, VL_hat, vbar, iters, np.array([0.1, 0.5, 1.0]), 1)  # s_0 != s^_0
    with pytest.raises(pkg.FsError):
        pkg.fs_select_shifts(s_hat, -VL_hat, vbar, iters, S_HAT, 1)
