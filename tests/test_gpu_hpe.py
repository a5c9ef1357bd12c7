"""Hopping parameter expansion of the last level (paper Sec. 3.1, the remark after
Eq. (sampled_single)): the CUDA path against the oracle.

The GPU computes the exact low orders from its own displacement-p distance-(K-1) colouring and
the order-K remainder with FP64 kappa H applications after the solve; the oracle's exact part
comes from its own probing (pinned against dense matrices on the CPU) or from the closed forms.
Tolerances: relative 1e-9 with FP64 solves at 1e-12."""

import numpy as np
import pytest

import inputs
from oracle import dirac as odirac
from oracle import estimators as oest
from oracle import hpe as ohpe
from oracle import philox
from oracle import probing as opr
from helpers import sample_err

pkg = pytest.importorskip("paper_2212_04430_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def make_ctx(dims, u):
    ctx = pkg.Context(dims, bc_t=-1, device=0)
    ctx.fs_set_gauge(u)
    return ctx


def _oracle_last_level(u, m, sig, g, p, K, n, seed, job, dims, solver, colors=None, ncolors=0, dilute=False):
    v = int(np.prod(dims))
    col, nc = opr.greedy_coloring(dims, K - 1, p)
    t_exact = ohpe.exact_part_probed(u, m, sig, g, p, K, dims, col, nc) if K > 1 else \
        (3 * v * np.trace(g) if p == 0 else 0.0) / (4.0 + m + sig)
    L = len(n) - 1
    out = []
    for s in range(n[L]):
        tot = t_exact
        for (j, a) in opr.pieces(ncolors, dilute):
            z = opr.probed_noise(v, seed, job, L, s, colors, j, a)
            tot += ohpe.stochastic_part(u, solver, z, m, sig, g, p, K, dims)
        out.append(tot)
    return np.array(out), t_exact


@pytest.mark.parametrize("p,K", [(0, 4), (1, 4), (2, 3)])
def test_last_level_with_the_expansion(p, K):
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=401, eps=0.5)
    m = -0.2
    sig = [0.05, 0.6]  # m + sigma_L = 0.4 > 0: the last level takes the expansion
    n = [3, 6]
    g = pkg.gamma_matrix("g3")
    go = odirac.gamma_product(["g3"])
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(m, sig, g, p, n, seed=21, job=1, hpe_order=K, estimator="diff", prec="f64", tol=1e-12,
                               rhs_tile=16)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, m, dims)
    ref, _ = _oracle_last_level(u, m, sig[1], go, p, K, n, 21, 1, dims, solver)
    assert sample_err(out["samples"][1], ref) < 1e-9
    # the level below is untouched
    ref0 = oest.level_samples(u, m, sig, go, p, n, 21, 1, dims, -1, oest.DIFF, solver)[0]
    assert sample_err(out["samples"][0], ref0) < 1e-9
    ctx.close()


def test_exact_part_matches_the_closed_form():
    """p = 1, K = 2: T_exact = kappa 3V tr(Gamma (1 + gamma_z)) / A for any gauge field, so each
    GPU sample minus the oracle's remainder is that number."""
    dims = (4, 4, 6, 4)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=402)
    m, sig = 0.1, [0.4]
    A = 4.0 + m + sig[0]
    for name in ("g3", "g5g3"):
        g = pkg.gamma_matrix(name)
        go = odirac.gamma_product([name[i:i + 2] for i in range(0, len(name), 2)])
        closed = 3 * v * np.trace(go @ (odirac.IDENT4 + odirac.GAMMA[2])) / (2 * A) / A
        ctx = make_ctx(dims, u)
        out = ctx.mlmc_level_trace(m, sig, g, 1, [2], seed=3, hpe_order=2, prec="f64", tol=1e-12, rhs_tile=8)
        ctx.close()
        solver = oest.make_solver(u, m, dims)
        for s in range(2):
            z = philox.z4_noise(v, 3, 0, 0, s)
            rem = ohpe.stochastic_part(u, solver, z, m, sig[0], go, 1, 2, dims)
            assert abs(out["samples"][0][s] - rem - closed) <= 1e-8 * max(1.0, abs(closed)), (name, s)


def test_expansion_with_probing_dilution_and_lanes():
    """The expansion's own colours and the caller's probing colours in one call (the exact part
    runs first), two lanes against one, and the server."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=403, eps=0.4)
    m, sig, p, K = -0.1, [0.1, 0.5], 1, 4
    n = [2, 2]
    g = pkg.gamma_matrix("g3")
    col, nc = opr.greedy_coloring(dims, 1, 1)
    ctx = make_ctx(dims, u)
    kw = dict(colors=col, ncolors=nc, dilute=True, hpe_order=K, prec="f64", tol=1e-12, rhs_tile=32)
    one = ctx.mlmc_level_trace(m, sig, g, p, n, seed=8, job=2, lanes=1, **kw)
    two = ctx.mlmc_level_trace(m, sig, g, p, n, seed=8, job=2, lanes=2, **kw)
    ctx.close()
    assert one["rc"] == 0 and two["rc"] == 0
    for lev in range(2):
        assert np.array_equal(one["samples"][lev], two["samples"][lev]), lev
    solver = oest.make_dense_solver(u, m, dims)
    ref, _ = _oracle_last_level(u, m, sig[1], odirac.gamma_product(["g3"]), p, K, n, 8, 2, dims, solver, col, nc,
                                True)
    assert sample_err(one["samples"][1], ref) < 1e-9
    srv = pkg.Server(device=0, hbm_budget_bytes=8 << 30, max_active=1)
    t = srv.submit(dims, u, m, sig, g, p, n, 8, job=2, **kw)
    r = srv.poll(t)
    srv.close()
    assert r["status"] == 0 and np.array_equal(r["trace"], one["trace"])


def test_expansion_reduces_the_last_level_variance():
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=404, eps=0.4)
    m, sig = -0.2, [0.8]
    g = pkg.gamma_matrix("g3")
    ctx = make_ctx(dims, u)
    kw = dict(prec="f32", tol=1e-9, rhs_tile=64)
    plain = ctx.mlmc_level_trace(m, sig, g, 1, [128], seed=30, **kw)
    hpe = ctx.mlmc_level_trace(m, sig, g, 1, [128], seed=30, hpe_order=4, **kw)
    ctx.close()
    assert hpe["var"][0] < 0.5 * plain["var"][0]
    se = np.sqrt(plain["var"][0] / 128 + hpe["var"][0] / 128)
    assert abs(hpe["trace"][0] - plain["trace"][0]) < 5 * se


def test_variance_sampling_with_the_expansion():
    """a_i is the order-K remainder at the shifts with m + s_i > 0 (the others keep the plain
    sample); b_ij is unchanged."""
    dims = (4, 4, 4, 4)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=405, eps=0.5)
    m, s_hat, K = -0.3, [0.1, 0.5, 1.0], 4
    g = pkg.gamma_matrix("g3")
    go = odirac.gamma_product(["g3"])
    ctx = make_ctx(dims, u)
    out = ctx.variance_sample(m, s_hat, g, [0, 2], 3, seed=14, job=0, hpe_order=K, prec="f64", tol=1e-12,
                              rhs_tile=12)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, m, dims)
    plain = oest.variance_sample(u, m, s_hat, go, [0, 2], 3, 14, 0, dims, -1, solver)
    a_ref = plain["a"].copy()
    for k in range(3):
        z = philox.z4_noise(v, 14, 0, philox.VARIANCE_SAMPLE_LEVEL, k)
        for pi, p in enumerate([0, 2]):
            for i, s in enumerate(s_hat):
                if m + s > 0:
                    a_ref[k, pi, i] = ohpe.stochastic_part(u, solver, z, m, s, go, p, K, dims)
    assert np.abs(out["a"] - a_ref).max() < 1e-9 * np.abs(a_ref).max()
    assert np.abs(out["b"] - plain["b"]).max() < 1e-9 * np.abs(plain["b"]).max()
    assert np.allclose(out["VL"], oest.practical_variance(a_ref), rtol=1e-7, atol=1e-12)
    ctx.close()


def test_expansion_edge_cases():
    """Order 1 (the exact part is order 0 alone, no probing); the product estimator's last level;
    m + sigma_L <= 0 leaves the samples plain; p >= Lz and orders outside 0..8 are refused."""
    dims = (4, 4, 4, 4)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=406, eps=0.4)
    g = pkg.gamma_matrix("g3")
    go = odirac.gamma_product(["g3"])
    ctx = make_ctx(dims, u)
    kw = dict(prec="f64", tol=1e-12, rhs_tile=8)
    solver = oest.make_dense_solver(u, -0.1, dims)
    # K = 1, p = 0: T_exact = 3V tr(Gamma) / A = 0 for gamma_3; the remainder takes one kappa H
    one = ctx.mlmc_level_trace(-0.1, [0.2, 0.5], g, 0, [1, 3], seed=4, estimator="product", hpe_order=1, **kw)
    assert one["rc"] == 0
    for s in range(3):
        z = philox.z4_noise(v, 4, 0, 1, s)
        ref = ohpe.stochastic_part(u, solver, z, -0.1, 0.5, go, 0, 1, dims)
        assert abs(one["samples"][1][s] - ref) < 1e-9 * max(1.0, abs(ref))
    # m + sigma_L <= 0: no expansion
    a = ctx.mlmc_level_trace(-0.6, [0.3], g, 1, [2], seed=5, hpe_order=4, **kw)
    b = ctx.mlmc_level_trace(-0.6, [0.3], g, 1, [2], seed=5, **kw)
    assert np.array_equal(a["samples"][0], b["samples"][0])
    for bad in (dict(p=4, hpe_order=4), dict(p=1, hpe_order=9), dict(p=1, hpe_order=-1)):
        with pytest.raises(pkg.FsError) as e:
            ctx.mlmc_level_trace(-0.1, [0.5], g, bad["p"], [1], seed=1, hpe_order=bad["hpe_order"], **kw)
        assert e.value.code == pkg.fsmlmc.FS_ERR_ARG
    ctx.close()
