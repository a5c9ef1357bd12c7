"""Probed and spin-colour diluted level traces (paper Sec. 2.1, Eq. (probing_vectors),
displacement-p probing; Sec. 3.1 full spin-colour dilution): the CUDA path against the oracle.

A sample is the sum of the level estimator over its pieces (the sample's Z4 vector restricted
to one colour and one spin-colour index). Tolerances as for plain level samples: relative 1e-9
with FP64 solves at 1e-12, 1e-6 with FP16 solves at 1e-10, normalised by max(|T|, mean |c|)."""

import numpy as np
import pytest

import inputs
from oracle import dirac as odirac
from oracle import estimators as oest
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


@pytest.mark.parametrize("est", ["diff", "split_even", "product"])
def test_probed_diluted_samples(est):
    """Displacement-1 distance-1 probing (4 colours) with full dilution: 48 pieces a sample,
    Gamma = gamma_3, Omega_1."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=301, eps=0.5)
    sig = [0.02, 0.3]
    n = [2, 2]
    col, nc = opr.greedy_coloring(dims, 1, 1)
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.3, sig, pkg.gamma_matrix("g3"), 1, n, seed=41, job=2, estimator=est,
                               colors=col, ncolors=nc, dilute=True, prec="f64", tol=1e-12, rhs_tile=32)
    assert out["rc"] == 0
    assert len(out["stats"]) == 12 * nc * (2 * n[0] + n[1])
    solver = oest.make_dense_solver(u, -0.3, dims)
    ref = opr.probed_level_samples(u, -0.3, sig, odirac.gamma_product(["g3"]), 1, n, 41, 2, dims, col, nc, True,
                                   estimator=oest.ESTIMATORS[est], solver=solver)
    for lev in range(2):
        assert sample_err(out["samples"][lev], ref[lev]) < 1e-9, (est, lev)
    ctx.close()


@pytest.mark.parametrize("mode", ["probing", "dilution"])
def test_probing_or_dilution_alone_mixed_precision(mode):
    """Colours without dilution (distance-2, displacement-2: 8 colours) or dilution without
    colours (12 pieces), FP16 storage, a ragged last tile."""
    dims = (4, 2, 8, 4)
    u = inputs.gauge_field(dims, "smooth", seed=302, eps=0.4)
    sig = [0.01, 0.1, 0.6]
    n = [3, 2, 1]
    if mode == "probing":
        col, nc = opr.greedy_coloring(dims, 2, 2)
        kw = dict(colors=col, ncolors=nc, dilute=False)
    else:
        col, nc = None, 0
        kw = dict(dilute=True)
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.25, sig, pkg.gamma_matrix("g5g3"), 2, n, seed=43, job=0, estimator="diff",
                               prec="f16", tol=1e-10, rhs_tile=24, **kw)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, -0.25, dims)
    ref = opr.probed_level_samples(u, -0.25, sig, odirac.gamma_product(["g5", "g3"]), 2, n, 43, 0, dims, col, nc,
                                   mode == "dilution", estimator=oest.DIFF, solver=solver)
    for lev in range(3):
        assert sample_err(out["samples"][lev], ref[lev]) < 1e-6, (mode, lev)
    ctx.close()


def test_single_site_colours_with_dilution_give_the_exact_trace():
    """Every site its own colour and full dilution: every piece has one non-zero entry, so each
    level sample is the exact level trace (checked against the dense level matrices, not the
    oracle's estimator)."""
    dims = (2, 2, 4, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=303)
    sig = [0.05, 0.5]
    col = np.arange(v, dtype=np.int32)
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.2, sig, pkg.gamma_matrix("g3"), 1, [1, 1], seed=7, estimator="diff",
                               colors=col, dilute=True, prec="f64", tol=1e-12, rhs_tile=64)
    assert out["rc"] == 0
    mats = oest.exact_level_matrices(u, -0.2, sig, odirac.gamma_product(["g3"]), 1, dims, -1, oest.DIFF)
    for lev in range(2):
        exact = np.trace(mats[lev])
        assert abs(out["samples"][lev][0] - exact) <= 1e-9 * max(abs(exact), 1.0), lev
        assert abs(out["var"][lev]) <= 1e-12 * max(abs(exact) ** 2, 1.0)  # one sample: no spread
    ctx.close()


def test_probing_reduces_the_variance():
    """Distance-1 probing with dilution against plain Z4 noise on the same lattice: both means
    agree with the exact trace, and the sampled variances follow the exact ones (the probed
    variance well below the plain one)."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=304, eps=0.4)
    sig = [0.4]
    col, nc = opr.greedy_coloring(dims, 1, 0)
    ctx = make_ctx(dims, u)
    kw = dict(prec="f32", tol=1e-9, rhs_tile=64)
    plain = ctx.mlmc_level_trace(-0.3, sig, np.eye(4), 0, [96], seed=5, **kw)
    probed = ctx.mlmc_level_trace(-0.3, sig, np.eye(4), 0, [8], seed=6, colors=col, dilute=True, **kw)
    a = oest.exact_level_matrices(u, -0.3, sig, odirac.IDENT4, 0, dims, -1, oest.DIFF)[0]
    m0, v_plain = opr.exact_mean_and_variance(a, opr.classes(dims, None, 0, False))
    _, v_prob = opr.exact_mean_and_variance(a, opr.classes(dims, col, nc, True))
    assert v_prob < 0.5 * v_plain
    assert abs(plain["trace"][0] - m0) < 5 * np.sqrt(v_plain / 96)
    assert abs(probed["trace"][0] - m0) < 5 * np.sqrt(v_prob / 8) + 1e-6 * abs(m0)
    assert 0.3 * v_plain < plain["var"][0] < 2.5 * v_plain
    assert probed["var"][0] < 4.0 * v_prob
    ctx.close()


def test_lanes_and_server_give_identical_probed_results():
    """The colour table is shared by the lanes and copied by the server: the same per-sample
    values as one lane on a context."""
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=305, eps=0.4)
    sig = [0.02, 0.2, 0.8]
    n = [3, 2, 2]
    col, nc = pkg.fs_probing_colors(dims, 2, 1)
    g = pkg.gamma_matrix("g3")
    kw = dict(prec="f16", tol=1e-8, rhs_tile=16)
    ctx = make_ctx(dims, u)
    one = ctx.mlmc_level_trace(-0.3, sig, g, 1, n, seed=9, job=4, colors=col, ncolors=nc, lanes=1, **kw)
    two = ctx.mlmc_level_trace(-0.3, sig, g, 1, n, seed=9, job=4, colors=col, ncolors=nc, lanes=2, **kw)
    ctx.close()
    for lev in range(3):
        assert np.array_equal(one["samples"][lev], two["samples"][lev]), lev
    srv = pkg.Server(device=0, hbm_budget_bytes=8 << 30, max_active=2)
    t = srv.submit(dims, u, -0.3, sig, g, 1, n, 9, job=4, colors=col, ncolors=nc, **kw)
    r = srv.poll(t)
    srv.close()
    assert r["status"] == 0 and r["solves"] == len(one["stats"])
    assert np.array_equal(r["trace"], one["trace"])
    assert np.array_equal(r["var"], one["var"])


def test_bad_colour_tables_are_refused():
    dims = (4, 4, 4, 4)
    u = inputs.unit_gauge(dims)
    ctx = make_ctx(dims, u)
    col = np.zeros(256, dtype=np.int32)
    col[::2] = 1
    for bad, nc in ((col, 3), (col - 1, 2), (col + 1, 2)):   # unused colour; out of range
        with pytest.raises(pkg.FsError) as e:
            ctx.mlmc_level_trace(-0.3, [0.1], np.eye(4), 0, [1], seed=1, colors=bad, ncolors=nc)
        assert e.value.code == pkg.fsmlmc.FS_ERR_ARG
    ctx.close()


# ---------------------------------------------------------------- variance sampling
def _cmp_variance(out, ref, tol):
    for key in ("a", "b"):
        scale = max(np.abs(ref[key]).max(), 1e-300)
        assert np.abs(out[key] - ref[key]).max() < tol * scale, key
    for key in ("VL", "Vbar"):
        scale = max(np.abs(ref["a" if key == "VL" else "b"]).max() ** 2, 1e-300)
        assert np.abs(out[key] - ref[key]).max() < 10 * tol * scale, key


def test_variance_sample_probed_and_diluted():
    """Full dilution takes y^(i) = +-gamma_5 x^(i) instead of the adjoint solve; the oracle solves
    the adjoint system as written, so this checks the shortcut along with the pieces."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=306, eps=0.5)
    s_hat = [0.02, 0.2, 0.8]
    col, nc = opr.greedy_coloring(dims, 1, 1)
    ctx = make_ctx(dims, u)
    out = ctx.variance_sample(-0.3, s_hat, pkg.gamma_matrix("g3"), [0, 1, 2], 2, seed=12, job=1, colors=col,
                              ncolors=nc, dilute=True, prec="f64", tol=1e-12, rhs_tile=30)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, -0.3, dims)
    ref = opr.probed_variance_sample(u, -0.3, s_hat, odirac.gamma_product(["g3"]), [0, 1, 2], 2, 12, 1, dims, col,
                                     nc, True, solver=solver)
    _cmp_variance(out, ref, 1e-9)
    ctx.close()


def test_variance_sample_probed_without_dilution_mixed_precision():
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=307, eps=0.4)
    s_hat = [0.05, 0.5]
    col, nc = opr.greedy_coloring(dims, 2, 0)
    ctx = make_ctx(dims, u)
    out = ctx.variance_sample(-0.25, s_hat, pkg.gamma_matrix("g5g3"), [1], 3, seed=13, colors=col, ncolors=nc,
                              prec="f32", tol=1e-10, rhs_tile=32)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, -0.25, dims)
    ref = opr.probed_variance_sample(u, -0.25, s_hat, odirac.gamma_product(["g5", "g3"]), [1], 3, 13, 0, dims, col,
                                     nc, False, solver=solver)
    _cmp_variance(out, ref, 1e-6)
    ctx.close()


def test_variance_sample_single_site_colours_is_exact():
    """Single-site colours and full dilution: a_i = Tr(Gamma Omega_p A_i) and
    b_ij = Tr(A_i Gamma Omega_p A_j) for every noise vector (dense matrices, not the oracle's
    sampling code), and both variances vanish."""
    from oracle import solve as osolve
    dims = (2, 2, 4, 2)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "haar", seed=308)
    s_hat = [0.1, 0.6]
    ctx = make_ctx(dims, u)
    out = ctx.variance_sample(-0.2, s_hat, pkg.gamma_matrix("g3"), [0, 1], 2, seed=3, colors=np.arange(v),
                              dilute=True, prec="f64", tol=1e-12, rhs_tile=64)
    assert out["rc"] == 0
    inv = [osolve.dense_inverse(u, -0.2, s, dims, -1) for s in s_hat]
    for pi, p in enumerate([0, 1]):
        g = osolve.dense_GammaOmega(u, odirac.gamma_product(["g3"]), p, dims)
        for i in range(2):
            ta = np.trace(g @ inv[i])
            assert np.abs(out["a"][:, pi, i] - ta).max() <= 1e-9 * abs(ta)
            for j in range(i, 2):
                tb = np.trace(inv[i] @ g @ inv[j])
                assert np.abs(out["b"][:, pi, i, j] - tb).max() <= 1e-9 * abs(tb)
    ctx.close()
