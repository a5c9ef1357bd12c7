"""The Wilson-clover operator on the GPU (fs_set_clover) against the FP64 oracle's clover term.

Sec. 4 computes with the clover discretisation; the oracle's reading of the term (oracle/clover.py,
pinned by tests/test_oracle_clover.py) is C(x) = (c_sw / 2) sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x).

Tolerances (from the arithmetic):
  * wilson_dslash with the clover term: the Wilson tolerances (FP64 1e-13, FP32 2e-6, FP16 4e-3,
    BF16 3e-2); the FP64 table comes from a Jacobi eigen-decomposition converged to 1e-15 of the
    block's norm, the FP32 table adds FP32 rounding (~1e-7), both far inside these bounds.
  * solutions: the oracle's true relative residual of D_sw <= tol, as the solver's stopping rule;
    dense LU at 1e-10 for FP64 solves at 1e-12.
  * level samples: relative 1e-9 (FP64 solves at 1e-12), 1e-6 (mixed solves at 1e-10).
"""

import numpy as np
import pytest

import inputs
from oracle import clover as oclover
from oracle import dirac as odirac
from oracle import estimators as oest
from oracle import solve as osolve
from helpers import lattice_u, rel_err, sample_err

pkg = pytest.importorskip("paper_2212_04430_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def cterm_of(u, dims, c_sw):
    return oclover.clover_term(lattice_u(u, dims), c_sw)


def oracle_Dsw(u, psi, m, sigma, dims, cterm, bc_t=-1):
    """(D_sw + sigma) psi with the oracle, canonical flat in/out [..., V, 4, 3]."""
    shp = odirac.lattice_shape(dims)
    lead = psi.shape[:-3]
    out = oclover.apply_Dsw(lattice_u(u, dims), psi.reshape(lead + shp + (4, 3)), m, sigma, bc_t, cterm)
    return out.reshape(psi.shape)


def rel_resid_sw(u, x, b, m, sigma, dims, cterm, bc_t=-1):
    r = b - oracle_Dsw(u, x, m, sigma, dims, cterm, bc_t)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel()))


def make_ctx(dims, u, c_sw, bc_t=-1):
    ctx = pkg.Context(dims, bc_t=bc_t, device=0)
    ctx.fs_set_gauge(u)
    ctx.fs_set_clover(c_sw)
    return ctx


DSLASH_TOL = {"f64": 1e-13, "f32": 2e-6, "f16": 4e-3, "bf16": 3e-2}


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("dims,bc_t,nrhs,kind", [((2, 2, 2, 2), -1, 1, "haar"), ((4, 4, 4, 4), -1, 3, "haar"),
                                                 ((4, 6, 2, 8), 1, 2, "smooth"), ((8, 4, 4, 8), -1, 32, "haar"),
                                                 ((4, 4, 2, 8), -1, 40, "smooth")])
def test_dslash_clover_parity(prec, dims, bc_t, nrhs, kind):
    u = inputs.gauge_field(dims, kind, seed=1201, eps=0.5)
    psi = inputs.random_spinor(dims, 17, nvec=nrhs)
    c_sw = 1.3
    ctx = make_ctx(dims, u, c_sw, bc_t)
    ref = oracle_Dsw(u, psi, -0.4, 0.15, dims, cterm_of(u, dims, c_sw), bc_t)
    # the clover term is a visible part of the result
    assert rel_err(oracle_Dsw(u, psi, -0.4, 0.15, dims, cterm_of(u, dims, 0.0), bc_t), ref) > 1e-2
    for nr in ((18,) if prec == "f64" else (18, 12)):
        got = ctx.wilson_dslash(-0.4, 0.15, psi, prec=prec, link_compress=nr)
        assert rel_err(got, ref) < DSLASH_TOL[prec], (prec, nr, rel_err(got, ref))
    ctx.close()


@pytest.mark.parametrize("plane", [(0, 1), (2, 3)])
def test_dslash_clover_constant_abelian_field(plane):
    """Degenerate blocks: on a constant abelian field every site's clover block has two eigenvalues,
    each three times (the colour identity), and the free field has C = 0 (the table's eigenvalues
    are all zero)."""
    dims = (4, 6, 4, 4)
    u, _ = inputs.abelian_field(dims, n=1, mu=plane[0], nu=plane[1])
    psi = inputs.random_spinor(dims, 18, nvec=4)
    ctx = make_ctx(dims, u, 1.7)
    got = ctx.wilson_dslash(-0.3, 0.0, psi, prec="f64")
    assert rel_err(got, oracle_Dsw(u, psi, -0.3, 0.0, dims, cterm_of(u, dims, 1.7))) < 1e-13
    ctx.fs_set_gauge(inputs.unit_gauge(dims))
    got = ctx.wilson_dslash(-0.3, 0.0, psi, prec="f64")
    from helpers import oracle_D
    assert rel_err(got, oracle_D(inputs.unit_gauge(dims), psi, -0.3, 0.0, dims)) < 1e-13
    ctx.close()


def test_clover_switching_and_new_gauge_field():
    """c_sw = 0 restores the Wilson operator bit for bit; a clover term set before the gauge field
    is built with it; a new gauge field rebuilds the table."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=1202)
    u2 = inputs.gauge_field(dims, "smooth", seed=1203, eps=0.6)
    psi = inputs.random_spinor(dims, 19, nvec=2)
    plain = pkg.Context(dims)
    plain.fs_set_gauge(u)
    wilson = plain.wilson_dslash(-0.2, 0.1, psi, prec="f32")
    ctx = pkg.Context(dims)
    ctx.fs_set_clover(0.9)  # before the gauge field
    ctx.fs_set_gauge(u)
    got = ctx.wilson_dslash(-0.2, 0.1, psi, prec="f64")
    assert rel_err(got, oracle_Dsw(u, psi, -0.2, 0.1, dims, cterm_of(u, dims, 0.9))) < 1e-13
    ctx.fs_set_gauge(u2)
    got = ctx.wilson_dslash(-0.2, 0.1, psi, prec="f64")
    assert rel_err(got, oracle_Dsw(u2, psi, -0.2, 0.1, dims, cterm_of(u2, dims, 0.9))) < 1e-13
    ctx.fs_set_gauge(u)
    ctx.fs_set_clover(0.0)
    assert np.array_equal(ctx.wilson_dslash(-0.2, 0.1, psi, prec="f32"), wilson)
    with pytest.raises(pkg.FsError) as e:
        ctx.fs_set_clover(float("nan"))
    assert e.value.code == pkg.fsmlmc.FS_ERR_INPUT
    ctx.close()
    plain.close()


@pytest.mark.parametrize("prec,tol,nr", [("f64", 1e-10, 18), ("f32", 1e-8, 18), ("f16", 1e-8, 12),
                                         ("bf16", 1e-8, 18)])
def test_shifted_solve_clover_residual(prec, tol, nr):
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=1204, eps=0.5)
    b = inputs.random_spinor(dims, 20, nvec=3)
    sig = [0.0, 0.3]
    c_sw = 1.1
    cterm = cterm_of(u, dims, c_sw)
    ctx = make_ctx(dims, u, c_sw)
    x, st, rc = ctx.shifted_solve(-0.3, sig, b, prec=prec, tol=tol, rhs_tile=6, link_compress=nr, verify=1)
    assert rc == 0
    for j, s in enumerate(sig):
        for k in range(3):
            r = rel_resid_sw(u, x[j, k], b[k], -0.3, s, dims, cterm)
            assert r <= tol * 1.05, (prec, j, k, r)
            stt = st[j * 3 + k]
            assert stt["status"] == 2 and abs(stt["true_resid"] - r) <= 0.05 * r + 1e-15
    ctx.close()


def test_shifted_solve_clover_matches_dense():
    dims = (2, 2, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1205, eps=0.6)
    b = inputs.random_spinor(dims, 21, nvec=2)
    cterm = cterm_of(u, dims, 1.0)
    ctx = make_ctx(dims, u, 1.0)
    x, st, rc = ctx.shifted_solve(-0.25, [0.05], b, prec="f64", tol=1e-12, rhs_tile=2)
    assert rc == 0
    dense = osolve.dense_operator(u, -0.25, 0.05, dims, -1, cterm)
    for k in range(2):
        ref = np.linalg.solve(dense, b[k].ravel()).reshape(b[k].shape)
        assert rel_err(x[0, k], ref) < 1e-10
    ctx.close()


@pytest.mark.parametrize("prec,tol,est", [("f64", 1e-9, "split_even"), ("f64", 1e-9, "diff"),
                                          ("f16", 1e-6, "split_even")])
def test_mlmc_clover_samples_against_dense(prec, tol, est):
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1206, eps=0.5)
    c_sw, m, sig, p = 1.2, -0.25, [0.0, 0.1, 0.5], 1
    cterm = cterm_of(u, dims, c_sw)
    gam = pkg.gamma_matrix("g5g3")
    n = [4, 3, 3]
    ctx = make_ctx(dims, u, c_sw)
    out = ctx.mlmc_level_trace(m, sig, gam, p, n, seed=91, job=2, estimator=est, prec=prec,
                               tol=1e-12 if prec == "f64" else 1e-10, rhs_tile=8)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, m, dims, -1, cterm)
    ref = oest.level_samples(u, m, sig, odirac.gamma_product(["g5", "g3"]), p, n, 91, 2, dims, -1,
                             oest.ESTIMATORS[est], solver)
    for lev in range(3):
        assert sample_err(out["samples"][lev], ref[lev]) < tol, (est, lev)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f16", 1e-6)])
def test_variance_sample_clover_against_dense(prec, tol):
    """Sec. 3.1's sampling (a_i, b_ij and the sampled variances) with the clover term: the adjoint
    solves use gamma_5-hermiticity, which D_sw keeps."""
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1209, eps=0.5)
    c_sw, m = 1.1, -0.3
    s_hat = [0.0, 0.1, 0.4]
    plist = [1, 0]
    ns = 3
    ctx = make_ctx(dims, u, c_sw)
    out = ctx.variance_sample(m, s_hat, pkg.gamma_matrix("g3"), plist, ns, seed=2006, job=1, prec=prec,
                              tol=1e-12 if prec == "f64" else 1e-10)
    solver = oest.make_dense_solver(u, m, dims, -1, cterm_of(u, dims, c_sw))
    ref = oest.variance_sample(u, m, s_hat, odirac.GAMMA[2], plist, ns, 2006, 1, dims, -1, solver)
    for pi in range(len(plist)):
        for i in range(len(s_hat)):
            assert sample_err(out["a"][:, pi, i], ref["a"][:, pi, i]) < tol
            for j in range(i, len(s_hat)):
                assert sample_err(out["b"][:, pi, i, j], ref["b"][:, pi, i, j]) < tol
    ctx.close()


def test_clover_tile_shapes_give_identical_systems():
    """The clover passes and the clover M-hat compute a system the same way in every tile shape:
    64-, 40- and 1-system tiles give bit-identical FP16 solutions."""
    dims = (8, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=1207, eps=0.4)
    b = inputs.random_spinor(dims, 22, nvec=40)
    ctx = make_ctx(dims, u, 1.0)
    kw = dict(prec="f16", tol=1e-8, link_compress=12)
    x64, _, rc = ctx.shifted_solve(-0.25, [0.02], np.concatenate([b, b[:24]]), rhs_tile=64, **kw)
    assert rc == 0
    x40, _, rc = ctx.shifted_solve(-0.25, [0.02], b, rhs_tile=40, **kw)
    assert rc == 0
    cterm = cterm_of(u, dims, 1.0)
    for k in (0, 23, 39):
        x1, _, rc = ctx.shifted_solve(-0.25, [0.02], b[k:k + 1], rhs_tile=1, **kw)
        assert rc == 0
        assert np.array_equal(x64[0, k], x1[0, 0]) and np.array_equal(x40[0, k], x1[0, 0]), k
        assert rel_resid_sw(u, x1[0, 0], b[k], -0.25, 0.02, dims, cterm) <= 1.05e-8
    ctx.close()


@pytest.mark.parametrize("p,K", [(0, 4), (1, 3), (0, 1)])
def test_last_level_with_the_generalised_expansion(p, K):
    """Sec. 3.1's expansion for the clover action: the last level's samples are T_exact +
    z^dag G Om K^K (D_sw + s)^-1 z, K = A(x)^-1 H / 2, against the oracle's own probing and dense
    solves."""
    from oracle import hpe as ohpe
    from oracle import philox as ophilox
    from oracle import probing as opr
    dims = (4, 4, 4, 4)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1210, eps=0.5)
    c_sw, m, sig = 1.0, -0.2, [0.05, 0.6]
    ct = cterm_of(u, dims, c_sw)
    n = [2, 4]
    ctx = make_ctx(dims, u, c_sw)
    out = ctx.mlmc_level_trace(m, sig, pkg.gamma_matrix("g3"), p, n, seed=22, job=1, hpe_order=K, estimator="diff",
                               prec="f64", tol=1e-12, rhs_tile=16)
    assert out["rc"] == 0
    go = odirac.gamma_product(["g3"])
    col, nc = opr.greedy_coloring(dims, K - 1, p)
    t_exact = ohpe.exact_part_probed(u, m, sig[1], go, p, K, dims, col, nc, cterm=ct)
    solver = oest.make_dense_solver(u, m, dims, -1, ct)
    ref = np.array([t_exact + ohpe.stochastic_part(u, solver, ophilox.z4_noise(v, 22, 1, 1, s), m, sig[1], go, p, K,
                                                   dims, cterm=ct) for s in range(n[1])])
    assert sample_err(out["samples"][1], ref) < 1e-9, (out["samples"][1], ref)
    # the exact part alone, through its own entry point
    got = ctx.hpe_exact_trace(m, sig[1], pkg.gamma_matrix("g3"), p, K)
    ctx.close()
    assert abs(got - t_exact) <= 1e-9 * max(1.0, abs(t_exact)), (got, t_exact)


def test_generalised_expansion_reduces_the_last_level_variance():
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=1211, eps=0.4)
    m, sig = -0.2, [0.8]
    g = pkg.gamma_matrix("g3")
    ctx = make_ctx(dims, u, 1.0)
    kw = dict(prec="f32", tol=1e-9, rhs_tile=64)
    plain = ctx.mlmc_level_trace(m, sig, g, 1, [128], seed=31, **kw)
    hpe = ctx.mlmc_level_trace(m, sig, g, 1, [128], seed=31, hpe_order=4, **kw)
    ctx.close()
    assert plain["rc"] == 0 and hpe["rc"] == 0
    assert hpe["var"][0] < 0.5 * plain["var"][0]
    se = np.sqrt(plain["var"][0] / 128 + hpe["var"][0] / 128)
    assert abs(hpe["trace"][0] - plain["trace"][0]) < 5 * se


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_cgnr_fallback_with_the_clover_term(prec):
    """BiCGStab cut short (max_iter = 2, from the host) hands every system to the FP64 CGNR
    fallback on the clover M-hat; the solutions meet tol by the oracle's D_sw residual and agree
    with dense LU."""
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1212, eps=0.5)
    b = inputs.random_spinor(dims, 25, nvec=2)
    sig, tol, c_sw, m = [0.0, 0.4], 1e-10, 1.0, -0.3
    ct = cterm_of(u, dims, c_sw)
    ctx = make_ctx(dims, u, c_sw)
    x, st, rc = ctx.shifted_solve(m, sig, b, prec=prec, tol=tol, max_iter=2, fallback_iter=20000, rhs_tile=4,
                                  verify=1)
    ctx.close()
    assert rc == 0
    for j, s in enumerate(sig):
        dense = osolve.dense_operator(u, m, s, dims, -1, ct)
        for k in range(2):
            stt = st[j * 2 + k]
            assert stt["status"] == 2 and stt["fallback_iters"] > 0, stt
            assert rel_resid_sw(u, x[j, k], b[k], m, s, dims, ct) <= tol * 1.05
            ref = np.linalg.solve(dense, b[k].ravel()).reshape(b[k].shape)
            assert rel_err(x[j, k], ref) < 1e-7


def test_server_runs_clover_and_wilson_jobs_as_a_context_does():
    """Jobs with and without the clover term on one worker (same lattice and field, so the field
    stays resident while the coefficient changes, then a new field): each result is bit-identical
    to the same call on a context of its own."""
    dims = (4, 4, 4, 4)
    u1 = inputs.gauge_field(dims, "smooth", seed=1213, eps=0.4)
    u2 = inputs.gauge_field(dims, "smooth", seed=1214, eps=0.4)
    m, sig, p, n = -0.2, [0.05, 0.5], 1, [3, 3]
    g = pkg.gamma_matrix("g3")
    kw = dict(prec="f32", tol=1e-10, rhs_tile=8)
    jobs = [(u1, 0.0), (u1, 1.0), (u1, 1.4), (u2, 1.4), (u2, 0.0)]
    srv = pkg.Server(device=0, hbm_budget_bytes=8 << 30, max_active=1)
    tickets = [srv.submit(dims, u, m, sig, g, p, n, 40 + i, job=i, c_sw=c, **kw) for i, (u, c) in enumerate(jobs)]
    res = [srv.poll(t) for t in tickets]
    srv.close()
    for i, (u, c) in enumerate(jobs):
        ctx = make_ctx(dims, u, c)
        ref = ctx.mlmc_level_trace(m, sig, g, p, n, seed=40 + i, job=i, lanes=1, **kw)
        ctx.close()
        assert res[i]["status"] == 0 and np.array_equal(res[i]["trace"], ref["trace"]), i


def test_clover_with_the_papers_noise_lanes_and_displacements():
    """The clover term composes with every other part of the path: probed, fully diluted noise and
    the generalised expansion (the paper's set-up) give bit-identical samples on one and two lanes,
    equal to the oracle's; several displacements from one set of solves equal single-displacement
    calls exactly."""
    from oracle import hpe as ohpe
    from oracle import probing as opr
    dims = (4, 4, 4, 4)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1215, eps=0.4)
    c_sw, m, sig, p, K = 1.0, -0.1, [0.1, 0.5], 1, 3
    ct = cterm_of(u, dims, c_sw)
    n = [2, 2]
    g = pkg.gamma_matrix("g3")
    col, nc = opr.greedy_coloring(dims, 1, 1)
    ctx = make_ctx(dims, u, c_sw)
    kw = dict(colors=col, ncolors=nc, dilute=True, hpe_order=K, prec="f64", tol=1e-12, rhs_tile=32, estimator="diff")
    one = ctx.mlmc_level_trace(m, sig, g, p, n, seed=9, job=3, lanes=1, **kw)
    two = ctx.mlmc_level_trace(m, sig, g, p, n, seed=9, job=3, lanes=2, **kw)
    assert one["rc"] == 0 and two["rc"] == 0
    for lev in range(2):
        assert np.array_equal(one["samples"][lev], two["samples"][lev]), lev
    go = odirac.gamma_product(["g3"])
    solver = oest.make_dense_solver(u, m, dims, -1, ct)
    ecol, enc = opr.greedy_coloring(dims, K - 1, p)
    t_exact = ohpe.exact_part_probed(u, m, sig[1], go, p, K, dims, ecol, enc, cterm=ct)
    ref = []
    for s in range(n[1]):
        tot = t_exact
        for (j, a) in opr.pieces(nc, True):
            z = opr.probed_noise(v, 9, 3, 1, s, col, j, a)
            tot += ohpe.stochastic_part(u, solver, z, m, sig[1], go, p, K, dims, cterm=ct)
        ref.append(tot)
    assert sample_err(one["samples"][1], np.array(ref)) < 1e-9
    # several displacements from one set of solves (plain noise, mixed precision)
    kw2 = dict(seed=12, job=1, estimator="split_even", prec="f32", tol=1e-9, rhs_tile=8)
    many = ctx.mlmc_level_trace(m, sig, g, [2, 0, 1], [3, 3], **kw2)
    for r in many:
        single = ctx.mlmc_level_trace(m, sig, g, r["p"], [3, 3], **kw2)
        for lev in range(2):
            assert np.array_equal(r["samples"][lev], single["samples"][lev]), (r["p"], lev)
    ctx.close()


def test_clover_call_with_more_shifts_than_the_kept_inverses():
    """34 shifts in one call on 32-system tiles (the paired passes): every shift gets its packed
    inverse, so every solution meets tol by the oracle's D_sw residual."""
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1216, eps=0.4)
    b = inputs.random_spinor(dims, 26, nvec=1)
    sig = list(np.linspace(0.0, 0.99, 34))
    ct = cterm_of(u, dims, 1.0)
    ctx = make_ctx(dims, u, 1.0)
    x, st, rc = ctx.shifted_solve(-0.2, sig, b, prec="f16", tol=1e-8, rhs_tile=32, link_compress=12)
    ctx.close()
    assert rc == 0
    for j, s in enumerate(sig):
        assert rel_resid_sw(u, x[j, 0], b[0], -0.2, s, dims, ct) <= 1.05e-8, (j, s)


def test_clover_16x32_dslash_and_solves_at_the_bench_precision():
    """The bench lattice, links and precision with the clover term: the FP16 dslash (12-real links,
    16-system tile, the paired clover pass) against the oracle's D_sw on sampled vectors, and solves
    at the bench's smallest and largest shift certified by the oracle's own D_sw residual."""
    dims = (16, 16, 16, 32)
    u = inputs.gauge_field(dims, "smooth", seed=1003, eps=0.4)
    c_sw = 1.0
    cterm = cterm_of(u, dims, c_sw)
    ctx = make_ctx(dims, u, c_sw)
    psi = inputs.random_spinor(dims, 23, nvec=16)
    got = ctx.wilson_dslash(-0.35, 0.03, psi, prec="f16", link_compress=12)
    for k in (0, 7, 15):
        ref = oracle_Dsw(u, psi[k], -0.35, 0.03, dims, cterm)
        assert rel_err(got[k], ref) < DSLASH_TOL["f16"], (k, rel_err(got[k], ref))
    del got, psi
    b = inputs.random_spinor(dims, 24, nvec=2)
    sig = [0.005, 0.6]
    x, st, rc = ctx.shifted_solve(-0.35, sig, b, prec="f16", tol=1e-8, rhs_tile=4, link_compress=12)
    assert rc == 0
    for j, s in enumerate(sig):
        for k in range(2):
            r = rel_resid_sw(u, x[j, k], b[k], -0.35, s, dims, cterm)
            assert r <= 1.05e-8, (s, k, r)
            assert st[j * 2 + k]["status"] == 2
    ctx.close()


def test_clover_16x32_last_level_sample_against_an_oracle_solve():
    """One last-level sample of the 16^3x32 job with the clover term (sigma_L = 0.6, the cheapest level
    for the oracle) against the contraction of the oracle's own D_sw BiCGStab solution on the same
    noise, at the mixed-precision tolerance of the level traces."""
    from oracle import philox as ophilox
    dims = (16, 16, 16, 32)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1003, eps=0.4)
    c_sw = 1.0
    ctx = make_ctx(dims, u, c_sw)
    sig = [0.005, 0.03, 0.15, 0.6]
    m, p, seed, job = -0.35, 4, 2003, 79
    out = ctx.mlmc_level_trace(m, sig, pkg.gamma_matrix("g3"), p, [1, 1, 1, 1], seed=seed, job=job, prec="f16",
                               tol=1e-8, rhs_tile=32, link_compress=12, estimator="diff")
    ctx.close()
    assert out["rc"] == 0
    z = ophilox.z4_noise(v, seed, job, 3, 0)
    solver = oest.make_solver(u, m, dims, -1, tol=1e-10, cterm=cterm_of(u, dims, c_sw))
    ref = oest.contract(u, z, solver(z, 0.6), odirac.GAMMA[2], p, dims)
    got = out["samples"][3][0]
    assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)
