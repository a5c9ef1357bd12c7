"""CUDA path against the FP64 oracle, element by element on identical seeded inputs.

Tolerances (from the arithmetic):
  * Z4 noise codes: bit-exact (integer work).
  * wilson_dslash: FP64 1e-13 (rounding order of 1320 flops); FP32 2e-6
    (~10 ulp of FP32); FP16 storage 4e-3 (half ulp 4.9e-4 on inputs and output,
    links in FP16); BF16 storage 3e-2 (bf16 ulp 3.9e-3).
  * solutions: oracle-computed true relative residual <= tol (1e-10 FP64,
    1e-8 mixed), as the solver's stopping rule.
  * level / variance samples: relative 1e-9 (FP64 solves at 1e-12), 1e-6 (mixed
    solves at 1e-8 ... 1e-10), normalised per level by max(|T|, mean |c|).
"""

import numpy as np
import pytest

import inputs
from oracle import dirac as odirac
from oracle import estimators as oest
from oracle import philox as ophilox
from helpers import oracle_D, rel_err, rel_resid, sample_err

pkg = pytest.importorskip("paper_2212_04430_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def make_ctx(dims, u, bc_t=-1):
    ctx = pkg.Context(dims, bc_t=bc_t, device=0)
    ctx.fs_set_gauge(u)
    return ctx


# ---------------------------------------------------------------- noise
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 8), (8, 8, 8, 8)])
def test_noise_codes_bit_exact(dims):
    v = int(np.prod(dims))
    ctx = pkg.Context(dims)
    for (seed, job, level, sample) in [(0, 0, 0, 0), (2002, 3, 1, 17), (2**40 + 5, 7, 0x80000000, 3),
                                       (2**64 - 1, 2**32 - 1, 2**32 - 1, 2**32 - 1)]:
        got = ctx.fs_noise_codes(seed, job, level, sample)
        ref = ophilox.z4_codes(v, seed, job, level, sample)
        assert np.array_equal(got, ref)
    ctx.close()


# ---------------------------------------------------------------- dslash
DSLASH_TOL = {"f64": 1e-13, "f32": 2e-6, "f16": 4e-3, "bf16": 3e-2}


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("dims,bc_t,nrhs", [((2, 2, 2, 2), -1, 1), ((4, 4, 4, 4), -1, 3),
                                            ((4, 6, 2, 8), 1, 2), ((8, 8, 8, 8), -1, 17),
                                            ((8, 4, 4, 8), -1, 32), ((4, 4, 4, 8), 1, 64),
                                            ((4, 4, 2, 8), -1, 40)])
def test_dslash_parity(prec, dims, bc_t, nrhs):
    u = inputs.gauge_field(dims, "haar", seed=1001)
    psi = inputs.random_spinor(dims, 7, nvec=nrhs)
    ctx = make_ctx(dims, u, bc_t)
    for nr in ((18,) if prec == "f64" else (18, 12)):
        got = ctx.wilson_dslash(-0.4, 0.15, psi, prec=prec, link_compress=nr)
        ref = oracle_D(u, psi, -0.4, 0.15, dims, bc_t)
        assert rel_err(got, ref) < DSLASH_TOL[prec], (prec, nr, rel_err(got, ref))
    ctx.close()


def test_dslash_ragged_tiles_and_empty():
    """nrhs above the 64-system tile (two chunks, ragged tail) and nrhs = 0."""
    dims = (4, 4, 2, 2)
    u = inputs.gauge_field(dims, "smooth", seed=5, eps=0.3)
    psi = inputs.random_spinor(dims, 8, nvec=70)
    ctx = make_ctx(dims, u)
    got = ctx.wilson_dslash(-0.2, 0.0, psi, prec="f64")
    assert rel_err(got, oracle_D(u, psi, -0.2, 0.0, dims)) < 1e-13
    empty = np.zeros((0, int(np.prod(dims)), 4, 3), dtype=complex)
    assert ctx.wilson_dslash(-0.2, 0.0, empty).shape == empty.shape
    ctx.close()


def test_dslash_free_field_plane_wave_16x32():
    """At 16^3x32 (no oracle needed): a plane wave is an eigenvector of the free
    operator in spin space, (D + s) e^{ikx} u = [M(k) + i gamma.sin k] e^{ikx} u."""
    dims = (16, 16, 16, 32)
    u = inputs.unit_gauge(dims)
    ctx = make_ctx(dims, u)
    lx, ly, lz, lt = dims
    n = np.array([3, 1, 5, 2])
    k = 2 * np.pi * n / np.array(dims, dtype=float)
    k[3] = (2 * n[3] + 1) * np.pi / lt  # antiperiodic in t
    s = np.arange(int(np.prod(dims)))
    x = np.stack([s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)])
    phase = np.exp(1j * (k[:, None] * x).sum(0))
    spin = np.array([1.0, 0.5j, -0.25, 0.75 - 0.1j])
    col = np.array([1.0, -1j, 0.3])
    psi = phase[:, None, None] * spin[None, :, None] * col[None, None, :]
    m, sigma = -0.35, 0.03
    dk = (m + sigma + np.sum(1 - np.cos(k))) * np.eye(4) + 1j * sum(
        odirac.GAMMA[mu] * np.sin(k[mu]) for mu in range(4))
    ref = phase[:, None, None] * (dk @ spin)[None, :, None] * col[None, None, :]
    for prec, tol in (("f64", 1e-12), ("f32", 2e-6)):
        got = ctx.wilson_dslash(m, sigma, psi, prec=prec)
        assert rel_err(got, ref) < tol
    ctx.close()


# ---------------------------------------------------------------- solves
@pytest.mark.parametrize("prec,tol,nr", [("f64", 1e-10, 18), ("f32", 1e-8, 18), ("f16", 1e-8, 12),
                                         ("bf16", 1e-8, 18)])
def test_shifted_solve_residual_4444(prec, tol, nr):
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=1000)
    b = inputs.random_spinor(dims, 9, nvec=3)
    sig = [0.0, 0.4]
    ctx = make_ctx(dims, u)
    x, st, rc = ctx.shifted_solve(-0.4, sig, b, prec=prec, tol=tol, rhs_tile=4, link_compress=nr, verify=1)
    assert rc == 0
    for j, s in enumerate(sig):
        for k in range(3):
            r = rel_resid(u, x[j, k], b[k], -0.4, s, dims)
            assert r <= tol * 1.05, (prec, j, k, r)
            stt = st[j * 3 + k]
            assert stt["status"] == 2 and stt["true_resid"] <= tol * 1.05
            assert abs(stt["true_resid"] - r) <= 0.05 * r + 1e-15
    ctx.close()


def test_shifted_solve_matches_dense_2222():
    """Smallest lattice (every direction wraps onto the same neighbour)."""
    from oracle import solve as osolve
    dims = (2, 2, 2, 2)
    u = inputs.gauge_field(dims, "haar", seed=3)
    b = inputs.random_spinor(dims, 4, nvec=2)
    ctx = make_ctx(dims, u)
    x, st, rc = ctx.shifted_solve(-0.3, [0.1], b, prec="f64", tol=1e-12, rhs_tile=1)
    dense = osolve.dense_operator(u, -0.3, 0.1, dims)
    for k in range(2):
        ref = np.linalg.solve(dense, b[k].ravel()).reshape(b[k].shape)
        assert rel_err(x[0, k], ref) < 1e-10
    ctx.close()


def test_shifted_solve_edge_cases():
    dims = (4, 4, 2, 2)
    u = inputs.gauge_field(dims, "smooth", seed=6, eps=0.3)
    ctx = make_ctx(dims, u)
    b = inputs.random_spinor(dims, 10, nvec=2)
    b[1] = 0.0  # zero right-hand side: x = 0, converged at once
    x, st, rc = ctx.shifted_solve(-0.2, [0.05], b, prec="f32")
    assert rc == 0 and np.all(x[0, 1] == 0) and st[1]["status"] == 2
    x, st, rc = ctx.shifted_solve(-0.2, [0.05], b[:1], prec="f64", max_iter=1, tol=1e-12)
    assert rc == pkg.fsmlmc.FS_ERR_NOCONV and st[0]["status"] == 3
    bad = b[:1].copy()
    bad[0, 3, 1, 2] = np.nan
    with pytest.raises(pkg.FsError) as e:
        ctx.shifted_solve(-0.2, [0.05], bad)
    assert e.value.code == pkg.fsmlmc.FS_ERR_INPUT
    ctx.close()
    with pytest.raises(pkg.FsError):
        pkg.Context((4, 3, 4, 4))


# ---------------------------------------------------------------- level traces
def _oracle_levels(u, m, sig, gam, p, n, seed, job, dims, est):
    solver = oest.make_dense_solver(u, m, dims)
    return oest.level_samples(u, m, sig, gam, p, n, seed, job, dims, -1, est, solver)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f16", 1e-6), ("bf16", 1e-6)])
def test_mlmc_config1_samples(prec, tol):
    """4^4 Haar links, m = -0.4, shifts {0, 0.4}, Gamma = I, p = 0, 64 Z4 vectors per level."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=1001)
    sig = [0.0, 0.4]
    n = [64, 64]
    ctx = make_ctx(dims, u)
    solve_tol = 1e-12 if prec == "f64" else 1e-10
    out = ctx.mlmc_level_trace(-0.4, sig, np.eye(4), 0, n, seed=2001, job=0, estimator="diff", prec=prec,
                               tol=solve_tol, rhs_tile=32)
    assert out["rc"] == 0
    ref = _oracle_levels(u, -0.4, sig, odirac.IDENT4, 0, n, 2001, 0, dims, oest.DIFF)
    for lev in range(2):
        assert sample_err(out["samples"][lev], ref[lev]) < tol, lev
        m2 = np.mean(np.abs(ref[lev]) ** 2)
        assert abs(out["var"][lev] - oest.practical_variance(ref[lev])) <= 10 * tol * m2
    ctx.close()


def test_mlmc_config2_samples_against_oracle_bicgstab():
    """Config 2: 8^4 smoothed links (eps = 0.3), m = -0.2, shifts {0.02, 0.1, 0.5}, Gamma =
    gamma5 gamma3, z-displacement p = 2, FP32 storage with FP64 reliable updates, 16-system tiles;
    the level samples against the oracle's own BiCGStab solutions (no dense inverse at this size)
    on the same noise, at the mixed-precision tolerance."""
    dims = (8, 8, 8, 8)
    m, sig, p, seed, job = -0.2, [0.02, 0.1, 0.5], 2, 2002, 0
    u = inputs.gauge_field(dims, "smooth", seed=1002, eps=0.3)
    n = [2, 2, 2]
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(m, sig, pkg.gamma_matrix("g5g3"), p, n, seed=seed, job=job, estimator="diff",
                               prec="f32", tol=1e-10, rhs_tile=16)
    assert out["rc"] == 0
    solver = oest.make_solver(u, m, dims, -1, tol=1e-12)
    ref = oest.level_samples(u, m, sig, odirac.gamma_product(["g5", "g3"]), p, n, seed, job, dims, -1, oest.DIFF,
                             solver)
    for lev in range(3):
        assert sample_err(out["samples"][lev], ref[lev]) < 1e-6, (lev, out["samples"][lev], ref[lev])
    ctx.close()


@pytest.mark.parametrize("est", ["split_even", "product"])
def test_mlmc_estimators_samples(est):
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=11, eps=0.5)
    sig = [0.0, 0.1, 0.5]
    gam = pkg.gamma_matrix("g5g3")
    n = [5, 4, 3]
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.2, sig, gam, 2, n, seed=77, job=5, estimator=est, prec="f64", tol=1e-12,
                               rhs_tile=8)
    ref = _oracle_levels(u, -0.2, sig, odirac.gamma_product(["g5", "g3"]), 2, n, 77, 5, dims,
                         oest.ESTIMATORS[est])
    for lev in range(3):
        assert sample_err(out["samples"][lev], ref[lev]) < 1e-9, (est, lev)
    ctx.close()


def test_mlmc_dense_expectation_config1():
    """Mean of the GPU level samples against the exact dense level traces (5 sigma)."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=1001)
    sig = [0.0, 0.4]
    n = [256, 256]
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.4, sig, np.eye(4), 0, n, seed=2001, job=1, estimator="diff", prec="f32", tol=1e-10)
    mats = oest.exact_level_matrices(u, -0.4, sig, odirac.IDENT4, 0, dims, -1, oest.DIFF)
    for lev in range(2):
        exact = np.trace(mats[lev])
        se = np.sqrt(oest.exact_z4_variance(mats[lev]) / n[lev])
        assert abs(out["trace"][lev] - exact) < 5 * se
    ctx.close()


# ---------------------------------------------------------------- variance sampling
@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-6)])
def test_variance_sample_parity(prec, tol):
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1005, eps=0.5)
    s_hat = [0.0, 0.05, 0.25, 0.5, 1.0]
    plist = [2, 0, 1]
    ns = 3
    ctx = make_ctx(dims, u)
    out = ctx.variance_sample(-0.38, s_hat, pkg.gamma_matrix("g3"), plist, ns, seed=2005, job=0, prec=prec,
                              tol=1e-12 if prec == "f64" else 1e-10)
    solver = oest.make_dense_solver(u, -0.38, dims)
    ref = oest.variance_sample(u, -0.38, s_hat, odirac.GAMMA[2], plist, ns, 2005, 0, dims, -1, solver)
    for pi in range(len(plist)):
        for i in range(5):
            assert sample_err(out["a"][:, pi, i], ref["a"][:, pi, i]) < tol
            for j in range(i, 5):
                assert sample_err(out["b"][:, pi, i, j], ref["b"][:, pi, i, j]) < tol
    m2a = np.mean(np.abs(ref["a"]) ** 2, axis=0)
    m2b = np.mean(np.abs(ref["b"]) ** 2, axis=0)
    assert np.all(np.abs(out["VL"] - ref["VL"]) <= 10 * tol * m2a)
    assert np.all(np.abs(out["Vbar"] - ref["Vbar"]) <= 10 * tol * m2b + 1e-300)
    ctx.close()


# ---------------------------------------------------------------- batching invariance
@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_results_identical_alone_and_in_a_mix(prec):
    """A level sample solved alone (1-system tile) equals the same sample solved inside a
    32-system tile with continuous slot refill: per-system kernels and fixed-order
    reductions make every system independent of its neighbours and its slot."""
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=21, eps=0.4)
    sig = [0.01, 0.1, 0.6]
    g = pkg.gamma_matrix("g3")
    ctx = make_ctx(dims, u)
    kw = dict(prec=prec, tol=1e-10 if prec == "f64" else 1e-8)
    mix = ctx.mlmc_level_trace(-0.3, sig, g, 1, [20, 20, 20], seed=5, job=9, rhs_tile=32, **kw)
    alone = ctx.mlmc_level_trace(-0.3, sig, g, 1, [1, 1, 1], seed=5, job=9, rhs_tile=1, **kw)
    for lev in range(3):
        assert mix["samples"][lev][0] == alone["samples"][lev][0], (lev, mix["samples"][lev][0],
                                                                  alone["samples"][lev][0])
    ctx.close()


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_tile_shapes_give_identical_systems(prec):
    """Every inner-precision hop variant computes a system the same way: a 64-system tile
    (the persistent kernel over two 32-system chunks), a 40-system tile (20 systems per
    warp, the prefetch kernel) and single-system tiles give bit-identical solutions, each
    within tolerance by the oracle's residual."""
    dims = (8, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=33, eps=0.4)
    b = inputs.random_spinor(dims, 41, nvec=40)
    sig = [0.02]
    ctx = make_ctx(dims, u)
    kw = dict(prec=prec, tol=1e-8, link_compress=12)
    x64, st64, rc = ctx.shifted_solve(-0.25, sig, np.concatenate([b, b[:24]]), rhs_tile=64, **kw)
    assert rc == 0
    x40, _, rc = ctx.shifted_solve(-0.25, sig, b, rhs_tile=40, **kw)
    assert rc == 0
    for k in (0, 17, 39):
        x1, _, rc = ctx.shifted_solve(-0.25, sig, b[k:k + 1], rhs_tile=1, **kw)
        assert rc == 0
        assert np.array_equal(x64[0, k], x1[0, 0]) and np.array_equal(x40[0, k], x1[0, 0]), k
        assert rel_resid(u, x1[0, 0], b[k], -0.25, 0.02, dims) <= 1.05e-8
    # the duplicated right-hand sides in the 64-system tile solve identically too
    assert np.array_equal(x64[0, 40:], x64[0, :24])
    ctx.close()


def test_product_chain_and_split_even_in_mixed_tiles():
    """Nested (product) and paired (split-even) systems with refill in a small tile."""
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=13, eps=0.5)
    sig = [0.0, 0.05, 0.3]
    n = [9, 7, 5]
    ctx = make_ctx(dims, u)
    for est in ("product", "split_even"):
        out = ctx.mlmc_level_trace(-0.25, sig, pkg.gamma_matrix("g4"), 1, n, seed=8, job=2, estimator=est,
                                   prec="f64", tol=1e-12, rhs_tile=3)
        ref = _oracle_levels(u, -0.25, sig, odirac.GAMMA[3], 1, n, 8, 2, dims, oest.ESTIMATORS[est])
        for lev in range(3):
            assert sample_err(out["samples"][lev], ref[lev]) < 1e-9, (est, lev)
    ctx.close()


@pytest.mark.parametrize("est", ["diff", "product"])
def test_lanes_give_identical_results(est):
    """Tiles solved at the same time (lanes, each on a stream and host thread of its own,
    sharing the gauge copies and the contraction paths) give exactly the per-sample values,
    traces, variances and per-system iteration counts of a single tile: a system's result
    does not depend on its tile, so lanes change only the schedule."""
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=23, eps=0.4)
    sig = [0.01, 0.1, 0.6]
    g = pkg.gamma_matrix("g3")
    n = [12, 10, 9]
    ctx = make_ctx(dims, u)
    kw = dict(prec="f16", tol=1e-8, rhs_tile=8)
    one = ctx.mlmc_level_trace(-0.3, sig, g, 2, n, seed=6, job=3, estimator=est, lanes=1, **kw)
    assert one["rc"] == 0
    for nl in (2, 3):
        many = ctx.mlmc_level_trace(-0.3, sig, g, 2, n, seed=6, job=3, estimator=est, lanes=nl, **kw)
        assert many["rc"] == 0
        for lev in range(3):
            assert np.array_equal(one["samples"][lev], many["samples"][lev]), (nl, lev)
        assert np.array_equal(one["trace"], many["trace"]) and np.array_equal(one["var"], many["var"])
        assert [s["iters"] for s in one["stats"]] == [s["iters"] for s in many["stats"]]
    ctx.close()


def test_autotuned_tile():
    """rhs_tile = 0 lets the library pick the tile: the autotuner times a BiCGStab iteration per
    system on the candidate tiles once per precision and link format, and the chosen tile gives
    exactly the results of the same call with that tile given explicitly."""
    dims = (4, 4, 4, 8)
    u = inputs.gauge_field(dims, "smooth", seed=29, eps=0.4)
    sig = [0.02, 0.3]
    g = pkg.gamma_matrix("g5")
    n = [10, 12]
    ctx = make_ctx(dims, u)
    assert ctx.tuned_tile("f16", 12) == 0
    kw = dict(prec="f16", tol=1e-8, link_compress=12)
    auto = ctx.mlmc_level_trace(-0.3, sig, g, 1, n, seed=4, job=1, rhs_tile=0, **kw)
    t = ctx.tuned_tile("f16", 12)
    assert t in (8, 16, 32) and auto["rc"] == 0  # 32 solves: the 64-system tile is not a candidate
    fixed = ctx.mlmc_level_trace(-0.3, sig, g, 1, n, seed=4, job=1, rhs_tile=t, lanes=1, **kw)
    for lev in range(2):
        assert np.array_equal(auto["samples"][lev], fixed["samples"][lev]), lev
    # measured once: a second call keeps the choice
    ctx.mlmc_level_trace(-0.3, sig, g, 1, n, seed=4, job=2, rhs_tile=0, **kw)
    assert ctx.tuned_tile("f16", 12) == t
    ctx.close()


def test_autotuned_launch_shape_changes_no_result():
    """On tiles of 32-system chunks the autotuner also picks the persistent hop's ring depth and
    resident blocks per SM (one of four shapes); a fresh context at the same tile, in the default
    shape, gives bit-identical samples."""
    dims = (8, 8, 8, 8)
    u = inputs.gauge_field(dims, "smooth", seed=31, eps=0.3)
    sig = [0.05, 0.4]
    g = pkg.gamma_matrix("g3")
    n = [48, 48]
    kw = dict(prec="f16", tol=1e-8, link_compress=12)
    ctx = make_ctx(dims, u)
    auto = ctx.mlmc_level_trace(-0.2, sig, g, 1, n, seed=6, job=3, rhs_tile=0, **kw)
    assert auto["rc"] == 0
    t, depth, blocks = ctx.tuned_shape("f16", 12)
    assert t in (8, 16, 32, 64)
    if t % 32 == 0:
        assert depth in (0, 3) and blocks in (0, 2), (depth, blocks)
    else:
        assert depth == 0 and blocks == 0
    ctx.close()
    fresh = make_ctx(dims, u)
    fixed = fresh.mlmc_level_trace(-0.2, sig, g, 1, n, seed=6, job=3, rhs_tile=t, lanes=1, **kw)
    for lev in range(2):
        assert np.array_equal(auto["samples"][lev], fixed["samples"][lev]), lev
    fresh.close()


def test_new_gauge_field_rebuilds_the_contraction_paths():
    """The straight z-paths W(x, x + p z) are cached per gauge field: after fs_set_gauge with a
    new field, a contraction at p > 0 equals the one of a fresh context holding that field."""
    dims = (4, 4, 4, 8)
    u1 = inputs.gauge_field(dims, "smooth", seed=51, eps=0.4)
    u2 = inputs.gauge_field(dims, "smooth", seed=52, eps=0.4)
    sig = [0.05, 0.5]
    g = pkg.gamma_matrix("g3")
    kw = dict(prec="f64", tol=1e-10, rhs_tile=4)
    ctx = make_ctx(dims, u1)
    ctx.mlmc_level_trace(-0.3, sig, g, 3, [3, 3], seed=9, job=1, **kw)
    ctx.fs_set_gauge(u2)
    again = ctx.mlmc_level_trace(-0.3, sig, g, 3, [3, 3], seed=9, job=1, **kw)
    ctx.close()
    fresh_ctx = make_ctx(dims, u2)
    fresh = fresh_ctx.mlmc_level_trace(-0.3, sig, g, 3, [3, 3], seed=9, job=1, **kw)
    fresh_ctx.close()
    for lev in range(2):
        assert np.array_equal(again["samples"][lev], fresh["samples"][lev]), lev


def test_contraction_with_a_dense_gamma():
    """A Gamma that is not a Clifford product (dense complex 4x4) takes the general path of
    the contraction; Clifford products take the permutation path (the tests above)."""
    dims = (4, 4, 2, 4)
    u = inputs.gauge_field(dims, "haar", seed=31)
    rng = np.random.default_rng(8)
    gam = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    sig = [0.05, 0.4]
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.3, sig, gam, 1, [4, 3], seed=12, job=4, estimator="split_even", prec="f64",
                               tol=1e-12, rhs_tile=4)
    ref = _oracle_levels(u, -0.3, sig, gam, 1, [4, 3], 12, 4, dims, oest.SPLIT_EVEN)
    for lev in range(2):
        assert sample_err(out["samples"][lev], ref[lev]) < 1e-9, lev
    ctx.close()


def test_shifted_solve_on_device_arrays():
    """shifted_solve_dev on torch device tensors gives the host call's solutions exactly (the same
    arithmetic), and refuses host memory."""
    torch = pytest.importorskip("torch")
    dims = (4, 4, 4, 8)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=31, eps=0.4)
    rng = np.random.default_rng(5)
    b = (rng.normal(size=(3, v, 4, 3)) + 1j * rng.normal(size=(3, v, 4, 3)))
    sig = [0.02, 0.3]
    ctx = make_ctx(dims, u)
    kw = dict(prec="f16", tol=1e-9, rhs_tile=4, link_compress=12)
    x_host, st_host, _ = ctx.shifted_solve(-0.3, sig, b, **kw)
    bd = torch.from_numpy(np.ascontiguousarray(b).view(np.float64).reshape(3, v, 24)).to("cuda:0")
    xd = torch.zeros((2, 3, v, 24), dtype=torch.float64, device="cuda:0")
    torch.cuda.synchronize()
    st = ctx.shifted_solve_dev(-0.3, sig, bd.data_ptr(), 3, xd.data_ptr(), **kw)
    x = xd.cpu().numpy().view(np.complex128).reshape(2, 3, v, 4, 3)
    assert np.array_equal(x, np.asarray(x_host).reshape(x.shape))
    assert [s["iters"] for s in st] == [s["iters"] for s in st_host]
    hb = np.zeros((3, v, 24))
    with pytest.raises(pkg.FsError) as e:
        ctx.shifted_solve_dev(-0.3, sig, hb.ctypes.data, 3, xd.data_ptr(), **kw)
    assert e.value.code == pkg.fsmlmc.FS_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("hpe_order", [0, 4])
def test_several_displacements_from_one_set_of_solves(hpe_order):
    """mlmc_level_traces: the traces for p = 3, 0, 1 from the same solves equal three
    single-displacement calls exactly (each displacement is its own sum in the one contraction
    pass), in the caller's order; with the expansion each p has its own exact part."""
    dims = (4, 4, 8, 4)
    u = inputs.gauge_field(dims, "smooth", seed=33, eps=0.4)
    sig = [0.02, 0.2, 0.7]
    n = [3, 2, 4]
    g = pkg.gamma_matrix("g3")
    ctx = make_ctx(dims, u)
    kw = dict(seed=12, job=1, estimator="split_even", prec="f32", tol=1e-9, rhs_tile=8, hpe_order=hpe_order)
    many = ctx.mlmc_level_trace(-0.2, sig, g, [3, 0, 1], n, **kw)
    assert [r["p"] for r in many] == [3, 0, 1]
    for r in many:
        one = ctx.mlmc_level_trace(-0.2, sig, g, r["p"], n, **kw)
        for lev in range(3):
            assert np.array_equal(r["samples"][lev], one["samples"][lev]), (r["p"], lev)
        assert np.array_equal(r["var"], one["var"])
    with pytest.raises(pkg.FsError):
        ctx.mlmc_level_trace(-0.2, sig, g, [1, 1], n, **kw)
    ctx.close()
