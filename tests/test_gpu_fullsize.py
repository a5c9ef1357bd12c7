"""Parity at the benchmark sizes: 16^3x32 (the FS-MLMC job of the benchmark) and
24^3x64 (variance sampling over p = 0..8).

The oracle cannot solve these systems within a test, so it checks what it can
compute one by one: the Z4 noise (bit-exact), the FP64 true residual of GPU
solutions with its own operator, and the Gamma Omega_p contractions of those
solutions against the GPU's level samples and variance samples. The GPU
solution of a system is bit-identical whichever entry point solved it (kernels
are per-system and reductions fixed-order), so shifted_solve exposes the very
vectors that mlmc_level_trace and variance_sample contracted.
"""

import numpy as np
import pytest

import inputs
from oracle import dirac as odirac
from oracle import estimators as oest
from oracle import philox as ophilox
from helpers import rel_resid

pkg = pytest.importorskip("paper_2212_04430_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_config3_16x32_last_level_sample_against_an_oracle_solve():
    """One last-level sample of the 16^3x32 job (sigma_L = 0.6, the cheapest level for the oracle)
    against the contraction of the oracle's own BiCGStab solution on the same noise, at the
    mixed-precision tolerance of the level traces."""
    dims = (16, 16, 16, 32)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1003, eps=0.4)
    ctx = pkg.Context(dims)
    ctx.fs_set_gauge(u)
    sig = [0.005, 0.03, 0.15, 0.6]
    m, p, seed, job = -0.35, 4, 2003, 78
    out = ctx.mlmc_level_trace(m, sig, pkg.gamma_matrix("g3"), p, [1, 1, 1, 1], seed=seed, job=job, prec="f16",
                               tol=1e-8, rhs_tile=32, link_compress=12)
    assert out["rc"] == 0
    ctx.close()
    z = ophilox.z4_noise(v, seed, job, 3, 0)
    solver = oest.make_solver(u, m, dims, -1, tol=1e-10)
    ref = oest.contract(u, z, solver(z, 0.6), odirac.GAMMA[2], p, dims)
    got = out["samples"][3][0]
    assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)


def test_config3_16x32_level_samples_and_residuals():
    dims = (16, 16, 16, 32)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1003, eps=0.4)
    ctx = pkg.Context(dims)
    ctx.fs_set_gauge(u)
    sig = [0.005, 0.03, 0.15, 0.6]
    m, p, seed, job = -0.35, 4, 2003, 77
    kw = dict(prec="f16", tol=1e-8, rhs_tile=32, link_compress=12)
    out = ctx.mlmc_level_trace(m, sig, pkg.gamma_matrix("g3"), p, [2, 2, 2, 2], seed=seed, job=job, estimator="diff",
                               **kw)
    assert out["rc"] == 0
    # sampled noise of the job, bit-exact at full size
    for lev in (0, 3):
        assert np.array_equal(ctx.fs_noise_codes(seed, job, lev, 1), ophilox.z4_codes(v, seed, job, lev, 1))
    # level 0, sample 0 (DIFF): c(s0) - c(s1) on z_{0,0}; level 3, sample 1: c(s3) on z_{1,3}
    cases = [(0, 0, [0.005, 0.03]), (3, 1, [0.6])]
    for lev, s, shifts in cases:
        z = ophilox.z4_noise(v, seed, job, lev, s)
        x, st, rc = ctx.shifted_solve(m, shifts, z, **kw)
        assert rc == 0
        c = []
        for j, sh in enumerate(shifts):
            r = rel_resid(u, x[j, 0], z, m, sh, dims)
            assert r <= 1.05e-8, (lev, sh, r)
            c.append(oest.contract(u, z, x[j, 0], odirac.GAMMA[2], p, dims))
        ref = c[0] - c[1] if len(c) == 2 else c[0]
        got = out["samples"][lev][s]
        assert abs(got - ref) <= 1e-9 * max(abs(ref), 1.0), (lev, got, ref)
    ctx.close()


def test_config5_24x64_variance_samples():
    dims = (24, 24, 24, 64)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1005, eps=0.5)
    ctx = pkg.Context(dims)
    ctx.fs_set_gauge(u)
    s_hat = [0.0, 0.05, 0.25, 0.5, 1.0]
    m, seed, job = -0.38, 2005, 3
    plist = list(range(9))
    kw = dict(prec="f16", tol=1e-8, rhs_tile=10, link_compress=12)
    out = ctx.variance_sample(m, s_hat, pkg.gamma_matrix("g3"), plist, 1, seed=seed, job=job, **kw)
    assert out["rc"] == 0
    assert np.array_equal(ctx.fs_noise_codes(seed, job, ophilox.VARIANCE_SAMPLE_LEVEL, 0),
                          ophilox.z4_codes(v, seed, job, ophilox.VARIANCE_SAMPLE_LEVEL, 0))
    # a_i(p) = z^dag gamma3 Omega_p x^(i) for the largest shift, recomputed by the oracle
    z = ophilox.z4_noise(v, seed, job, ophilox.VARIANCE_SAMPLE_LEVEL, 0)
    x, st, rc = ctx.shifted_solve(m, [1.0], z, **kw)
    assert rc == 0
    assert rel_resid(u, x[0, 0], z, m, 1.0, dims) <= 1.05e-8
    for p in (0, 1, 5, 8):
        ref = oest.contract(u, z, x[0, 0], odirac.GAMMA[2], p, dims)
        got = out["a"][0, p, 4]
        assert abs(got - ref) <= 1e-9 * max(abs(ref), 1.0), (p, got, ref)
    ctx.close()


def test_expansion_exact_part_closed_forms_16x32():
    """The hopping parameter expansion's exact low orders at the benchmark size, against closed
    forms that hold for any gauge field (paths of length k < K from x + p z back to x): p = 1,
    K = 2 gives 3V kappa tr(G (1 + g_z)) / A; p = 3, K = 4 (only the straight path,
    (1 + g_z)^3 = 4 (1 + g_z)) gives 12V kappa^3 tr(G (1 + g_z)) / A; p = 0, K = 4 gives
    3V tr(G) / A; p = 4, K = 4 gives 0 (no path is short enough)."""
    dims = (16, 16, 16, 32)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1003, eps=0.4)
    m, s = -0.35, 0.6
    A = 4.0 + m + s
    kappa = 1.0 / (2.0 * A)
    ctx = pkg.Context(dims, bc_t=-1, device=0)
    ctx.fs_set_gauge(u)
    for name, go in (("g3", odirac.gamma_product(["g3"])), ("g5g3", odirac.gamma_product(["g5", "g3"])),
                     ("1", odirac.IDENT4)):
        g = go if name == "1" else pkg.gamma_matrix(name)
        t1 = np.trace(go @ (odirac.IDENT4 + odirac.GAMMA[2]))
        cases = [(1, 2, 3 * v * kappa * t1 / A), (3, 4, 12 * v * kappa ** 3 * t1 / A),
                 (0, 4, 3 * v * np.trace(go) / A), (4, 4, 0.0)]
        for p, K, ref in cases:
            got = ctx.hpe_exact_trace(m, s, g, p, K, seed=7)
            assert abs(got - ref) <= 1e-11 * max(1.0, abs(3 * v / A)), (name, p, K, got, ref)
    ctx.close()


def test_expansion_remainder_16x32():
    """The last level with the hopping parameter expansion at the benchmark size (sigma_L = 0.6,
    p = 4, K = 4: the exact part is 0, no path of length < 4 reaches back): each GPU sample equals
    z^dag gamma_3 Omega_4 (kappa H)^4 x with the oracle's H applied to the GPU solution x (the same
    system solved through shifted_solve, bit-identical)."""
    from oracle import hpe as ohpe
    dims = (16, 16, 16, 32)
    v = int(np.prod(dims))
    u = inputs.gauge_field(dims, "smooth", seed=1003, eps=0.4)
    m, s = -0.35, 0.6
    kw = dict(prec="f16", tol=1e-8, rhs_tile=2, link_compress=12)
    ctx = pkg.Context(dims)
    ctx.fs_set_gauge(u)
    out = ctx.mlmc_level_trace(m, [s], pkg.gamma_matrix("g3"), 4, [2], seed=2003, job=9, hpe_order=4, **kw)
    assert out["rc"] == 0
    kappa = 1.0 / (2.0 * (4.0 + m + s))
    for smp in range(2):
        z = ophilox.z4_noise(v, 2003, 9, 0, smp)
        x, st, rc = ctx.shifted_solve(m, [s], z, **kw)
        y = x[0, 0]
        for _ in range(4):
            y = kappa * ohpe.apply_H(u, y, dims)
        ref = oest.contract(u, z, y, odirac.GAMMA[2], 4, dims)
        got = out["samples"][0][smp]
        assert abs(got - ref) <= 1e-9 * max(abs(ref), 1.0), (smp, got, ref)
    ctx.close()
