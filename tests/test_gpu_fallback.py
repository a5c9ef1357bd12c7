"""CGNR fallback: systems BiCGStab leaves unconverged are re-solved by FP64 CG on the
normal equations M^dag M x = M^dag b (M^dag = gamma5 M gamma5).

The fallback is triggered from the host by cutting BiCGStab short (max_iter = 2):
no GPU fault or device-side injection is involved. Its solutions are checked like
every other solve: the oracle's true residual <= tol, and agreement with the dense
solve; level samples against the oracle's.
"""

import numpy as np
import pytest

import inputs
from oracle import dirac as odirac
from oracle import estimators as oest
from oracle import solve as osolve
from helpers import rel_err, rel_resid, sample_err

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


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_fallback_solves_what_bicgstab_did_not(prec):
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=1000)
    b = inputs.random_spinor(dims, 19, nvec=3)
    sig = [0.0, 0.4]
    tol = 1e-10
    ctx = make_ctx(dims, u)
    x, st, rc = ctx.shifted_solve(-0.4, sig, b, prec=prec, tol=tol, max_iter=2, fallback_iter=20000, rhs_tile=4,
                                  verify=1)
    assert rc == 0
    for j, s in enumerate(sig):
        dense = osolve.dense_operator(u, -0.4, s, dims)
        for k in range(3):
            stt = st[j * 3 + k]
            assert stt["status"] == 2 and stt["fallback_iters"] > 0, stt
            assert rel_resid(u, x[j, k], b[k], -0.4, s, dims) <= tol * 1.05
            ref = np.linalg.solve(dense, b[k].ravel()).reshape(b[k].shape)
            assert rel_err(x[j, k], ref) < 1e-7
    ctx.close()


def test_fallback_off_reports_noconv():
    dims = (4, 4, 2, 2)
    u = inputs.gauge_field(dims, "smooth", seed=6, eps=0.3)
    b = inputs.random_spinor(dims, 10, nvec=1)
    ctx = make_ctx(dims, u)
    x, st, rc = ctx.shifted_solve(-0.2, [0.05], b, prec="f32", tol=1e-10, max_iter=2, fallback_iter=-1)
    assert rc == pkg.fsmlmc.FS_ERR_NOCONV
    assert st[0]["status"] == 3 and st[0]["fallback_iters"] == 0
    # a fallback budget too small to converge also ends FS_SYS_NOCONV, after exactly that budget
    x, st, rc = ctx.shifted_solve(-0.2, [0.05], b, prec="f32", tol=1e-10, max_iter=2, fallback_iter=3)
    assert rc == pkg.fsmlmc.FS_ERR_NOCONV
    assert st[0]["status"] == 3 and st[0]["fallback_iters"] == 3
    ctx.close()


@pytest.mark.parametrize("est", ["diff", "product"])
def test_fallback_inside_level_traces(est):
    """Every system of the job goes through the fallback (both phases of the product
    estimator's nested solves); the samples still match the oracle's."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "smooth", seed=1011, eps=0.3)
    sig = [0.05, 0.3]
    n = [6, 6]
    gam = pkg.gamma_matrix("g3")
    ctx = make_ctx(dims, u)
    out = ctx.mlmc_level_trace(-0.3, sig, gam, 1, n, seed=77, job=2, estimator=est, prec="f16", tol=1e-11,
                               max_iter=2, fallback_iter=20000, rhs_tile=8)
    assert out["rc"] == 0
    solver = oest.make_dense_solver(u, -0.3, dims)
    e = {"diff": oest.DIFF, "product": oest.PRODUCT}[est]
    ref = oest.level_samples(u, -0.3, sig, odirac.GAMMA[2], 1, n, 77, 2, dims, -1, e, solver)
    for lev in range(2):
        assert sample_err(out["samples"][lev], ref[lev]) < 1e-7, lev
    ctx.close()


def test_iteration_bound_runs_out_with_timeout_and_the_context_recovers():
    """The host solve loops' watchdog (fs_set_iteration_bound), made to run out on the host: a
    bound of 8 BiCGStab iterations is far below what a 1e-10 solve needs, so the call returns
    FS_ERR_TIMEOUT with its message; no GPU fault or device-side injection is involved. The
    context stays usable: with the built-in bound restored the same solve, and a level trace on
    several lanes, reach their tolerance (the oracle's residual)."""
    dims = (4, 4, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=1000)
    b = inputs.random_spinor(dims, 23, nvec=6)
    ctx = make_ctx(dims, u)
    kw = dict(prec="f16", tol=1e-10, rhs_tile=4)
    ctx.set_iteration_bound(8)
    with pytest.raises(pkg.FsError) as e:
        ctx.shifted_solve(-0.4, [0.05], b, **kw)
    assert e.value.code == pkg.fsmlmc.FS_ERR_TIMEOUT
    assert "iteration bound" in str(e.value)
    with pytest.raises(pkg.FsError) as e:
        ctx.mlmc_level_trace(-0.4, [0.05, 0.4], np.eye(4), 0, [6, 6], seed=31, job=2, lanes=2, **kw)
    assert e.value.code == pkg.fsmlmc.FS_ERR_TIMEOUT
    with pytest.raises(pkg.FsError) as e:
        ctx.set_iteration_bound(-1)
    assert e.value.code == pkg.fsmlmc.FS_ERR_ARG
    ctx.set_iteration_bound(0)
    x, st, rc = ctx.shifted_solve(-0.4, [0.05], b, **kw)
    assert rc == 0
    for k in range(6):
        assert rel_resid(u, x[0, k], b[k], -0.4, 0.05, dims) <= 1.05e-10, k
    out = ctx.mlmc_level_trace(-0.4, [0.05, 0.4], np.eye(4), 0, [6, 6], seed=31, job=2, lanes=2, **kw)
    assert out["rc"] == 0
    ctx.close()
