"""The allocation-free dslash entry point, through the C ABI.

wilson_dslash_noalloc serves callers that may not allocate device memory while
they run (stream capture, fixed device-memory budgets, latency-critical loops):
it keeps its scratch in one static device array instead of context buffers.
Two calls in a row on fresh inputs must each reproduce the regular
wilson_dslash to the FP64 dslash tolerance of the parity tests, and the second
call must not change the device's free memory. This file sorts last so that a
run stopping at its first failure has run every other test already.
"""

import ctypes

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

FP64_DSLASH_TOL = 1e-13


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2212_04430_gb300 import fsmlmc
    return fsmlmc


def test_noalloc_dslash_matches_wilson_dslash_twice(lib):
    torch = pytest.importorskip("torch")
    dims = (8, 8, 4, 8)
    nrhs = 3
    m, sigma = -0.4, 0.07
    u = inputs.gauge_field(dims, "haar", seed=4242)
    ctx = lib.Context(dims, bc_t=-1, device=0)
    ctx.fs_set_gauge(u)
    dev = torch.device("cuda", 0)
    U_d = torch.from_numpy(np.ascontiguousarray(u).view(np.float64).ravel().copy()).to(dev)
    stream = torch.cuda.current_stream()
    free_after_first = None
    for call in range(2):
        psi = inputs.random_spinor(dims, 300 + call, nvec=nrhs)
        ref = ctx.wilson_dslash(m, sigma, psi, prec="f64")
        in_d = torch.from_numpy(np.ascontiguousarray(psi).view(np.float64).ravel().copy()).to(dev)
        out_d = torch.full_like(in_d, float("nan"))
        torch.cuda.synchronize()
        if call == 1:
            free_after_first = torch.cuda.mem_get_info(0)[0]
        rc = lib.wilson_dslash_noalloc(dims, -1, m, sigma, U_d.data_ptr(), in_d.data_ptr(), out_d.data_ptr(),
                                       nrhs, stream.cuda_stream)
        assert rc == 0, ("wilson_dslash_noalloc returned", rc)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info(0)[0] == free_after_first
        got = out_d.cpu().numpy().view(np.complex128).reshape(psi.shape)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < FP64_DSLASH_TOL, (call, err)
    ctx.close()


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 8), 3), ((4, 4, 4, 8), 37), ((4, 4, 4, 8), 64)])
@pytest.mark.parametrize("bc_t", [-1, 1])
def test_noalloc_tile_shapes_and_boundary_conditions(lib, dims, nrhs, bc_t):
    """More than 32 right-hand sides (two system blocks of a tile, a ragged one for 37) and
    both time boundary conditions, against wilson_dslash, two calls in a row."""
    torch = pytest.importorskip("torch")
    m, sigma = -0.3, 0.11
    u = inputs.gauge_field(dims, "smooth", seed=4300 + nrhs, eps=0.4)
    ctx = lib.Context(dims, bc_t=bc_t, device=0)
    ctx.fs_set_gauge(u)
    dev = torch.device("cuda", 0)
    U_d = torch.from_numpy(np.ascontiguousarray(u).view(np.float64).ravel().copy()).to(dev)
    stream = torch.cuda.current_stream()
    for call in range(2):
        psi = inputs.random_spinor(dims, 500 + 7 * call + nrhs, nvec=nrhs)
        ref = ctx.wilson_dslash(m, sigma, psi, prec="f64")
        in_d = torch.from_numpy(np.ascontiguousarray(psi).view(np.float64).ravel().copy()).to(dev)
        out_d = torch.full_like(in_d, float("nan"))
        rc = lib.wilson_dslash_noalloc(dims, bc_t, m, sigma, U_d.data_ptr(), in_d.data_ptr(), out_d.data_ptr(),
                                       nrhs, stream.cuda_stream)
        assert rc == 0, ("wilson_dslash_noalloc returned", rc)
        torch.cuda.synchronize()
        got = out_d.cpu().numpy().view(np.complex128).reshape(psi.shape)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < FP64_DSLASH_TOL, (call, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    torch = pytest.importorskip("torch")
    dims = (16, 16, 16, 32)  # 576 V + 384 V > 32 MiB already at one right-hand side
    dev = torch.device("cuda", 0)
    buf = torch.zeros(8, dtype=torch.float64, device=dev)  # never touched: rejected before any launch
    rc = lib.wilson_dslash_noalloc(dims, -1, -0.4, 0.0, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 1, 0)
    assert rc == lib.FS_ERR_BUDGET
    assert lib.wilson_dslash_noalloc((8, 8, 8, 8), -1, -0.4, 0.0, buf.data_ptr(), buf.data_ptr(),
                                     buf.data_ptr(), 65, 0) == lib.FS_ERR_ARG
