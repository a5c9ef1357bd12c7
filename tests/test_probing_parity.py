"""Probing colours and the probed solve count: the library (host code, no GPU) against the
oracle (paper Sec. 2.1, Eq. (probing_vectors), displacement-p probing; Sec. 3.1, the count
12 c m N_s of full spin-colour dilution). Colours are integers: compared bit-exactly."""

import ctypes

import numpy as np
import pytest

from oracle import probing as opr

pkg = pytest.importorskip("paper_2212_04430_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("dims,k,p", [
    ((4, 4, 4, 4), 1, 0),
    ((4, 4, 4, 8), 2, 0),
    ((4, 4, 8, 4), 3, 0),       # ball wider than the short axes: offsets wrap onto one site
    ((4, 4, 8, 4), 1, 2),
    ((4, 2, 8, 4), 2, 3),
    ((6, 4, 6, 2), 4, 1),
    ((2, 2, 4, 2), 2, 2),       # p = Lz / 2: x + p z and x - p z are the same site
    ((3, 5, 7, 2), 2, 1),       # odd sizes (the colouring itself needs no even-odd split)
])
def test_colors_match_the_oracle(dims, k, p):
    col, nc = pkg.fs_probing_colors(dims, k, p)
    ref, nref = opr.greedy_coloring(dims, k, p)
    assert nc == nref
    assert np.array_equal(col.astype(np.int64), ref)


def test_distance_one_is_the_checkerboard_at_16x32():
    dims = (16, 16, 16, 32)
    col, nc = pkg.fs_probing_colors(dims, 1, 0)
    x = np.indices(dims[::-1]).reshape(4, -1)[::-1]  # x fastest
    assert nc == 2
    assert np.array_equal(col, x.sum(axis=0) % 2)


def test_paper_sized_colorings_are_valid_and_fast():
    """p4k4 and p8k7 on a 16^3 x 32 lattice (the paper's probing sets, its own generator gives
    14 and 16 colours; the greedy count may differ): validity checked on sampled sites."""
    dims = (16, 16, 16, 32)
    rng = np.random.default_rng(3)
    for (p, k) in ((4, 4), (8, 7)):
        col, nc = pkg.fs_probing_colors(dims, k, p)
        assert col.min() == 0 and col.max() == nc - 1
        assert len(np.unique(col)) == nc
        for i in rng.integers(0, col.size, 20):
            x = np.array([i % 16, (i // 16) % 16, (i // 256) % 16, i // 4096])
            for sgn in (1, -1):
                c = x.copy()
                c[2] = (c[2] + sgn * p) % 16
                # every site within distance k of x +- p z, except x itself
                for d in _ball(k):
                    y = (c + d) % np.array(dims)
                    j = y[0] + 16 * (y[1] + 16 * (y[2] + 16 * y[3]))
                    if j != i:
                        assert col[j] != col[i]


def _ball(k):
    r = np.arange(-k, k + 1)
    d = np.stack(np.meshgrid(r, r, r, r, indexing="ij"), -1).reshape(-1, 4)
    return d[np.abs(d).sum(1) <= k]


def test_bad_arguments_are_refused():
    L = pkg.load_library()
    out = np.empty(256, dtype=np.int32)
    n = ctypes.c_int(0)
    ptr = out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    for dims, k, p in (((4, 4, 4, 4), 0, 0), ((4, 4, 4, 4), 17, 0), ((4, 4, 4, 4), 1, 4), ((4, 4, 4, 4), 1, -1),
                       ((4, 0, 4, 4), 1, 0)):
        d = (ctypes.c_int * 4)(*dims)
        assert L.fs_probing_colors(d, k, p, ptr, ctypes.byref(n)) == 1
    assert L.fs_probing_colors(None, 1, 0, ptr, ctypes.byref(n)) == 1


def _num_solves(n_samples, colors=None, ncolors=None, dilute=False):
    from paper_2212_04430_gb300.fsmlmc import MlmcParams, _set_probing
    L = pkg.load_library()
    ns = np.ascontiguousarray(n_samples, dtype=np.int32)
    P = MlmcParams()
    P.nlev = ns.size
    P.n_samples = ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    keep = _set_probing(P, colors, ncolors, dilute)  # noqa: F841
    return L.fs_mlmc_num_solves(ctypes.byref(P))


def test_solve_count_with_probing_and_dilution():
    col = np.zeros(16, dtype=np.int32)
    col[::2] = 1
    assert _num_solves([4, 3, 2]) == 2 * 4 + 2 * 3 + 2
    assert _num_solves([4, 3, 2], dilute=True) == 12 * (2 * 4 + 2 * 3 + 2)
    assert _num_solves([4, 3, 2], col, 2) == 2 * (2 * 4 + 2 * 3 + 2)
    # one shift, N_s samples, c colours, full dilution: 12 c N_s (the paper's count for m = 1)
    assert _num_solves([5], col, 2, True) == 12 * 2 * 5
    assert _num_solves([5], col, 0) == -1           # colours without a count
    assert _num_solves([1 << 20] * 2, col, 1 << 10, True) == -1   # beyond 2^31 - 1
