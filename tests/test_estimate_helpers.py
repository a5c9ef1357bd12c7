"""The FS estimate, its variance and the sampled level variances are formed by the C ABI
(fs_trace_total, fs_sampled_level_variances), so a C caller gets them too; called here through
the binding's ctypes marshalling on hand-worked numbers (host code, no GPU)."""

import numpy as np
import pytest

import paper_2212_04430_gb300 as pkg


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def test_trace_total_and_v_fs():
    """Eq. (fs_trace_est) summed over levels, Eq. (total_var): three levels, two displacement rows."""
    trace = np.array([[[1.0, -2.0], [0.5, 0.25], [-3.0, 1.0]],
                      [[2.0, 0.0], [0.0, 4.0], [1.0, -1.0]]])
    var = np.array([[8.0, 3.0, 5.0],
                    [1.0, 0.0, 2.5]])
    ns = [4, 3, 10]
    total, v_fs = pkg.fs_trace_total(trace, var, ns)
    assert np.array_equal(total, [[-1.5, -0.75], [3.0, 3.0]])
    # 8/4 + 3/3 + 5/10 = 3.5 ; 1/4 + 0 + 2.5/10 = 0.5
    assert np.allclose(v_fs, [3.5, 0.5], rtol=0, atol=1e-15)


def test_trace_total_rejects_bad_inputs():
    with pytest.raises(pkg.FsError) as e:
        pkg.fs_trace_total(np.zeros((1, 2, 2)), np.zeros((1, 2)), [3, 0])  # a level without samples
    assert e.value.code == 1
    with pytest.raises(pkg.FsError) as e:
        pkg.fs_trace_total(np.zeros((1, 2, 2)), np.array([[1.0, np.nan]]), [3, 3])
    assert e.value.code == 2


def test_sampled_level_variances():
    """Eq. (sampled_prod): V_l(s_i, s_j) = (s_j - s_i)^2 Vbar_l(s_i, s_j) above the diagonal."""
    s_hat = np.array([0.0, 0.05, 0.25, 0.5, 1.0])
    m = s_hat.size
    vbar = np.zeros((2, m, m))
    for q in range(2):
        for i in range(m):
            for j in range(i, m):
                vbar[q, i, j] = 10.0 * (q + 1) + i + 0.5 * j
    vl = pkg.fs_sampled_level_variances(s_hat, vbar)
    assert vl.shape == vbar.shape
    assert vl[0, 0, 4] == pytest.approx(1.0 * 12.0, rel=1e-15)         # (1 - 0)^2 (10 + 0 + 2)
    assert vl[1, 1, 2] == pytest.approx(0.04 * 22.0, rel=1e-14)        # (0.25 - 0.05)^2 (20 + 1 + 1)
    assert vl[0, 3, 3] == 0.0                                           # equal shifts
    assert np.all(np.tril(vl[0], -1) == 0.0) and np.all(np.tril(vl[1], -1) == 0.0)
