"""fs_measure_peak, the measured FP32 and FP64 roofs the bench compares the hop kernels with:
each kind runs and reports a rate inside wide bounds for this GPU class (the nominal FP32 rate of
a GB300 is about 80 TFLOP/s, FP64 about 1.25), and bad arguments are refused before any launch."""

import pytest

pkg = pytest.importorskip("paper_2212_04430_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("kind,lo,hi", [("f32", 20.0, 200.0), ("f32x2", 20.0, 200.0), ("f64", 0.2, 100.0)])
def test_measured_peak_in_range(kind, lo, hi):
    tf, ms = pkg.fs_measure_peak(kind, 0.2)
    assert lo < tf < hi, (kind, tf)
    assert 50.0 < ms < 2000.0, (kind, ms)


def test_measure_peak_rejects_bad_arguments():
    lib = pkg.load_library()
    import ctypes
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.fs_measure_peak(7, 1.0, ctypes.byref(tf), ctypes.byref(ms)) == pkg.fsmlmc.FS_ERR_ARG
    assert lib.fs_measure_peak(0, 0.0, ctypes.byref(tf), ctypes.byref(ms)) == pkg.fsmlmc.FS_ERR_ARG
    assert lib.fs_measure_peak(0, 61.0, ctypes.byref(tf), ctypes.byref(ms)) == pkg.fsmlmc.FS_ERR_ARG
