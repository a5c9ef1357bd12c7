"""GB300-native Frequency-Splitting MLMC trace estimation (arXiv:2212.04430).

The compute path is the CUDA library libfsmlmc.so (C ABI: include/fsmlmc.h);
this package holds its build script, a thin ctypes binding with the same entry
point names, and the Dirac matrix table used to build Gamma insertions.
"""

from .fsmlmc import (  # noqa: F401
    Context,
    Server,
    FsError,
    PREC,
    ESTIMATOR,
    load_library,
    fs_ctx_create,
    fs_set_gauge,
    fs_set_clover,
    wilson_dslash,
    shifted_solve,
    mlmc_level_trace,
    variance_sample,
    fs_noise_codes,
    fs_interp_variances,
    fs_select_shifts,
    fs_sample_allocation,
    fs_eval_grid,
    fs_probing_colors,
    fs_trace_total,
    fs_sampled_level_variances,
    fs_measure_peak,
)
from .gamma import gamma_matrix, gamma_mu, gamma5  # noqa: F401
