"""Plain FP64 CPU oracle for Frequency-Splitting MLMC trace estimation.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA path; the two meet only in the seeded inputs of the
``inputs`` package and in the counter-based RNG, which each side implements
separately from the published Philox4x32-10 definition.

Everything here is slow and literal: numpy arrays over the 4-d lattice,
operators applied term by term as written, textbook BiCGStab, dense LU from
numpy.linalg for tiny lattices. Each function cites the passage of the paper
(arXiv:2212.04430, Whyte, Stathopoulos, Romero, Orginos) it follows.

Modules:
  dirac       Wilson-Dirac operator D, gamma matrices, Gamma and Omega_p
  philox      Philox4x32-10 counter RNG and the Z4 noise vectors
  solve       textbook BiCGStab, dense operator and inverse
  estimators  level traces (Eq. fs_trace_est), practical variance
              (Eq. practical_variance), variance sampling (Sec. 3.1 algorithm)
  freefield   momentum-space closed form for free-field traces and spectrum
  clover      the clover (Sheikholeslami-Wohlert) term of the Wilson-clover operator
"""

from . import dirac, philox, solve, estimators, freefield, clover  # noqa: F401
