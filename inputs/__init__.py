"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module generates *inputs only*: gauge fields, gauge transformations and
random spinor fields, all from numpy's PCG64 generator seeded by an integer.
It contains none of the trace-estimation arithmetic (no Dirac operator, no
solver, no noise, no contraction), so the oracle and the CUDA path can both
consume its bytes without sharing any of the method's code.

Canonical host layouts (identical to the C-ABI's):
  site index   s = x + Lx*(y + Ly*(z + Lz*t))
  gauge field  complex128[4][V][3][3]   U[mu][s] is the link s -> s+mu_hat
               (mu = 0,1,2,3 for x,y,z,t); as doubles: [4][V][3][3][2]
  spinor field complex128[V][4][3]      as doubles: [V][4][3][2]
"""

from .gauge import (
    lattice_volume,
    haar_su3,
    smoothed_su3,
    gauge_field,
    unit_gauge,
    abelian_field,
    random_gauge_rotation,
    gauge_transform,
    random_spinor,
    as_real_view,
)

__all__ = [
    "lattice_volume",
    "haar_su3",
    "smoothed_su3",
    "gauge_field",
    "unit_gauge",
    "abelian_field",
    "random_gauge_rotation",
    "gauge_transform",
    "random_spinor",
    "as_real_view",
]
