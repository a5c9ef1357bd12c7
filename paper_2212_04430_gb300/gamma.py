"""Dirac matrices in the DeGrand-Rossi (chiral) basis, for building Gamma insertions.

gamma_mu = [[0, G_mu], [G_mu^dag, 0]] with
  G_1 = [[0, i], [i, 0]],  G_2 = [[0, -1], [1, 0]],  G_3 = diag(i, -i),  G_4 = 1,
and gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1). This is the
basis the library's Wilson operator uses; a Gamma for `mlmc_level_trace` or
`variance_sample` must be written in it.
"""

import numpy as np

_G = {
    1: np.array([[0, 1j], [1j, 0]]),
    2: np.array([[0, -1], [1, 0]], dtype=complex),
    3: np.array([[1j, 0], [0, -1j]]),
    4: np.eye(2, dtype=complex),
}


def gamma_mu(mu):
    """gamma_mu for mu in 1..4 as a 4x4 complex matrix."""
    g = np.zeros((4, 4), dtype=complex)
    g[:2, 2:] = _G[mu]
    g[2:, :2] = _G[mu].conj().T
    return g


def gamma5():
    return gamma_mu(1) @ gamma_mu(2) @ gamma_mu(3) @ gamma_mu(4)


def gamma_matrix(spec):
    """Product of gamma matrices from a string such as "1", "g3", "g5g3", "g1g2" ("1"/"I": identity)."""
    s = spec.replace(" ", "").lower()
    out = np.eye(4, dtype=complex)
    if s in ("1", "i", "id", ""):
        return out
    parts = [p for p in s.split("g") if p]
    for p in parts:
        k = int(p)
        out = out @ (gamma5() if k == 5 else gamma_mu(k))
    return out


def to_abi(g):
    """4x4 complex -> contiguous double[4][4][2] for the C ABI."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.complex128).reshape(4, 4))
    return np.ascontiguousarray(g.view(np.float64).reshape(4, 4, 2))
