"""Hopping parameter expansion of the single-shift trace (test infrastructure: the oracle).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module; the library's
own implementation shares no code with it.

Follows arXiv:2212.04430, Sec. 3.1 (the remark after Eq. (sampled_single)): when m + s > 0 the
variance of the estimator of Tr(Gamma Omega_p (D + s)^-1) is reduced with the (generalised)
hopping parameter expansion truncated at order K (K = 4 in the paper), and the trace of the
terms of order k < K is computed exactly with distance-(K-1) displacement-p probing vectors.

For the Wilson operator (no clover term, so the expansion is the classical one):
    D + s = A (1 - kappa H),  A = 4 + m + s,  kappa = 1 / (2 A),
    (H psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x + mu) + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu),
    (D + s)^-1 = sum_{k<K} (kappa H)^k / A + (kappa H)^K (D + s)^-1,
so  Tr(G Om (D+s)^-1) = T_exact + E_z[ z^dag G Om (kappa H)^K (D+s)^-1 z ],
    T_exact = sum_{k<K} Tr(G Om (kappa H)^k) / A.
The geometric series converges when ||kappa H|| < 1; ||H|| <= 8, so A > 4, i.e. m + s > 0.
"""

import numpy as np

from . import dirac, probing, solve


def apply_H(u, psi, dims, bc_t=-1):
    """H psi on canonical flat vectors [..., V, 4, 3]: the hopping term, H = 2 (4 - D_{m=0})."""
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))
    lead = psi.shape[:-3]
    x = psi.reshape(lead + shp + (4, 3))
    out = 2.0 * (4.0 * x - dirac.apply_D(ul, x, 0.0, 0.0, bc_t))
    return out.reshape(psi.shape)


def stochastic_part(u, solver, z, m, sigma, gamma, p, K, dims, bc_t=-1):
    """z^dag Gamma Omega_p (kappa H)^K x, x = (D + sigma)^-1 z: the remainder after order K."""
    from . import estimators as est
    kappa = 1.0 / (2.0 * (4.0 + m + sigma))
    y = solver(z, sigma)
    for _ in range(K):
        y = kappa * apply_H(u, y, dims, bc_t)
    return est.contract(u, z, y, gamma, p, dims)


def exact_part_dense(u, m, sigma, gamma, p, K, dims, bc_t=-1):
    """T_exact = sum_{k<K} Tr(Gamma Omega_p (kappa H)^k) / A from dense matrices (tiny lattices)."""
    A = 4.0 + m + sigma
    n = 12 * int(np.prod(dims))
    h = 2.0 * (A * np.eye(n) - solve.dense_operator(u, m, sigma, dims, bc_t))  # H = 2 (A - (D + s))
    go = solve.dense_GammaOmega(u, gamma, p, dims)
    t = 0j
    pw = np.eye(n, dtype=np.complex128)
    for k in range(K):
        t += np.trace(go @ pw)
        pw = (h @ pw) / (2.0 * A)
    return complex(t / A)


def exact_part_probed(u, m, sigma, gamma, p, K, dims, colors, ncolors, bc_t=-1):
    """The same sum from probing vectors (the paper's route): sum over the colours j and the 12
    spin-colour indices a of e_ja^dag Gamma Omega_p sum_{k<K} (kappa H)^k e_ja / A, with
    e_ja = 1 on the sites of colour j at index a. Exact when no two distinct sites of one colour
    are linked by Gamma Omega_p H^k, k < K: a displacement-p distance-(K-1) colouring."""
    from . import estimators as est
    v = int(np.prod(dims))
    A = 4.0 + m + sigma
    kappa = 1.0 / (2.0 * A)
    t = 0j
    for (j, a) in probing.pieces(ncolors, True):
        e = np.zeros((v, 4, 3), dtype=np.complex128)
        e[np.asarray(colors) == j, a // 3, a % 3] = 1.0
        y = e / A
        for k in range(K):
            t += est.contract(u, e, y, gamma, p, dims)
            y = kappa * apply_H(u, y, dims, bc_t)
    return complex(t)


def remainder_matrix(u, m, sigma, gamma, p, K, dims, bc_t=-1):
    """Dense Gamma Omega_p (kappa H)^K (D + sigma)^-1 (its Z4 variance is the HPE estimator's)."""
    A = 4.0 + m + sigma
    n = 12 * int(np.prod(dims))
    d = solve.dense_operator(u, m, sigma, dims, bc_t)
    kh = (A * np.eye(n) - d) / A  # kappa H = (A - (D + s)) / A
    return solve.dense_GammaOmega(u, gamma, p, dims) @ np.linalg.matrix_power(kh, K) @ np.linalg.inv(d)
