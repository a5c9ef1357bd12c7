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

The generalised expansion (the Wilson-clover operator of `clover`, passed as cterm): the site
factor is a 12x12 block per site, A(x) = (4 + m + s) 1 + C(x), and
    D_sw + s = A (1 - K),  K = A^-1 H / 2,
    (D_sw + s)^-1 = sum_{k<K} K^k A^-1 + K^K (D_sw + s)^-1,
so T_exact = sum_{k<K} Tr(G Om K^k A^-1) and the remainder is z^dag G Om K^K (D_sw + s)^-1 z. With
C = 0 this is the classical expansion (K = kappa H, A^-1 = 1 / A). The identity is exact for any
order; the series converges where the smallest eigenvalue of A(x) exceeds 4.
"""

import numpy as np

from . import clover, dirac, probing, solve


def site_factor(cterm, A, v):
    """A(x) = A 1 + C(x) as 12x12 blocks per canonical site: complex128[V, 12, 12]."""
    blocks = np.broadcast_to(A * np.eye(12, dtype=np.complex128), (v, 12, 12)).copy()
    if cterm is not None:
        blocks = blocks + clover.site_blocks(cterm)
    return blocks


def apply_site_inverse(blocks, psi):
    """A(x)^-1 psi(x) site by site (a 12x12 solve per site), psi [..., V, 4, 3]."""
    v = psi.shape[-3]
    x = psi.reshape(psi.shape[:-3] + (v, 12, 1))
    return np.linalg.solve(blocks, x)[..., 0].reshape(psi.shape)


def dense_site_factor(blocks):
    """The block-diagonal dense matrix of A(x) (index 12 site + 3 spin + colour)."""
    v = blocks.shape[0]
    out = np.zeros((12 * v, 12 * v), dtype=np.complex128)
    for i in range(v):
        out[12 * i:12 * i + 12, 12 * i:12 * i + 12] = blocks[i]
    return out


def apply_H(u, psi, dims, bc_t=-1):
    """H psi on canonical flat vectors [..., V, 4, 3]: the hopping term, H = 2 (4 - D_{m=0})."""
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))
    lead = psi.shape[:-3]
    x = psi.reshape(lead + shp + (4, 3))
    out = 2.0 * (4.0 * x - dirac.apply_D(ul, x, 0.0, 0.0, bc_t))
    return out.reshape(psi.shape)


def stochastic_part(u, solver, z, m, sigma, gamma, p, K, dims, bc_t=-1, cterm=None):
    """z^dag Gamma Omega_p (kappa H)^K x, x = (D + sigma)^-1 z: the remainder after order K
    (with cterm: K = A^-1 H / 2 applied K times to x = (D_sw + sigma)^-1 z)."""
    from . import estimators as est
    y = solver(z, sigma)
    if cterm is None:
        kappa = 1.0 / (2.0 * (4.0 + m + sigma))
        for _ in range(K):
            y = kappa * apply_H(u, y, dims, bc_t)
    else:
        blocks = site_factor(cterm, 4.0 + m + sigma, int(np.prod(dims)))
        for _ in range(K):
            y = apply_site_inverse(blocks, 0.5 * apply_H(u, y, dims, bc_t))
    return est.contract(u, z, y, gamma, p, dims)


def exact_part_dense(u, m, sigma, gamma, p, K, dims, bc_t=-1, cterm=None):
    """T_exact = sum_{k<K} Tr(Gamma Omega_p (kappa H)^k) / A from dense matrices (tiny lattices);
    with cterm sum_{k<K} Tr(Gamma Omega_p K^k A^-1)."""
    A = 4.0 + m + sigma
    n = 12 * int(np.prod(dims))
    go = solve.dense_GammaOmega(u, gamma, p, dims)
    if cterm is not None:
        a = dense_site_factor(site_factor(cterm, A, n // 12))
        ainv = np.linalg.inv(a)
        kmat = ainv @ (a - solve.dense_operator(u, m, sigma, dims, bc_t, cterm))  # K = A^-1 (A - (D_sw + s))
        t = 0j
        pw = ainv
        for k in range(K):
            t += np.trace(go @ pw)
            pw = kmat @ pw
        return complex(t)
    h = 2.0 * (A * np.eye(n) - solve.dense_operator(u, m, sigma, dims, bc_t))  # H = 2 (A - (D + s))
    t = 0j
    pw = np.eye(n, dtype=np.complex128)
    for k in range(K):
        t += np.trace(go @ pw)
        pw = (h @ pw) / (2.0 * A)
    return complex(t / A)


def exact_part_probed(u, m, sigma, gamma, p, K, dims, colors, ncolors, bc_t=-1, cterm=None):
    """The same sum from probing vectors (the paper's route): sum over the colours j and the 12
    spin-colour indices a of e_ja^dag Gamma Omega_p sum_{k<K} (kappa H)^k e_ja / A, with
    e_ja = 1 on the sites of colour j at index a. Exact when no two distinct sites of one colour
    are linked by Gamma Omega_p H^k, k < K: a displacement-p distance-(K-1) colouring. With cterm
    the pieces take e^dag Gamma Omega_p K^k A^-1 e (A^-1 is site-local, so the same colours serve)."""
    from . import estimators as est
    v = int(np.prod(dims))
    A = 4.0 + m + sigma
    kappa = 1.0 / (2.0 * A)
    blocks = site_factor(cterm, A, v) if cterm is not None else None
    t = 0j
    for (j, a) in probing.pieces(ncolors, True):
        e = np.zeros((v, 4, 3), dtype=np.complex128)
        e[np.asarray(colors) == j, a // 3, a % 3] = 1.0
        y = e / A if blocks is None else apply_site_inverse(blocks, e)
        for k in range(K):
            t += est.contract(u, e, y, gamma, p, dims)
            if blocks is None:
                y = kappa * apply_H(u, y, dims, bc_t)
            else:
                y = apply_site_inverse(blocks, 0.5 * apply_H(u, y, dims, bc_t))
    return complex(t)


def remainder_matrix(u, m, sigma, gamma, p, K, dims, bc_t=-1, cterm=None):
    """Dense Gamma Omega_p (kappa H)^K (D + sigma)^-1 (its Z4 variance is the HPE estimator's);
    with cterm Gamma Omega_p K^K (D_sw + sigma)^-1."""
    A = 4.0 + m + sigma
    n = 12 * int(np.prod(dims))
    d = solve.dense_operator(u, m, sigma, dims, bc_t, cterm)
    if cterm is not None:
        a = dense_site_factor(site_factor(cterm, A, n // 12))
        kh = np.linalg.solve(a, a - d)  # K = A^-1 (A - (D_sw + s))
    else:
        kh = (A * np.eye(n) - d) / A  # kappa H = (A - (D + s)) / A
    return solve.dense_GammaOmega(u, gamma, p, dims) @ np.linalg.matrix_power(kh, K) @ np.linalg.inv(d)
