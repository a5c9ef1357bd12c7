"""Textbook BiCGStab and dense inverses for the shifted systems (oracle).

Solves Eq. (shifted_linear_systems), (D + s I) x = z, on the full,
unpreconditioned lattice: no even-odd splitting, no mixed precision, no
batching. BiCGStab follows H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13
(1992) 631, in its usual unpreconditioned form. The adjoint system
Eq. (conj_shifted_linear_systems) is solved through gamma_5-hermiticity,
(D + s)^-dag = gamma_5 (D + s)^-1 gamma_5 (Sec. 3.1).

For tiny lattices the dense matrix of D + s I is assembled column by column by
applying the operator to unit vectors, and inverted by LU (numpy.linalg).
"""

import numpy as np

from . import dirac


class SolveResult:
    def __init__(self, x, iters, rel_resid, converged):
        self.x = x
        self.iters = iters
        self.rel_resid = rel_resid
        self.converged = converged


def bicgstab(apply_A, b, tol=1e-12, max_iter=20000, x0=None):
    """Unpreconditioned BiCGStab for A x = b on flat complex vectors.

    Stops when ||b - A x|| <= tol ||b|| for the recursively updated residual,
    then reports the true residual.
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return SolveResult(np.zeros_like(b), 0, 0.0, True)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    r = b - apply_A(x)
    r_hat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    converged = np.linalg.norm(r) <= tol * nb
    while not converged and it < max_iter:
        it += 1
        rho = np.vdot(r_hat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_A(p)
        alpha = rho / np.vdot(r_hat, v)
        s = r - alpha * v
        t = apply_A(s)
        tt = np.vdot(t, t).real
        omega = np.vdot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        converged = np.linalg.norm(r) <= tol * nb
        if not np.isfinite(np.linalg.norm(r)):
            break
    true_r = np.linalg.norm(b - apply_A(x)) / nb
    return SolveResult(x, it, true_r, bool(true_r <= 10 * tol))


def shifted_solve(u, z, m, sigma, dims, bc_t=-1, tol=1e-12, max_iter=20000, cterm=None):
    """x = (D + sigma I)^-1 z by BiCGStab. z, x: canonical flat complex128[V][4][3].
    cterm: the clover term of `clover` (D_sw in place of D_W), or None."""
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))

    def apply_A(vec):
        f = vec.reshape(shp + (4, 3))
        out = dirac.apply_D(ul, f, m, sigma, bc_t)
        if cterm is not None:
            out = out + np.einsum("...satb,...tb->...sa", cterm, f)
        return out.ravel()

    res = bicgstab(apply_A, z.ravel(), tol=tol, max_iter=max_iter)
    res.x = res.x.reshape(z.shape)
    return res


def site_coords(dims):
    """(x, y, z, t) of every canonical site index."""
    lx, ly, lz, lt = dims
    s = np.arange(lx * ly * lz * lt)
    return np.stack([s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)])


def site_index(c, dims):
    lx, ly, lz, lt = dims
    return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))


def neighbour(dims, mu, step):
    """Canonical index of x + step*mu_hat (periodic wrap) and the bc flag of the wrap."""
    c = site_coords(dims)
    n = c.copy()
    n[mu] = c[mu] + step
    wrapped = (n[mu] < 0) | (n[mu] >= dims[mu])
    n[mu] %= dims[mu]
    return site_index(n, dims), wrapped


def dense_operator(u, m, sigma, dims, bc_t=-1, cterm=None):
    """Dense matrix of D + sigma I, complex128[12V, 12V], index = 12 site + 3 spin + colour.

    Assembled block by block from the definition in `dirac`:
      [x, x]      (4 + m + sigma) I            (+ the clover block C(x) for D_sw)
      [x, x+mu]   -1/2 (1 - gamma_mu) (x) U_mu(x)          (times bc_t on a t wrap)
      [x, x-mu]   -1/2 (1 + gamma_mu) (x) U_mu(x-mu)^dag   (times bc_t on a t wrap)
    """
    v = int(np.prod(dims))
    mat = np.zeros((v, 12, v, 12), dtype=np.complex128)
    sites = np.arange(v)
    mat[sites, :, sites, :] += (4.0 + m + sigma) * np.eye(12)
    if cterm is not None:
        mat[sites, :, sites, :] += cterm.reshape(v, 12, 12)
    for mu in range(4):
        fwd, fw_wrap = neighbour(dims, mu, +1)
        bwd, bw_wrap = neighbour(dims, mu, -1)
        ph_f = np.where(fw_wrap & (mu == 3), bc_t, 1.0)
        ph_b = np.where(bw_wrap & (mu == 3), bc_t, 1.0)
        blk_f = np.einsum("st,xab->xsatb", dirac.IDENT4 - dirac.GAMMA[mu], u[mu]).reshape(v, 12, 12)
        u_bwd_dag = np.conj(np.swapaxes(u[mu][bwd], 1, 2))
        blk_b = np.einsum("st,xab->xsatb", dirac.IDENT4 + dirac.GAMMA[mu], u_bwd_dag).reshape(v, 12, 12)
        np.add.at(mat, (sites, slice(None), fwd, slice(None)), -0.5 * ph_f[:, None, None] * blk_f)
        np.add.at(mat, (sites, slice(None), bwd, slice(None)), -0.5 * ph_b[:, None, None] * blk_b)
    return mat.reshape(12 * v, 12 * v)


def dense_inverse(u, m, sigma, dims, bc_t=-1, cterm=None):
    return np.linalg.inv(dense_operator(u, m, sigma, dims, bc_t, cterm))


def dense_GammaOmega(u, gamma, p, dims):
    """Dense matrix of Gamma Omega_p: block [x, x + p z] = Gamma (x) W(x) (Sec. 1)."""
    v = int(np.prod(dims))
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))
    w = dirac.wilson_line(ul, p).reshape(v, 3, 3)
    c = site_coords(dims)
    c[2] = (c[2] + p) % dims[2]
    tgt = site_index(c, dims)
    mat = np.zeros((v, 12, v, 12), dtype=np.complex128)
    blk = np.einsum("st,xab->xsatb", gamma, w).reshape(v, 12, 12)
    np.add.at(mat, (np.arange(v), slice(None), tgt, slice(None)), blk)
    return mat.reshape(12 * v, 12 * v)


def dense_gamma5(dims):
    v = int(np.prod(dims))
    return np.kron(np.eye(v), np.kron(dirac.GAMMA5, np.eye(3)))
