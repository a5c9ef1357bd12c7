"""FS-MLMC level traces, practical variance and variance sampling (oracle).

Follows arXiv:2212.04430:
  * Hutchinson estimator with Z4 noise, Eq. (test)
  * telescoping levels over shifts sigma_0 < ... < sigma_L, Eq. (tele_sum),
    Eq. (tele_sum_prod_disp), and the FS trace estimator Eq. (fs_trace_est)
  * practical variance, Eq. (practical_variance)
  * variance sampling of V_L and bar V_l, Sec. 3.1 algorithm, with
    Eq. (sampled_single) and Eq. (bar_vl)

Readings of the paper adopted here:
  * Level samples use N samples indexed 0..N-1 and weight 1/N (Eq. (test)
    prints 1/s, Eq. (fs_trace_est) sums s = 0..N_l).
  * Three estimators of a level l < L, all with expectation
    Tr(Gamma Omega_p [(D+sigma_l)^-1 - (D+sigma_{l+1})^-1]):
      DIFF        z^dag Gamma Omega_p (x_l - x_{l+1}),  x_k = (D+sigma_k)^-1 z
                  (the two inverses of Eq. (tele_sum) on the same noise)
      SPLIT_EVEN  (sigma_{l+1}-sigma_l) y_l^dag Gamma Omega_p x_{l+1},
                  y_l = (D+sigma_l)^-dag z        (Eq. (fs_trace_est))
      PRODUCT     (sigma_{l+1}-sigma_l) z^dag Gamma Omega_p (D+sigma_l)^-1 (D+sigma_{l+1})^-1 z
                  (Eq. (tele_sum_prod_disp0), the "standard random-noise" form)
    The last level is z^dag Gamma Omega_p (D+sigma_L)^-1 z for all three.
  * The adjoint solution is y = (D+s)^-dag z = gamma_5 (D+s)^-1 gamma_5 z,
    i.e. a solve with right-hand side gamma_5 z (the paper's y = gamma_5 x of
    Sec. 3.1 step 4 holds only with spin dilution).
  * Practical variance uses 1/N as printed (the biased form).
  * The exact variance of z^dag A z for Z4 noise is ||A||_F^2 - sum_i |A_ii|^2;
    Eq. (test_var) prints twice that (exact for real Z2 noise on a real
    symmetric A). Both are provided.
"""

import numpy as np

from . import dirac, philox, solve

DIFF = 0
SPLIT_EVEN = 1
PRODUCT = 2
ESTIMATORS = {"diff": DIFF, "split_even": SPLIT_EVEN, "product": PRODUCT}


def contract(u, left, right, gamma, p, dims):
    """left^dag Gamma Omega_p right = sum_x left(x)^dag Gamma W(x) right(x + p z_hat)."""
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))
    r = right.reshape(shp + (4, 3))
    go = dirac.apply_GammaOmega(ul, gamma, r, p)
    return complex(np.vdot(left.ravel(), go.ravel()))


def practical_variance(samples):
    """Eq. (practical_variance): (1/N) sum_k |c_k|^2 - |t|^2, t = (1/N) sum_k c_k."""
    c = np.asarray(samples, dtype=np.complex128)
    n = c.shape[0]
    t = c.sum(axis=0) / n
    return (np.abs(c) ** 2).sum(axis=0) / n - np.abs(t) ** 2


def exact_z4_variance(a):
    """Variance of z^dag A z over Z4 noise: ||A||_F^2 - sum_i |A_ii|^2."""
    return float((np.abs(a) ** 2).sum() - (np.abs(np.diag(a)) ** 2).sum())


def exact_var_paper(a):
    """Eq. (test_var) as printed: 2 (||A||_F^2 - sum_i |A_ii|^2)."""
    return 2.0 * exact_z4_variance(a)


def make_solver(u, m, dims, bc_t=-1, tol=1e-12, cterm=None):
    """Returns solve(z, sigma) -> (D + sigma)^-1 z by BiCGStab (canonical flat arrays); with
    cterm (`clover.clover_term`) the operator is the Wilson-clover D_sw."""
    def _solve(z, sigma):
        res = solve.shifted_solve(u, z, m, sigma, dims, bc_t, tol=tol, cterm=cterm)
        if not res.converged:
            raise RuntimeError("oracle BiCGStab did not converge (sigma=%g, resid=%g)"
                               % (sigma, res.rel_resid))
        return res.x
    return _solve


def make_dense_solver(u, m, dims, bc_t=-1, cterm=None):
    """Same interface, through dense LU inverses (tiny lattices only)."""
    cache = {}
    v = int(np.prod(dims))

    def _solve(z, sigma):
        if sigma not in cache:
            cache[sigma] = solve.dense_inverse(u, m, sigma, dims, bc_t, cterm)
        return (cache[sigma] @ z.ravel()).reshape(v, 4, 3)
    return _solve


def adjoint_solution(solver, z, sigma):
    """y = (D + sigma)^-dag z = gamma_5 (D + sigma)^-1 gamma_5 z."""
    return dirac.spin_mul(dirac.GAMMA5, solver(dirac.spin_mul(dirac.GAMMA5, z), sigma))


def level_sample(u, solver, z, sigmas, level, gamma, p, dims, estimator):
    """One sample of level `level` on noise z (Eq. (fs_trace_est) and its variants)."""
    L = len(sigmas) - 1
    if level == L:
        return contract(u, z, solver(z, sigmas[L]), gamma, p, dims)
    s0, s1 = sigmas[level], sigmas[level + 1]
    if estimator == DIFF:
        x0 = solver(z, s0)
        x1 = solver(z, s1)
        return contract(u, z, x0, gamma, p, dims) - contract(u, z, x1, gamma, p, dims)
    if estimator == SPLIT_EVEN:
        y = adjoint_solution(solver, z, s0)
        x1 = solver(z, s1)
        return (s1 - s0) * contract(u, y, x1, gamma, p, dims)
    if estimator == PRODUCT:
        x1 = solver(z, s1)
        x01 = solver(x1, s0)
        return (s1 - s0) * contract(u, z, x01, gamma, p, dims)
    raise ValueError("unknown estimator")


def level_samples(u, m, sigmas, gamma, p, n_samples, seed, job, dims, bc_t=-1,
                  estimator=DIFF, solver=None, levels=None, sample_ids=None):
    """Per-level sample values c_{s,l} with independent Z4 noise z_{s,l} per level.

    Returns a list over levels of complex128 arrays [N_l].
    `levels` / `sample_ids` restrict the work to a subset (for sampled parity).
    """
    v = int(np.prod(dims))
    if solver is None:
        solver = make_solver(u, m, dims, bc_t)
    L = len(sigmas) - 1
    out = []
    for lev in range(L + 1):
        if levels is not None and lev not in levels:
            out.append(None)
            continue
        ids = range(n_samples[lev]) if sample_ids is None else sample_ids
        vals = []
        for s in ids:
            z = philox.z4_noise(v, seed, job, lev, s)
            vals.append(level_sample(u, solver, z, sigmas, lev, gamma, p, dims, estimator))
        out.append(np.array(vals, dtype=np.complex128))
    return out


def mlmc_level_trace(u, m, sigmas, gamma, p, n_samples, seed, job, dims, bc_t=-1,
                     estimator=DIFF, solver=None):
    """FS trace estimate, Eq. (fs_trace_est): per-level means T_l, practical variances
    V_l (Eq. (practical_variance)), the total trace sum_l T_l and V_FS = sum_l V_l/N_l
    (Eq. (total_var))."""
    samples = level_samples(u, m, sigmas, gamma, p, n_samples, seed, job, dims, bc_t,
                            estimator, solver)
    traces = np.array([c.mean() for c in samples])
    var = np.array([practical_variance(c) for c in samples])
    n = np.array(n_samples, dtype=np.float64)
    return {"samples": samples, "trace": traces, "var": var,
            "total": complex(traces.sum()), "v_fs": float((var / n).sum())}


def variance_sample(u, m, s_hat, gamma, p_list, n_s, seed, job, dims, bc_t=-1,
                    solver=None):
    """Sec. 3.1 algorithm: sampled V_L(s_i) (Eq. (sampled_single)) and
    bar V_l(s_i, s_j), j >= i (Eq. (bar_vl)), for every displacement p in p_list.

    For each noise z_k and each shift s_i: x^(i) = (D+s_i)^-1 z_k and
    y^(i) = (D+s_i)^-dag z_k. Then a_i = z_k^dag Gamma Omega_p x^(i) and
    b_ij = y^(i)^dag Gamma Omega_p x^(j); both feed Eq. (practical_variance).
    Returns a [Ns, np, m], b [Ns, np, m, m] (zero below the diagonal),
    VL [np, m], Vbar [np, m, m] (zero below the diagonal) and
    V_l = (s_j - s_i)^2 Vbar (Eq. (sampled_prod)).
    """
    v = int(np.prod(dims))
    if solver is None:
        solver = make_solver(u, m, dims, bc_t)
    ms = len(s_hat)
    npl = len(p_list)
    a = np.zeros((n_s, npl, ms), dtype=np.complex128)
    b = np.zeros((n_s, npl, ms, ms), dtype=np.complex128)
    for k in range(n_s):
        z = philox.z4_noise(v, seed, job, philox.VARIANCE_SAMPLE_LEVEL, k)
        xs = [solver(z, s) for s in s_hat]
        ys = [adjoint_solution(solver, z, s) for s in s_hat]
        for pi, p in enumerate(p_list):
            for i in range(ms):
                a[k, pi, i] = contract(u, z, xs[i], gamma, p, dims)
                for j in range(i, ms):
                    b[k, pi, i, j] = contract(u, ys[i], xs[j], gamma, p, dims)
    VL = practical_variance(a)
    Vbar = practical_variance(b)
    iu = np.triu_indices(ms)
    mask = np.zeros((ms, ms), dtype=bool)
    mask[iu] = True
    Vbar = np.where(mask[None], Vbar, 0.0)
    sh = np.asarray(s_hat, dtype=np.float64)
    Vl = (sh[None, None, :] - sh[None, :, None]) ** 2 * Vbar
    return {"a": a, "b": b, "VL": VL, "Vbar": Vbar, "Vl": Vl}


# ---- exact (dense) counterparts, tiny lattices only ----

def exact_level_matrices(u, m, sigmas, gamma, p, dims, bc_t=-1, estimator=DIFF):
    """Dense matrices A_l whose Z4 Hutchinson estimator is the level-l sample."""
    inv = [solve.dense_inverse(u, m, s, dims, bc_t) for s in sigmas]
    go = solve.dense_GammaOmega(u, gamma, p, dims)
    L = len(sigmas) - 1
    mats = []
    for lev in range(L):
        ds = sigmas[lev + 1] - sigmas[lev]
        if estimator == DIFF:
            mats.append(go @ (inv[lev] - inv[lev + 1]))
        elif estimator == SPLIT_EVEN:
            mats.append(ds * inv[lev] @ go @ inv[lev + 1])
        else:
            mats.append(ds * go @ inv[lev] @ inv[lev + 1])
    mats.append(go @ inv[L])
    return mats
