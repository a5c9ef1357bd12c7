"""Probing colorings and probed / diluted Z4 noise (test infrastructure: the oracle).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module; the library's
own implementation shares no code with it.

Follows arXiv:2212.04430:
  * Sec. 2.1 (Probing): a distance-k coloring of the graph of A, i.e. a distance-1 coloring
    of A^k, computed greedily; probing vectors z_j(i) = [color(i) = j], Eq. (probing_vectors).
  * Sec. 2.1, displacement-p probing: the coloring of the symmetric part of Pi_p A^k, i.e.
    site x must differ in color from every site within distance k of x + p z and of x - p z.
  * Sec. 2.1: probing vectors combined with random noise are Hutchinson steps on
    Pi_p A^-1 (elementwise) Z Z^T.
  * Sec. 3.1: full spin-color dilution, each noise vector restricted to the sites of one
    color and one spin-color index (12 c inversions per noise vector and shift).

Readings (where the paper is silent):
  * the graph of the Wilson operator links nearest neighbours on the periodic 4D lattice, so
    "distance" is the hop (L1) distance on the torus; the z axis is lattice axis 2;
  * the greedy order is the canonical site order (x fastest, then y, z, t) and each site takes
    the smallest color not used by an already colored site it conflicts with;
  * the pieces of one sample share one underlying Z4 vector and differ only by their masks.
"""

import itertools

import numpy as np

from . import dirac, philox


def _offsets(k):
    """All 4D displacements with 1 <= L1 norm <= k."""
    out = []
    for d in itertools.product(range(-k, k + 1), repeat=4):
        n = sum(abs(c) for c in d)
        if 1 <= n <= k:
            out.append(d)
    return out


def _site(dims, x):
    return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))


def _coords(dims, i):
    x0 = i % dims[0]
    i //= dims[0]
    x1 = i % dims[1]
    i //= dims[1]
    x2 = i % dims[2]
    return (x0, x1, x2, i // dims[2])


def conflicts(dims, k, p=0):
    """conflict[i]: the sites that must not share site i's color (a symmetric relation)."""
    v = int(np.prod(dims))
    offs = _offsets(k)
    if p == 0:
        centres = [(0, 0, 0, 0)]
        shifts = offs
    else:
        # neighbourhoods (distance <= k, centre included) of x + p z and x - p z
        centres = [(0, 0, p, 0), (0, 0, -p, 0)]
        shifts = [(0, 0, 0, 0)] + offs
    out = []
    for i in range(v):
        x = _coords(dims, i)
        s = set()
        for c in centres:
            for d in shifts:
                y = tuple((x[m] + c[m] + d[m]) % dims[m] for m in range(4))
                j = _site(dims, y)
                if j != i:
                    s.add(j)
        out.append(s)
    return out


def greedy_coloring(dims, k, p=0):
    """Distance-k (displacement-p) probing colors, int[V], and the number of colors."""
    conf = conflicts(dims, k, p)
    v = len(conf)
    color = -np.ones(v, dtype=np.int64)
    for i in range(v):
        used = {int(color[j]) for j in conf[i] if color[j] >= 0}
        c = 0
        while c in used:
            c += 1
        color[i] = c
    return color, int(color.max()) + 1


def pieces(ncolors, dilute):
    """(color, spin-color component) of every piece of one sample; None = no restriction."""
    cols = range(ncolors) if ncolors else [None]
    comps = range(12) if dilute else [None]
    return [(j, a) for j in cols for a in comps]


def probed_noise(v, seed, job, level, sample, colors=None, color=None, comp=None, gamma5=False):
    """One piece of a probed / diluted Z4 sample: the sample's Z4 vector on the sites of
    `color` (all sites if None) and the spin-color index `comp` = 3 spin + colour (all if None)."""
    z = philox.z4_noise(v, seed, job, level, sample, gamma5)
    if color is not None:
        z = z * (np.asarray(colors) == color)[:, None, None]
    if comp is not None:
        m = np.zeros((4, 3))
        m[comp // 3, comp % 3] = 1.0
        z = z * m[None]
    return z


def probed_level_samples(u, m, sigmas, gamma, p, n_samples, seed, job, dims, colors, ncolors, dilute,
                         bc_t=-1, estimator=0, solver=None):
    """Per-level samples of Eq. (fs_trace_est) with probed / diluted noise: a sample is the sum
    of the level estimator over all pieces of its Z4 vector."""
    from . import estimators as est
    v = int(np.prod(dims))
    if solver is None:
        solver = est.make_solver(u, m, dims, bc_t)
    out = []
    for lev in range(len(sigmas)):
        vals = []
        for s in range(n_samples[lev]):
            tot = 0j
            for (j, a) in pieces(ncolors, dilute):
                z = probed_noise(v, seed, job, lev, s, colors, j, a)
                tot += est.level_sample(u, solver, z, sigmas, lev, gamma, p, dims, estimator)
            vals.append(tot)
        out.append(np.array(vals, dtype=np.complex128))
    return out


def classes(dims, colors, ncolors, dilute):
    """Index sets (into the flat V*12 vector) of the pieces: the support of each piece."""
    v = int(np.prod(dims))
    idx = np.arange(v * 12).reshape(v, 12)
    out = []
    for (j, a) in pieces(ncolors, dilute):
        site_ok = np.ones(v, dtype=bool) if j is None else (np.asarray(colors) == j)
        comp_ok = np.ones(12, dtype=bool)
        if a is not None:
            comp_ok[:] = False
            comp_ok[a] = True
        out.append(idx[site_ok][:, comp_ok].ravel())
    return out


def exact_mean_and_variance(a, cls):
    """Expectation and variance over Z4 noise of sum_pieces z_piece^dag A z_piece, where the
    pieces restrict one Z4 vector to the disjoint index sets cls. The expectation is
    sum_i A_ii over the union (Tr A when the sets cover everything); the pieces are
    independent and each contributes the off-diagonal squares inside its set."""
    mean = 0j
    var = 0.0
    for c in cls:
        sub = a[np.ix_(c, c)]
        mean += np.trace(sub)
        var += float((np.abs(sub) ** 2).sum() - (np.abs(np.diag(sub)) ** 2).sum())
    return complex(mean), var


def probed_variance_sample(u, m, s_hat, gamma, p_list, n_s, seed, job, dims, colors, ncolors, dilute,
                           bc_t=-1, solver=None):
    """Sec. 3.1 variance sampling with probed / diluted noise: for each noise vector z_k the
    sums over its pieces z_piece of a_i = z_piece^dag Gamma Omega_p x^(i) and
    b_ij = y^(i)^dag Gamma Omega_p x^(j), with x^(i) = (D+s_i)^-1 z_piece and
    y^(i) = (D+s_i)^-dag z_piece (the adjoint solve taken as written, no shortcut), then the
    practical variances of Eq. (practical_variance). Same outputs as
    estimators.variance_sample."""
    from . import estimators as est
    v = int(np.prod(dims))
    if solver is None:
        solver = est.make_solver(u, m, dims, bc_t)
    ms = len(s_hat)
    npl = len(p_list)
    a = np.zeros((n_s, npl, ms), dtype=np.complex128)
    b = np.zeros((n_s, npl, ms, ms), dtype=np.complex128)
    for k in range(n_s):
        for (j, comp) in pieces(ncolors, dilute):
            z = probed_noise(v, seed, job, philox.VARIANCE_SAMPLE_LEVEL, k, colors, j, comp)
            xs = [solver(z, s) for s in s_hat]
            ys = [est.adjoint_solution(solver, z, s) for s in s_hat]
            for pi, p in enumerate(p_list):
                for i in range(ms):
                    a[k, pi, i] += est.contract(u, z, xs[i], gamma, p, dims)
                    for jj in range(i, ms):
                        b[k, pi, i, jj] += est.contract(u, ys[i], xs[jj], gamma, p, dims)
    VL = est.practical_variance(a)
    Vbar = np.where(np.triu(np.ones((ms, ms), dtype=bool))[None], est.practical_variance(b), 0.0)
    sh = np.asarray(s_hat, dtype=np.float64)
    Vl = (sh[None, None, :] - sh[None, :, None]) ** 2 * Vbar
    return {"a": a, "b": b, "VL": VL, "Vbar": Vbar, "Vl": Vl}
