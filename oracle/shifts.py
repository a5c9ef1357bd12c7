"""Shift selection and MLMC sample allocation (test infrastructure: the oracle).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module; the
library's own implementation (fs_shifts.cu) shares no code with it.

Follows the paper, Sec. 3 (Methods):
  * Sec. 3.2 Interpolation: the sampled variances V_L(s^_i) and Vbar_l(s^_i, s^_j) are
    interpolated in log space with piecewise cubic Hermite interpolating polynomials
    (PCHIP, Fritsch & Carlson 1980), linear where only two points exist; the 2-D manifold
    of Vbar_l follows the three stages of the interpolation algorithm (figure "boundary"):
    fixed sampled second shift, the diagonal, then fixed evaluation first shift.
  * Eq. (solver_cost_shift) with next-neighbour interpolation of the iteration counts.
  * Eq. (ml_cost_shifts) and Eq. (opt_shifts): the optimal shifts minimise
    C_FS = eps^-2 (sum_l sqrt(C_l V_l))^2 over all choices of L evaluation shifts after
    sigma_0 = s_0 (brute force over all combinations, as the paper does). The paper has
    s_0 = 0; with a positive first sampling shift (sigma_0 = the first listed shift) the
    evaluation set starts at that shift instead.
  * Eq. (num_samples) and Eq. (total_var): N_l = mu sqrt(V_l / C_l),
    mu = eps^-2 sum_l sqrt(V_l C_l), V_FS = sum_l V_l / N_l.

Readings (where the paper is silent or garbled):
  * stage 3 of the 2-D interpolation uses, for a fixed first shift s_i, the diagonal value
    Vbar(s_i, s_i) and the stage-1 values Vbar(s_i, s^_j) at the sampled s^_j > s_i (the
    prose of Sec. 3.2); V_l(s_i, s_k) = (s_k - s_i)^2 Vbar(s_i, s_k) for s_k > s_i only;
  * the level cost is the iteration count of the level's solves: C_l = r(sigma_l) +
    r(sigma_{l+1}) for l < L (x at sigma_{l+1} and y at sigma_l), C_L = r(sigma_L); the
    common factor 12c of Eq. (solver_cost_shift) does not move the argmin and is omitted;
  * r(s) = r(s^_j) for s^_{j-1} < s <= s^_j ("s^+j" read as s^_j), r(s^_0) at s = s^_0;
  * variances are floored at 1e-300 before the logarithm.
"""

import itertools
import math

import numpy as np

VAR_FLOOR = 1e-300


# ---------------------------------------------------------------- PCHIP
def pchip_slopes(x, y):
    """Node derivatives of the shape-preserving piecewise cubic Hermite interpolant.

    Interior nodes: 0 where the neighbouring secants change sign or vanish, else the
    weighted harmonic mean of the secants (Fritsch & Butland 1984, the weights
    w1 = 2 h_k + h_{k-1}, w2 = h_k + 2 h_{k-1}). End nodes: the one-sided three-point
    formula, set to 0 if its sign differs from the first secant, and limited to three
    times that secant if the secants change sign (Moler, Numerical Computing with MATLAB)."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    n = len(x)
    h = np.diff(x)
    delta = np.diff(y) / h
    d = np.zeros(n)
    if n == 2:
        d[:] = delta[0]
        return d
    for k in range(1, n - 1):
        if delta[k - 1] * delta[k] > 0:
            w1 = 2 * h[k] + h[k - 1]
            w2 = h[k] + 2 * h[k - 1]
            d[k] = (w1 + w2) / (w1 / delta[k - 1] + w2 / delta[k])
        else:
            d[k] = 0.0

    def end(h0, h1, del0, del1):
        e = ((2 * h0 + h1) * del0 - h0 * del1) / (h0 + h1)
        if np.sign(e) != np.sign(del0):
            return 0.0
        if np.sign(del0) != np.sign(del1) and abs(e) > abs(3 * del0):
            return 3 * del0
        return e

    d[0] = end(h[0], h[1], delta[0], delta[1])
    d[-1] = end(h[-1], h[-2], delta[-1], delta[-2])
    return d


def interpolate(x, y, xq):
    """The paper's "Interpolate": PCHIP through (x, y), linear when only two points exist;
    evaluated at xq (the end polynomials extend beyond [x_0, x_{n-1}])."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    xq = np.atleast_1d(np.asarray(xq, dtype=float))
    if len(x) < 2:
        raise ValueError("at least two points are needed")
    if len(x) == 2:
        return y[0] + (y[1] - y[0]) * (xq - x[0]) / (x[1] - x[0])
    d = pchip_slopes(x, y)
    k = np.clip(np.searchsorted(x, xq, side="right") - 1, 0, len(x) - 2)
    h = x[k + 1] - x[k]
    t = (xq - x[k]) / h
    h00 = 2 * t**3 - 3 * t**2 + 1
    h10 = t**3 - 2 * t**2 + t
    h01 = -2 * t**3 + 3 * t**2
    h11 = t**3 - t**2
    return h00 * y[k] + h10 * h * d[k] + h01 * y[k + 1] + h11 * h * d[k + 1]


# ---------------------------------------------------------------- variance manifolds
def interp_single(s_hat, VL_hat, s):
    """V_L(s_k) = exp(q(s_k)), q = Interpolate(s^, ln V_L(s^))."""
    w = np.log(np.maximum(np.asarray(VL_hat, dtype=float), VAR_FLOOR))
    return np.exp(interpolate(s_hat, w, s))


def interp_pair(s_hat, Vbar_hat, s):
    """Predicted V_l(s_i, s_k) for s_k > s_i (NaN elsewhere) from the sampled
    Vbar_l(s^_i, s^_j), j >= i, in the three stages of the interpolation algorithm."""
    s_hat = np.asarray(s_hat, dtype=float)
    s = np.asarray(s, dtype=float)
    m, n = len(s_hat), len(s)
    lv = np.log(np.maximum(np.asarray(Vbar_hat, dtype=float), VAR_FLOOR))
    # stage 1: for each sampled second shift s^_j, interpolate over the first shift
    stage1 = np.full((n, m), np.nan)  # ln Vbar(s_k, s^_j)
    for j in range(1, m):
        stage1[:, j] = interpolate(s_hat[: j + 1], lv[: j + 1, j], s)
    # stage 2: the diagonal
    diag = interpolate(s_hat, np.diag(lv), s)  # ln Vbar(s_k, s_k)
    # stage 3: for each evaluation first shift s_i, interpolate over the second shift
    V = np.full((n, n), np.nan)
    for i in range(n):
        xs = [s[i]]
        ws = [diag[i]]
        for j in range(1, m):
            if s_hat[j] > s[i]:
                xs.append(s_hat[j])
                ws.append(stage1[i, j])
        if len(xs) < 2:
            continue  # s_i at or beyond the largest sampled shift: no s_k > s_i to predict
        for k in range(i + 1, n):
            V[i, k] = (s[k] - s[i]) ** 2 * math.exp(float(interpolate(xs, ws, [s[k]])[0]))
    return V


def iteration_cost(s_hat, r_hat, s):
    """r(s) = r(s^_j) with s^_{j-1} < s <= s^_j (next-neighbour from above)."""
    s_hat = np.asarray(s_hat, dtype=float)
    out = np.empty(len(s))
    for k, sk in enumerate(s):
        j = int(np.searchsorted(s_hat, sk, side="left"))
        out[k] = r_hat[min(j, len(s_hat) - 1)]
    return out


# ---------------------------------------------------------------- selection
def level_terms(idx, VL, Vl, r):
    """Per-level (V_l, C_l) of the shift indices idx (idx[0] = 0)."""
    L = len(idx) - 1
    V, C = [], []
    for l in range(L):
        a, b = idx[l], idx[l + 1]
        V.append(Vl[a, b])
        C.append(r[a] + r[b])
    V.append(VL[idx[L]])
    C.append(r[idx[L]])
    return np.array(V), np.array(C)


def select_shifts(s_hat, VL_hat, Vbar_hat, r_hat, s, L):
    """Eq. (opt_shifts): brute force over 1 <= j_1 < ... < j_L <= n-1 (sigma_0 = s_0 = s^_0).
    Returns (idx, F) with F = sum_l sqrt(C_l V_l) (C_FS = eps^-2 F^2)."""
    s = np.asarray(s, dtype=float)
    if s[0] != s_hat[0]:
        raise ValueError("the evaluation set starts at sigma_0 = s^_0")
    VL = interp_single(s_hat, VL_hat, s)
    Vl = interp_pair(s_hat, Vbar_hat, s)
    r = iteration_cost(s_hat, r_hat, s)
    best, best_idx = math.inf, None
    for comb in itertools.combinations(range(1, len(s)), L):
        idx = (0,) + comb
        V, C = level_terms(idx, VL, Vl, r)
        if np.any(np.isnan(V)):
            continue
        F = float(np.sum(np.sqrt(C * V)))
        if F < best:
            best, best_idx = F, idx
    return list(best_idx), best


def sample_allocation(V, C, eps2):
    """Eq. (num_samples), Eq. (total_var): N_l = mu sqrt(V_l / C_l), mu = eps^-2 sum sqrt(V_l C_l);
    returns (N, mu, V_FS, C_FS) with the continuous (unrounded) N_l."""
    V = np.asarray(V, dtype=float)
    C = np.asarray(C, dtype=float)
    mu = float(np.sum(np.sqrt(V * C))) / eps2
    N = mu * np.sqrt(V / C)
    V_FS = float(np.sum(V / N))
    C_FS = float(np.sum(N * C))
    return N, mu, V_FS, C_FS


def paper_evaluation_set(s_hat):
    """Sec. 3.3: [logspace(-5,-2,4) logspace(log10(1e-2+1e-3),0,76)] with the sampling shifts
    added; it contains the sampling set and starts at sigma_0 = s^_0 (0 in the paper)."""
    s_hat = np.asarray(s_hat, dtype=float)
    grid = np.concatenate([np.logspace(-5, -2, 4), np.logspace(np.log10(1e-2 + 1e-3), 0, 76)])
    return np.unique(np.concatenate([s_hat, grid[grid >= s_hat[0]]]))
