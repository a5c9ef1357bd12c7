// Shift selection and MLMC sample allocation (host code; paper Sec. 3.2-3.3).
//
// From the variances sampled by variance_sample (V_L at the m sampling shifts, Vbar_l at
// every pair s^_i <= s^_j) and the iteration counts at the sampling shifts, predict V_L,
// V_l and the solver cost on an evaluation set s that starts at the first sampling shift
// (s_0 = s^_0; 0 in the paper, whose sigma_0 = 0), then choose the L shifts after
// sigma_0 = s_0 that minimise the multilevel cost, Eq. (ml_cost_shifts),
//   C_FS = eps^-2 F^2,  F = sum_l sqrt(C_l V_l),
// and the per-level sample counts N_l = mu sqrt(V_l / C_l), Eq. (num_samples).
//
// Interpolation (Sec. 3.2): in log space, shape-preserving piecewise cubic Hermite
// (Fritsch-Carlson monotone cubics with the Fritsch-Butland weighted-harmonic-mean node
// slopes and one-sided three-point end slopes), linear through two points. The 2-D
// manifold Vbar(a, b), a <= b, is built in three stages: (1) for each sampled b = s^_j,
// along a over s^_0..s^_j; (2) along the diagonal a = b; (3) for each evaluation a = s_i,
// along b through the diagonal value and the stage-1 values at the sampled s^_j > s_i.
// V_l(s_i, s_k) = (s_k - s_i)^2 Vbar(s_i, s_k) for s_k > s_i.
//
// Costs: r(s) = r(s^_j) for s^_{j-1} < s <= s^_j (next neighbour from above); level l < L
// solves at sigma_l and sigma_{l+1}, C_l = r(sigma_l) + r(sigma_{l+1}); C_L = r(sigma_L).
//
// Argmin of Eq. (opt_shifts) over 0 = j_0 < j_1 < ... < j_L <= n-1: F is a sum of terms
// that each depend on consecutive indices, so the exact minimum is a shortest path of L
// steps on the ordered evaluation shifts (dynamic programming, O(L n^2)) instead of the
// paper's enumeration of all C(n-1, L) combinations; both give the same minimiser.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "fsmlmc.h"

namespace {

constexpr double kVarFloor = 1e-300;
const double kNaN = std::numeric_limits<double>::quiet_NaN();

int sgn(double v) { return (v > 0) - (v < 0); }

// Monotone piecewise cubic Hermite interpolant through (x_k, y_k), k < n; linear for n == 2.
struct Pchip {
  std::vector<double> x, y, d;
  Pchip(const double* xs, const double* ys, int n) : x(xs, xs + n), y(ys, ys + n), d(n, 0.0) {
    if (n == 2) {
      d[0] = d[1] = (y[1] - y[0]) / (x[1] - x[0]);
      return;
    }
    std::vector<double> h(n - 1), s(n - 1);
    for (int k = 0; k + 1 < n; k++) {
      h[k] = x[k + 1] - x[k];
      s[k] = (y[k + 1] - y[k]) / h[k];
    }
    for (int k = 1; k + 1 < n; k++) {
      if (s[k - 1] * s[k] <= 0.0) continue;  // local extremum or flat: zero slope
      const double a = 2.0 * h[k] + h[k - 1], b = h[k] + 2.0 * h[k - 1];
      d[k] = (a + b) / (a / s[k - 1] + b / s[k]);
    }
    auto end_slope = [](double h0, double h1, double s0, double s1) {
      double e = ((2.0 * h0 + h1) * s0 - h0 * s1) / (h0 + h1);
      if (sgn(e) != sgn(s0)) e = 0.0;
      else if (sgn(s0) != sgn(s1) && std::fabs(e) > 3.0 * std::fabs(s0)) e = 3.0 * s0;
      return e;
    };
    d[0] = end_slope(h[0], h[1], s[0], s[1]);
    d[n - 1] = end_slope(h[n - 2], h[n - 3], s[n - 2], s[n - 3]);
  }
  // the end cubics continue beyond [x_0, x_{n-1}]
  double operator()(double q) const {
    const int n = (int)x.size();
    int k = (int)(std::upper_bound(x.begin(), x.end(), q) - x.begin()) - 1;
    k = std::min(std::max(k, 0), n - 2);
    const double h = x[k + 1] - x[k], t = (q - x[k]) / h;
    const double t2 = t * t, t3 = t2 * t;
    return (2 * t3 - 3 * t2 + 1) * y[k] + (t3 - 2 * t2 + t) * h * d[k] + (-2 * t3 + 3 * t2) * y[k + 1] +
           (t3 - t2) * h * d[k + 1];
  }
};

double lnv(double v) { return std::log(std::max(v, kVarFloor)); }

bool increasing(const double* v, int n) {
  for (int k = 0; k < n; k++)
    if (!std::isfinite(v[k]) || (k > 0 && !(v[k] > v[k - 1]))) return false;
  return true;
}

int check_inputs(const double* s_hat, int m, const double* VL_hat, const double* Vbar_hat, const double* s,
                 int n) {
  if (!s_hat || !VL_hat || !Vbar_hat || !s || m < 2 || n < 2) return FS_ERR_ARG;
  // sigma_0 is the first sampling shift (0 in the paper), and the evaluation set starts there
  if (!increasing(s_hat, m) || !increasing(s, n) || s[0] != s_hat[0]) return FS_ERR_ARG;
  for (int i = 0; i < m; i++) {
    if (!std::isfinite(VL_hat[i]) || VL_hat[i] < 0.0) return FS_ERR_INPUT;
    for (int j = i; j < m; j++)
      if (!std::isfinite(Vbar_hat[i * m + j]) || Vbar_hat[i * m + j] < 0.0) return FS_ERR_INPUT;
  }
  return FS_OK;
}

// V_L(s_k) and V_l(s_i, s_k) (row-major [n][n], NaN for k <= i or no prediction)
void interpolate_all(const double* s_hat, int m, const double* VL_hat, const double* Vbar_hat, const double* s,
                     int n, std::vector<double>& VL, std::vector<double>& Vl) {
  std::vector<double> w(m);
  for (int i = 0; i < m; i++) w[i] = lnv(VL_hat[i]);
  const Pchip single(s_hat, w.data(), m);
  VL.assign(n, 0.0);
  for (int k = 0; k < n; k++) VL[k] = std::exp(single(s[k]));
  // stage 1: ln Vbar(s_k, s^_j) along the first shift, for each sampled second shift
  std::vector<double> st1((size_t)n * m, kNaN);
  for (int j = 1; j < m; j++) {
    std::vector<double> col(j + 1);
    for (int i = 0; i <= j; i++) col[i] = lnv(Vbar_hat[i * m + j]);
    const Pchip q(s_hat, col.data(), j + 1);
    for (int k = 0; k < n; k++) st1[(size_t)k * m + j] = q(s[k]);
  }
  // stage 2: the diagonal
  for (int i = 0; i < m; i++) w[i] = lnv(Vbar_hat[i * m + i]);
  const Pchip diag(s_hat, w.data(), m);
  // stage 3: along the second shift for each evaluation first shift
  Vl.assign((size_t)n * n, kNaN);
  std::vector<double> xs, ws;
  for (int i = 0; i < n; i++) {
    xs.assign(1, s[i]);
    ws.assign(1, diag(s[i]));
    for (int j = 1; j < m; j++)
      if (s_hat[j] > s[i]) {
        xs.push_back(s_hat[j]);
        ws.push_back(st1[(size_t)i * m + j]);
      }
    if (xs.size() < 2) continue;
    const Pchip q(xs.data(), ws.data(), (int)xs.size());
    for (int k = i + 1; k < n; k++) {
      const double ds = s[k] - s[i];
      Vl[(size_t)i * n + k] = ds * ds * std::exp(q(s[k]));
    }
  }
}

}  // namespace

extern "C" {

int fs_interp_variances(const double* s_hat, int m, const double* VL_hat, const double* Vbar_hat, const double* s,
                        int n, double* VL, double* Vl) {
  if (int rc = check_inputs(s_hat, m, VL_hat, Vbar_hat, s, n)) return rc;
  if (!VL || !Vl) return FS_ERR_ARG;
  std::vector<double> a, b;
  interpolate_all(s_hat, m, VL_hat, Vbar_hat, s, n, a, b);
  std::copy(a.begin(), a.end(), VL);
  std::copy(b.begin(), b.end(), Vl);
  return FS_OK;
}

int fs_select_shifts(const double* s_hat, int m, const double* VL_hat, const double* Vbar_hat,
                     const double* iters_hat, const double* s, int n, int L, int* idx, double* V, double* C,
                     double* F) {
  if (int rc = check_inputs(s_hat, m, VL_hat, Vbar_hat, s, n)) return rc;
  if (!iters_hat || !idx || !V || !C || !F || L < 1 || L > n - 1) return FS_ERR_ARG;
  for (int i = 0; i < m; i++)
    if (!std::isfinite(iters_hat[i]) || iters_hat[i] < 0.0) return FS_ERR_INPUT;
  std::vector<double> VL, Vl;
  interpolate_all(s_hat, m, VL_hat, Vbar_hat, s, n, VL, Vl);
  std::vector<double> r(n);
  for (int k = 0; k < n; k++) {
    const int j = (int)(std::lower_bound(s_hat, s_hat + m, s[k]) - s_hat);
    r[k] = iters_hat[std::min(j, m - 1)];
  }
  // best[l][b]: least sum over the first l levels with sigma_l = s_b; from[l][b]: sigma_{l-1}
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> best((size_t)(L + 1) * n, inf);
  std::vector<int> from((size_t)(L + 1) * n, -1);
  best[0] = 0.0;
  for (int l = 1; l <= L; l++)
    for (int b = l; b < n; b++)
      for (int a = l - 1; a < b; a++) {
        const double pa = best[(size_t)(l - 1) * n + a], v = Vl[(size_t)a * n + b];
        if (!(pa < inf) || std::isnan(v)) continue;
        const double t = pa + std::sqrt((r[a] + r[b]) * v);
        if (t < best[(size_t)l * n + b]) {
          best[(size_t)l * n + b] = t;
          from[(size_t)l * n + b] = a;
        }
      }
  int last = -1;
  double tot = inf;
  for (int b = L; b < n; b++) {
    const double t = best[(size_t)L * n + b] + std::sqrt(r[b] * VL[b]);
    if (t < tot) {
      tot = t;
      last = b;
    }
  }
  if (last < 0) return FS_ERR_ARG;  // no admissible choice of L shifts
  idx[L] = last;
  for (int l = L; l > 0; l--) idx[l - 1] = from[(size_t)l * n + idx[l]];
  for (int l = 0; l < L; l++) {
    V[l] = Vl[(size_t)idx[l] * n + idx[l + 1]];
    C[l] = r[idx[l]] + r[idx[l + 1]];
  }
  V[L] = VL[idx[L]];
  C[L] = r[idx[L]];
  *F = tot;
  return FS_OK;
}

int fs_sample_allocation(const double* V, const double* C, int nlev, double eps2, double* N, double* mu,
                         double* V_FS, double* C_FS) {
  if (!V || !C || !N || nlev < 1 || !(eps2 > 0.0) || !std::isfinite(eps2)) return FS_ERR_ARG;
  double sum = 0.0;
  for (int l = 0; l < nlev; l++) {
    if (!std::isfinite(V[l]) || !std::isfinite(C[l]) || V[l] < 0.0 || !(C[l] > 0.0)) return FS_ERR_INPUT;
    sum += std::sqrt(V[l] * C[l]);
  }
  const double m = sum / eps2;
  double vfs = 0.0, cfs = 0.0;
  for (int l = 0; l < nlev; l++) {
    N[l] = m * std::sqrt(V[l] / C[l]);
    if (N[l] > 0.0) vfs += V[l] / N[l];
    cfs += N[l] * C[l];
  }
  if (mu) *mu = m;
  if (V_FS) *V_FS = vfs;
  if (C_FS) *C_FS = cfs;
  return FS_OK;
}

int fs_trace_total(const double* trace, const double* var, const int* n_samples, int nlev, int np, double* total,
                   double* v_fs) {
  if (!trace || !var || !n_samples || !total || !v_fs || nlev < 1 || np < 1) return FS_ERR_ARG;
  for (int l = 0; l < nlev; l++)
    if (n_samples[l] < 1) return FS_ERR_ARG;
  for (int q = 0; q < np; q++) {
    double tr = 0.0, ti = 0.0, v = 0.0;
    for (int l = 0; l < nlev; l++) {
      const size_t k = (size_t)q * nlev + l;
      if (!std::isfinite(trace[2 * k]) || !std::isfinite(trace[2 * k + 1]) || !std::isfinite(var[k]))
        return FS_ERR_INPUT;
      tr += trace[2 * k];  // Eq. (fs_trace_est): the level estimates add up to the trace
      ti += trace[2 * k + 1];
      v += var[k] / n_samples[l];  // Eq. (total_var): independent levels, V_l / N_l each
    }
    total[2 * q] = tr;
    total[2 * q + 1] = ti;
    v_fs[q] = v;
  }
  return FS_OK;
}

int fs_sampled_level_variances(const double* s_hat, int m, const double* Vbar, int np, double* Vl) {
  if (!s_hat || !Vbar || !Vl || m < 1 || np < 1) return FS_ERR_ARG;
  for (int q = 0; q < np; q++)
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) {
        const size_t k = ((size_t)q * m + i) * m + j;
        if (j < i) {
          Vl[k] = 0.0;
          continue;
        }
        if (!std::isfinite(Vbar[k])) return FS_ERR_INPUT;
        const double ds = s_hat[j] - s_hat[i];
        Vl[k] = ds * ds * Vbar[k];  // Eq. (sampled_prod)
      }
  return FS_OK;
}

int fs_eval_grid(const double* s_hat, int m, double* s, int cap, int* n) {
  if (!s_hat || !n || m < 1 || !increasing(s_hat, m)) return FS_ERR_ARG;
  std::vector<double> v(s_hat, s_hat + m);
  const double lo = std::log10(1e-2 + 1e-3);
  for (int k = 0; k < 80; k++) {
    // logspace(-5, -2, 4), then logspace(lo, 0, 76) with its last point exactly 1
    const double x = k < 4 ? std::pow(10.0, -5.0 + k) : (k == 79 ? 1.0 : std::pow(10.0, lo - lo * (k - 4) / 75.0));
    if (x >= s_hat[0]) v.push_back(x);  // the set starts at sigma_0 = s_hat[0]
  }
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  *n = (int)v.size();
  if (!s) return FS_OK;  // size query
  if (cap < (int)v.size()) return FS_ERR_ARG;
  std::copy(v.begin(), v.end(), s);
  return FS_OK;
}

}  // extern "C"
