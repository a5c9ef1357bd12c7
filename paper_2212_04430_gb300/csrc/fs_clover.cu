// Clover table of a gauge field: the field strength from the clover leaves, the two chiral 6x6
// blocks of C(x), and their eigen-decomposition (fs_clover.cuh describes the operator and layout).
#include <algorithm>
#include <cmath>
#include <vector>

#include "fs_engine.h"

namespace fs {

namespace {

// 3x3 complex matrices, row-major
struct M3 {
  double r[9], i[9];
};

__device__ __forceinline__ M3 load_u(const double* gauge, const Geom& g, int mu, const int (&y)[4]) {
  const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  const double* p = gauge + ((size_t)(par * 4 + mu) * g.Vh + cb_index(g, y)) * 18;
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    m.r[k] = p[2 * k];
    m.i[k] = p[2 * k + 1];
  }
  return m;
}

__device__ __forceinline__ M3 dag(const M3& a) {
  M3 d;
#pragma unroll
  for (int x = 0; x < 3; x++)
#pragma unroll
    for (int y = 0; y < 3; y++) {
      d.r[x * 3 + y] = a.r[y * 3 + x];
      d.i[x * 3 + y] = -a.i[y * 3 + x];
    }
  return d;
}

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int x = 0; x < 3; x++)
#pragma unroll
    for (int y = 0; y < 3; y++) {
      double re = 0, im = 0;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        re += a.r[x * 3 + k] * b.r[k * 3 + y] - a.i[x * 3 + k] * b.i[k * 3 + y];
        im += a.r[x * 3 + k] * b.i[k * 3 + y] + a.i[x * 3 + k] * b.r[k * 3 + y];
      }
      c.r[x * 3 + y] = re;
      c.i[x * 3 + y] = im;
    }
  return c;
}

__device__ __forceinline__ void step(int (&y)[4], const Geom& g, int mu, int s) {
  y[mu] = (y[mu] + s + g.L[mu]) % g.L[mu];
}

// Q_{mu nu}(x): the four counter-clockwise plaquettes of the (mu, nu) plane that touch x
__device__ M3 leaves(const double* gauge, const Geom& g, const int (&x)[4], int mu, int nu) {
  int y[4];
  auto at = [&](int dm, int dn) {
    for (int k = 0; k < 4; k++) y[k] = x[k];
    if (dm) step(y, g, mu, dm);
    if (dn) step(y, g, nu, dn);
  };
  at(0, 0); const M3 um_x = load_u(gauge, g, mu, y), un_x = load_u(gauge, g, nu, y);
  at(1, 0); const M3 un_xpm = load_u(gauge, g, nu, y);
  at(0, 1); const M3 um_xpn = load_u(gauge, g, mu, y);
  at(-1, 1); const M3 um_xpnmm = load_u(gauge, g, mu, y);
  at(-1, 0); const M3 un_xmm = load_u(gauge, g, nu, y), um_xmm = load_u(gauge, g, mu, y);
  at(-1, -1); const M3 un_xmmmn = load_u(gauge, g, nu, y), um_xmmmn = load_u(gauge, g, mu, y);
  at(0, -1); const M3 un_xmn = load_u(gauge, g, nu, y), um_xmn = load_u(gauge, g, mu, y);
  at(1, -1); const M3 un_xpmmn = load_u(gauge, g, nu, y);
  const M3 l1 = mul(mul(mul(um_x, un_xpm), dag(um_xpn)), dag(un_x));
  const M3 l2 = mul(mul(mul(un_x, dag(um_xpnmm)), dag(un_xmm)), um_xmm);
  const M3 l3 = mul(mul(mul(dag(um_xmm), dag(un_xmmmn)), um_xmmmn), un_xmn);
  const M3 l4 = mul(mul(mul(dag(un_xmn), um_xmn), un_xpmmn), dag(um_x));
  M3 q;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    q.r[k] = l1.r[k] + l2.r[k] + l3.r[k] + l4.r[k];
    q.i[k] = l1.i[k] + l2.i[k] + l3.i[k] + l4.i[k];
  }
  return q;
}

// Cyclic Jacobi for a Hermitian 6x6 matrix (ar + i ai): on return a is diagonal (lam), and the
// columns of v are the eigenvectors, a = v diag(lam) v^dag. Each rotation acts on a pair (p, q):
// with h = a_pq = t e^{i phi}, J = diag(1, e^{-i phi}) R(theta) in that plane zeroes a_pq, theta
// from the smaller root tau = tan theta of tau^2 + 2 zeta tau - 1 = 0, zeta = (a_pp - a_qq) / (2t)
// (the (p, q) entry of R^T [[a_pp, t], [t, a_qq]] R, R = [[c, -s], [s, c]], is
// t (c^2 - s^2) + c s (a_qq - a_pp)).
// Sweeps stop when the off-diagonal part has fallen below 1e-30 of the diagonal (at most 40).
__device__ void jacobi6(double (&ar)[36], double (&ai)[36], double (&vr)[36], double (&vi)[36], double (&lam)[6]) {
  for (int k = 0; k < 36; k++) {
    vr[k] = (k % 7 == 0) ? 1.0 : 0.0;
    vi[k] = 0.0;
  }
  for (int sweep = 0; sweep < 40; sweep++) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < 6; p++) {
      dia += ar[p * 7] * ar[p * 7];
      for (int q = p + 1; q < 6; q++) off += ar[p * 6 + q] * ar[p * 6 + q] + ai[p * 6 + q] * ai[p * 6 + q];
    }
    if (off <= 1e-30 * dia || off == 0.0) break;
    for (int p = 0; p < 5; p++)
      for (int q = p + 1; q < 6; q++) {
        const double hr = ar[p * 6 + q], hi = ai[p * 6 + q];
        const double t = sqrt(hr * hr + hi * hi);
        if (t == 0.0) continue;
        const double zeta = (ar[p * 7] - ar[q * 7]) / (2.0 * t);
        const double tau = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + tau * tau), s = tau * c;
        const double er = hr / t, ei = -hi / t;  // e = e^{-i phi} = conj(h) / t
        // columns: A' = A J, J = [[c, -s], [s e, c e]]
        for (int k = 0; k < 6; k++) {
          const double pr = ar[k * 6 + p], pi = ai[k * 6 + p], qr = ar[k * 6 + q], qi = ai[k * 6 + q];
          const double eqr = er * qr - ei * qi, eqi = er * qi + ei * qr;  // e a_kq
          ar[k * 6 + p] = c * pr + s * eqr;
          ai[k * 6 + p] = c * pi + s * eqi;
          ar[k * 6 + q] = -s * pr + c * eqr;
          ai[k * 6 + q] = -s * pi + c * eqi;
          const double vpr = vr[k * 6 + p], vpi = vi[k * 6 + p], vqr = vr[k * 6 + q], vqi = vi[k * 6 + q];
          const double evr = er * vqr - ei * vqi, evi = er * vqi + ei * vqr;
          vr[k * 6 + p] = c * vpr + s * evr;
          vi[k * 6 + p] = c * vpi + s * evi;
          vr[k * 6 + q] = -s * vpr + c * evr;
          vi[k * 6 + q] = -s * vpi + c * evi;
        }
        // rows: A'' = J^dag A', J^dag = [[c, s conj(e)], [-s, c conj(e)]]
        for (int k = 0; k < 6; k++) {
          const double pr = ar[p * 6 + k], pi = ai[p * 6 + k], qr = ar[q * 6 + k], qi = ai[q * 6 + k];
          const double eqr = er * qr + ei * qi, eqi = er * qi - ei * qr;  // conj(e) a_qk
          ar[p * 6 + k] = c * pr + s * eqr;
          ai[p * 6 + k] = c * pi + s * eqi;
          ar[q * 6 + k] = -s * pr + c * eqr;
          ai[q * 6 + k] = -s * pi + c * eqi;
        }
        ar[p * 6 + q] = ai[p * 6 + q] = ar[q * 6 + p] = ai[q * 6 + p] = 0.0;
        ai[p * 7] = ai[q * 7] = 0.0;
      }
  }
  for (int p = 0; p < 6; p++) lam[p] = ar[p * 7];
}

struct ClovBuild {
  const double* gauge;   // FP64 links [2][4][Vh][18]
  double* t64;           // [2][Vh][2][CLV_REALS]
  float* t32;
  Geom g;
  double sig[6][2][8];   // sigma_{mu nu} blocks per plane (01, 02, 03, 12, 13, 23) and chirality,
                         // 2x2 complex [s][t][re, im], times c_sw / 2
};

// one thread per (parity, site)
__global__ void __launch_bounds__(64) clover_build_kernel(ClovBuild b) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= 2 * b.g.Vh) return;
  const int parity = id / b.g.Vh, site = id - parity * b.g.Vh;
  int x[4];
  cb_coords(b.g, parity, site, x);
  double cr[2][36], ci[2][36];
  for (int k = 0; k < 36; k++) cr[0][k] = ci[0][k] = cr[1][k] = ci[1][k] = 0.0;
  int plane = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++, plane++) {
      const M3 q = leaves(b.gauge, b.g, x, mu, nu);
      // F = (Q - Q^dag) / (8 i): with D = Q - Q^dag, F = -i D / 8
      double fr[9], fi[9];
      for (int a = 0; a < 3; a++)
        for (int c = 0; c < 3; c++) {
          const double dr = q.r[a * 3 + c] - q.r[c * 3 + a], di = q.i[a * 3 + c] + q.i[c * 3 + a];
          fr[a * 3 + c] = di / 8.0;
          fi[a * 3 + c] = -dr / 8.0;
        }
      // C_b[(s, a), (t, c)] += sigma_b[s][t] F[a][c]
      for (int blk = 0; blk < 2; blk++)
        for (int s = 0; s < 2; s++)
          for (int t = 0; t < 2; t++) {
            const double sr = b.sig[plane][blk][(s * 2 + t) * 2], si = b.sig[plane][blk][(s * 2 + t) * 2 + 1];
            if (sr == 0.0 && si == 0.0) continue;
            for (int a = 0; a < 3; a++)
              for (int c = 0; c < 3; c++) {
                const int k = (s * 3 + a) * 6 + t * 3 + c;
                cr[blk][k] += sr * fr[a * 3 + c] - si * fi[a * 3 + c];
                ci[blk][k] += sr * fi[a * 3 + c] + si * fr[a * 3 + c];
              }
          }
    }
  for (int blk = 0; blk < 2; blk++) {
    const size_t o = ((size_t)id * 2 + blk) * CLV_REALS;
    // packed C (before the rotations overwrite it): diagonal, then the entries above it
    for (int i = 0; i < 6; i++) {
      b.t64[o + CLV_C + i] = cr[blk][i * 7];
      b.t32[o + CLV_C + i] = (float)cr[blk][i * 7];
      for (int j = i + 1; j < 6; j++) {
        const size_t u = o + CLV_C + 6 + 2 * clv_upper(i, j);
        b.t64[u] = cr[blk][i * 6 + j];
        b.t64[u + 1] = ci[blk][i * 6 + j];
        b.t32[u] = (float)cr[blk][i * 6 + j];
        b.t32[u + 1] = (float)ci[blk][i * 6 + j];
      }
    }
    double vr[36], vi[36], lam[6];
    jacobi6(cr[blk], ci[blk], vr, vi, lam);
    for (int k = 0; k < 36; k++) {
      b.t64[o + 2 * k] = vr[k];
      b.t64[o + 2 * k + 1] = vi[k];
      b.t32[o + 2 * k] = (float)vr[k];
      b.t32[o + 2 * k + 1] = (float)vi[k];
    }
    for (int j = 0; j < 6; j++) {
      b.t64[o + 72 + j] = lam[j];
      b.t32[o + 72 + j] = (float)lam[j];
    }
  }
}

// G_mu: the upper-right 2x2 block of gamma_mu = [[0, G_mu], [G_mu^dag, 0]] (DeGrand-Rossi)
void g_block(int mu, double (&re)[4], double (&im)[4]) {
  for (int k = 0; k < 4; k++) re[k] = im[k] = 0.0;
  if (mu == 0) { im[1] = 1; im[2] = 1; }        // [[0, i], [i, 0]]
  else if (mu == 1) { re[1] = -1; re[2] = 1; }  // [[0, -1], [1, 0]]
  else if (mu == 2) { im[0] = 1; im[3] = -1; }  // diag(i, -i)
  else { re[0] = 1; re[3] = 1; }                // 1
}

// 2x2 complex products: out = A B (adjA / adjB: take the adjoint of that factor first)
void mul2(const double (&ar)[4], const double (&ai)[4], bool adjA, const double (&br)[4], const double (&bi)[4],
          bool adjB, double (&cr)[4], double (&ci)[4]) {
  for (int s = 0; s < 2; s++)
    for (int t = 0; t < 2; t++) {
      double re = 0, im = 0;
      for (int k = 0; k < 2; k++) {
        const double xr = adjA ? ar[k * 2 + s] : ar[s * 2 + k], xi = adjA ? -ai[k * 2 + s] : ai[s * 2 + k];
        const double yr = adjB ? br[t * 2 + k] : br[k * 2 + t], yi = adjB ? -bi[t * 2 + k] : bi[k * 2 + t];
        re += xr * yr - xi * yi;
        im += xr * yi + xi * yr;
      }
      cr[s * 2 + t] = re;
      ci[s * 2 + t] = im;
    }
}

// The packed (A + C_b)^-1 of one shift, from the eigen-decomposition: P_ij = sum_k V_ik conj(V_jk) /
// (A + lambda_k), i <= j; one thread per (parity, site), FP64, stored in FP64 and FP32.
__global__ void __launch_bounds__(128) clover_inverse_kernel(const double* __restrict__ eig, double* o64, float* o32,
                                                             int n2, double A) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n2) return;
  for (int b = 0; b < 2; b++) {
    const double* t = eig + ((size_t)id * 2 + b) * CLV_REALS;
    double f[6];
    for (int k = 0; k < 6; k++) f[k] = 1.0 / (A + t[72 + k]);
    double* d64 = o64 + ((size_t)id * 2 + b) * CLV_PACKED;
    float* d32 = o32 + ((size_t)id * 2 + b) * CLV_PACKED;
    for (int i = 0; i < 6; i++)
      for (int j = i; j < 6; j++) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < 6; k++) {
          // V_ik conj(V_jk) f_k
          const double ar = t[2 * (i * 6 + k)], ai = t[2 * (i * 6 + k) + 1];
          const double br = t[2 * (j * 6 + k)], bi = t[2 * (j * 6 + k) + 1];
          re += (ar * br + ai * bi) * f[k];
          im += (ai * br - ar * bi) * f[k];
        }
        if (i == j) {
          d64[i] = re;
          d32[i] = (float)re;
        } else {
          const int u = 6 + 2 * clv_upper(i, j);
          d64[u] = re;
          d64[u + 1] = im;
          d32[u] = (float)re;
          d32[u + 1] = (float)im;
        }
      }
  }
}

}  // namespace

void clover_inverses_free(Ctx* c) {
  const size_t n = (size_t)2 * c->g.Vh * 2 * CLV_PACKED;
  for (auto& kv : c->clv_inv) {
    cudaFree(kv.second.t64);
    cudaFree(kv.second.t32);
    c->extra_bytes -= n * (sizeof(double) + sizeof(float));
  }
  c->clv_inv.clear();
}

int clover_inverses(Ctx* c, double m, const double* sigma, int n, SolveOpts& o) {
  o.clv_inv = nullptr;
  if (c->c_sw == 0.0 || c->clover64 == nullptr) return 0;
  if (c->shared) return c->fail(1, "a lane takes its owner's clover inverses");
  std::vector<double> want;
  for (int k = 0; k < n; k++) want.push_back(4.0 + m + sigma[k]);  // the A of init_state, bit for bit
  constexpr size_t MAX_SHIFTS = 32;
  if (c->clv_inv.size() + want.size() > MAX_SHIFTS) {
    // drop the entries this call does not name (no kernel reads them between calls)
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) return c->cuda_fail(e, "clover inverses");
    const size_t bytes = (size_t)2 * c->g.Vh * 2 * CLV_PACKED * (sizeof(double) + sizeof(float));
    for (auto it = c->clv_inv.begin(); it != c->clv_inv.end();) {
      if (std::find(want.begin(), want.end(), it->first) == want.end()) {
        cudaFree(it->second.t64);
        cudaFree(it->second.t32);
        c->extra_bytes -= bytes;
        it = c->clv_inv.erase(it);
      } else {
        ++it;
      }
    }
  }
  const size_t cnt = (size_t)2 * c->g.Vh * 2 * CLV_PACKED;
  const int n2 = 2 * c->g.Vh;
  // every shift the call names gets its table (the paired pass relies on it: a system without
  // one would take its partner's), however many; only the kept tables of other calls are capped
  for (double A : want) {
    if (c->clv_inv.count(A)) continue;
    ClvInv t;
    if (cudaMalloc(&t.t64, cnt * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return c->fail(3, "device allocation of a clover inverse failed");
    }
    if (cudaMalloc(&t.t32, cnt * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(t.t64);
      return c->fail(3, "device allocation of a clover inverse failed");
    }
    c->extra_bytes += cnt * (sizeof(double) + sizeof(float));
    clover_inverse_kernel<<<(n2 + 127) / 128, 128, 0, c->stream>>>(c->clover64, t.t64, t.t32, n2, A);
    note_launch();
    if (cudaError_t e = cudaGetLastError()) {
      cudaFree(t.t64);
      cudaFree(t.t32);
      c->extra_bytes -= cnt * (sizeof(double) + sizeof(float));
      return c->cuda_fail(e, "clover inverse");
    }
    c->clv_inv[A] = t;
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);  // the lanes read them on their own streams
  if (e) return c->cuda_fail(e, "clover inverses");
  o.clv_inv = &c->clv_inv;
  return 0;
}

int clover_build(Ctx* c, double c_sw) {
  if (cudaError_t e = cudaStreamSynchronize(c->stream)) return c->cuda_fail(e, "clover table");
  clover_inverses_free(c);  // they belong to the old table
  const size_t n = (size_t)2 * c->g.Vh * 2 * CLV_REALS;
  if (!c->clover64) {
    if (cudaMalloc(&c->clover64, n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->clover64 = nullptr;
      return c->fail(3, "device allocation of the clover table failed");
    }
    if (cudaMalloc(&c->clover32, n * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->clover64);
      c->clover64 = nullptr;
      c->clover32 = nullptr;
      return c->fail(3, "device allocation of the clover table failed");
    }
    c->extra_bytes += n * (sizeof(double) + sizeof(float));
  }
  ClovBuild b{};
  b.gauge = (const double*)c->gauge64;
  b.t64 = c->clover64;
  b.t32 = c->clover32;
  b.g = c->g;
  // sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu] = diag((i/2)(G_mu G_nu^dag - G_nu G_mu^dag),
  //                                                  (i/2)(G_mu^dag G_nu - G_nu^dag G_mu)), times c_sw / 2
  int plane = 0;
  for (int mu = 0; mu < 4; mu++)
    for (int nu = mu + 1; nu < 4; nu++, plane++) {
      double gmr[4], gmi[4], gnr[4], gni[4];
      g_block(mu, gmr, gmi);
      g_block(nu, gnr, gni);
      for (int blk = 0; blk < 2; blk++) {
        double ar[4], ai[4], br[4], bi[4];
        if (blk == 0) {
          mul2(gmr, gmi, false, gnr, gni, true, ar, ai);
          mul2(gnr, gni, false, gmr, gmi, true, br, bi);
        } else {
          mul2(gmr, gmi, true, gnr, gni, false, ar, ai);
          mul2(gnr, gni, true, gmr, gmi, false, br, bi);
        }
        for (int k = 0; k < 4; k++) {
          // (i/2)(a - b) (c_sw / 2)
          const double dr = ar[k] - br[k], di = ai[k] - bi[k];
          b.sig[plane][blk][2 * k] = -0.5 * di * 0.5 * c_sw;
          b.sig[plane][blk][2 * k + 1] = 0.5 * dr * 0.5 * c_sw;
        }
      }
    }
  const int threads = 64;
  const int blocks = (int)((2 * (size_t)c->g.Vh + threads - 1) / threads);
  clover_build_kernel<<<blocks, threads, 0, c->stream>>>(b);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return c->cuda_fail(e, "clover table");
  c->c_sw = c_sw;
  return 0;
}

}  // namespace fs
