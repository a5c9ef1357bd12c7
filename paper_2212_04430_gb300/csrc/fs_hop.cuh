// Even-odd Wilson hopping kernel over a tile of N systems, with a fused axpy
// epilogue and fused dot-product partials.
//
// Wilson operator (r = 1, DeGrand-Rossi basis, gamma_mu = [[0, G_mu], [G_mu^dag, 0]]):
//   D = (4 + m) - 1/2 H,
//   (H psi)(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu),
// with the t-hop that wraps multiplied by bc_t. The 4x4 projectors have rank 2:
//   (1 + S g_mu) psi = [h; S G^dag h],  h = psi_up + S G psi_dn,
// so each hop is one SU(3) product on a 2-spin half spinor (1320 flop per site).
// The kernel computes, for output parity p and systems selected by `mask`:
//   out = a X + b (H in) + c Y
// with per-system (a, b, c) chosen by COEF from the system's shift, and
// optionally per-system dot partials over fixed 8-site groups (deterministic,
// independent of N and of the other systems in the tile).
#pragma once

#include "fs_common.cuh"

namespace fs {

enum Coef {
  COEF_PLAIN = 0,    // out = H in
  COEF_MHAT = 1,     // out = A X - H in / (4A)            Schur operator M = A - H_eo H_oe / (4A)
  COEF_DSLASH = 2,   // out = A X - H in / 2              (D + sigma) on one parity
  COEF_PREP = 3,     // out = X + H in / (2A)             bhat_e = z_e - D_eo A^-1 z_o
  COEF_RECON = 4,    // out = X / A + H in / (2A)         x_o = A^-1 (z_o - D_oe x_e)
  COEF_TRUERES = 5,  // out = Y - A X + H in / (4A)       r = bhat - M x
  COEF_FULLRES = 6,  // out = Y - A X + H in / 2          r = z - (D + sigma) x on one parity
  COEF_KAPPA = 7,    // out = H in / (2A) = kappa H in     hopping parameter expansion, D + s = A (1 - kappa H)
};

// Dot products a hop kernel forms with its output (out) per (8-site group, system):
//   DOT_R:    <R, out>                                        (out = v, R = rhat)
//   DOT_TS:   <out, X>, ||out||^2, ||X||^2, <R, X>, <R, out>  (out = t, X = s, R = rhat)
//   DOT_NORM: ||out||^2
enum Dot { DOT_NONE = 0, DOT_R = 1, DOT_TS = 2, DOT_NORM = 3 };
template <int DOT> struct DotK { static constexpr int K = 0; };
template <> struct DotK<DOT_R> { static constexpr int K = 2; };
template <> struct DotK<DOT_TS> { static constexpr int K = 8; };
template <> struct DotK<DOT_NORM> { static constexpr int K = 1; };

// The reliable updates of a mixed-precision solve by their index k (SysState::updates): k = 0
// MASK_UPDATE_FIRST, odd k MASK_UPDATE_LATER (full FP64 residual), even k >= 2 MASK_UPDATE_CORR
// (the previous residual corrected by the iterate's change); an update that may end the solve
// (FLAG_CHECK) is MASK_UPDATE_LATER whatever its index
enum Mask { MASK_ALL = 0, MASK_ACTIVE = 1, MASK_UPDATE = 2, MASK_INIT = 3, MASK_HARVEST = 4, MASK_CG = 5,
            MASK_CG_CHECK = 6, MASK_HPE = 7, MASK_UPDATE_FIRST = 8, MASK_UPDATE_LATER = 9,
            MASK_UPDATE_CORR = 10, MASK_HARVEST_HX = 11, MASK_HARVEST_HOP = 12 };

__device__ __forceinline__ bool selected(const SysState* st, int sys, int mask) {
  if (mask == MASK_ALL) return true;
  const int s = st[sys].status, f = st[sys].flags;
  // a system that broke down earlier in this iteration sits out until its restart
  if (mask == MASK_ACTIVE) return s == SYS_ACTIVE && !(f & (FLAG_RESTART | FLAG_CG));
  if (mask == MASK_UPDATE) return s == SYS_ACTIVE && (f & FLAG_UPDATE) && !(f & FLAG_CG);
  if (mask == MASK_UPDATE_FIRST || mask == MASK_UPDATE_LATER || mask == MASK_UPDATE_CORR) {
    if (!(s == SYS_ACTIVE && (f & FLAG_UPDATE) && !(f & FLAG_CG))) return false;
    const int k = st[sys].updates;
    const bool check = (f & FLAG_CHECK) != 0;  // a possible last update: always full FP64
    if (mask == MASK_UPDATE_LATER) return (k & 1) != 0 || check;
    return !check && (mask == MASK_UPDATE_FIRST ? k == 0 : k >= 2 && !(k & 1));
  }
  // CGNR fallback systems, and those of them due a true-residual check
  if (mask == MASK_CG) return s == SYS_ACTIVE && (f & FLAG_CG);
  if (mask == MASK_CG_CHECK) return s == SYS_ACTIVE && (f & FLAG_CG) && (f & FLAG_UPDATE);
  if (mask == MASK_INIT) return (f & FLAG_INIT) != 0;
  if (mask == MASK_HPE) return (f & FLAG_HPE) != 0;
  // harvested systems split by whether H_oe x_e of the final residual is still at hand
  if (mask == MASK_HARVEST_HX) return (f & FLAG_HARVEST) && (f & FLAG_HX);
  if (mask == MASK_HARVEST_HOP) return (f & FLAG_HARVEST) && !(f & FLAG_HX);
  return (f & FLAG_HARVEST) != 0;
}

// Thread/block shape shared by all tile kernels: a block covers SB sites x NB
// systems (sys fastest); grid.y splits the tile's N systems into chunks of NB.
struct Shape {
  int N, NB, SB, nchunk;  // nchunk = ceil(Vh / SB)
};

struct HopArgs {
  void* out;
  const void* in;
  const void* X;
  const void* Y;
  const void* R;
  const void* gauge;
  const SysState* st;
  double* partial;  // [N][K][Vh/8]
  const int* gate;  // kernel returns at once if *gate == 0 (nullptr: always run)
  unsigned long long* work;  // optional: += number of (site, system) pairs computed
  Geom g;
  Shape sh;
  int p_out;
  int mask;
  int sysmajor;  // 1: every field operand in the system-major layout (hop_kernel only)
  int clover;    // 1: the Wilson-clover operator (hop_kernel only; the site terms come from passes)
};

// ---- fixed-order arithmetic ------------------------------------------------------
// Multiply-adds with a fixed rounding sequence (no compiler contraction choices):
// every hop kernel variant forms its products, epilogues and dot products through
// these, so a system's iterates are bit-identical whichever variant (tile shape)
// computed them.
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// (re, im) += conj(a) b for one complex entry a = a0 + i a1, b = b0 + i b1
template <typename Tm>
__device__ __forceinline__ void dot_acc(Tm& re, Tm& im, Tm a0, Tm a1, Tm b0, Tm b1) {
  re = fmadd(a0, b0, re);
  re = fmadd(a1, b1, re);
  im = fmadd(a0, b1, im);
  im = fmadd(-a1, b0, im);
}
template <typename Tm>
__device__ __forceinline__ void norm_acc(Tm& n, Tm a0, Tm a1) {
  n = fmadd(a0, a0, n);
  n = fmadd(a1, a1, n);
}
// a x + b y
template <typename Tm>
__device__ __forceinline__ Tm axpby(Tm a, Tm x, Tm b, Tm y) { return fmadd(b, y, a * x); }

// The DOT_TS values of one site: t = M s, rhat. Each accumulator runs over the
// entries in index order (the chunked persistent kernel keeps the same order).
template <typename Tm>
__device__ __forceinline__ void ts_dots(double (&dv)[8], const Tm (&t)[24], const Tm (&s)[24],
                                        const Tm (&r)[24]) {
  Tm tsr = 0, tsi = 0, tt = 0, ss = 0, rsr = 0, rsi = 0, rtr = 0, rti = 0;
#pragma unroll
  for (int k = 0; k < 24; k += 2) {
    dot_acc(tsr, tsi, t[k], t[k + 1], s[k], s[k + 1]);
    norm_acc(tt, t[k], t[k + 1]);
    norm_acc(ss, s[k], s[k + 1]);
    dot_acc(rsr, rsi, r[k], r[k + 1], s[k], s[k + 1]);
    dot_acc(rtr, rti, r[k], r[k + 1], t[k], t[k + 1]);
  }
  dv[0] = (double)tsr; dv[1] = (double)tsi; dv[2] = (double)tt; dv[3] = (double)ss;
  dv[4] = (double)rsr; dv[5] = (double)rsi; dv[6] = (double)rtr; dv[7] = (double)rti;
}

// ---- links -----------------------------------------------------------------
// Third row of a special unitary matrix from its first two: u2 = conj(u0 x u1),
// in one fixed multiply-add order.
template <typename Tm>
__device__ __forceinline__ void link_row3(Tm (&u)[18]) {
  auto cross = [&](int i, int j, Tm& re, Tm& im) {  // component of u0 x u1: a_i b_j - a_j b_i
    const Tm air = u[2 * i], aii = u[2 * i + 1], ajr = u[2 * j], aji = u[2 * j + 1];
    const Tm bir = u[6 + 2 * i], bii = u[6 + 2 * i + 1], bjr = u[6 + 2 * j], bji = u[6 + 2 * j + 1];
    re = air * bjr;
    re = fmadd(-aii, bji, re);
    re = fmadd(-ajr, bir, re);
    re = fmadd(aji, bii, re);
    im = air * bji;
    im = fmadd(aii, bjr, im);
    im = fmadd(-ajr, bii, im);
    im = fmadd(-aji, bir, im);
  };
  Tm re, im;
  cross(1, 2, re, im); u[12] = re; u[13] = -im;
  cross(2, 0, re, im); u[14] = re; u[15] = -im;
  cross(0, 1, re, im); u[16] = re; u[17] = -im;
}

template <typename Tg, typename Tm, int NR>
__device__ __forceinline__ void load_link(const Tg* __restrict__ gauge, int Vh, int parity, int mu,
                                          int site, Tm (&u)[18]) {
  constexpr int RP = link_pad<Tg>(NR);
  constexpr int VW = Store<Tg>::VW;
  const Tg* b = gauge + ((size_t)(parity * 4 + mu) * Vh + site) * RP;
  Tm tmp[RP];
#pragma unroll
  for (int c = 0; c < RP / VW; c++) load_vec<Tg, Tm>(b + c * VW, tmp + c * VW);
#pragma unroll
  for (int k = 0; k < NR; k++) u[k] = tmp[k];
  if constexpr (NR == 12) link_row3(u);
}

// chi = U h  or  U^dag h  for one colour vector (3 complex). Each real output is
// one multiply-add chain (one product, five fused multiply-adds).
template <bool DAG, typename Tm>
__device__ __forceinline__ void su3_mul(const Tm (&u)[18], const Tm* h, Tm* chi) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    Tm re, im;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const int k = DAG ? (b * 3 + a) * 2 : (a * 3 + b) * 2;
      const Tm ur = u[k];
      const Tm ui = DAG ? -u[k + 1] : u[k + 1];
      if (b == 0) {
        re = ur * h[0];
        im = ur * h[1];
      } else {
        re = fmadd(ur, h[2 * b], re);
        im = fmadd(ur, h[2 * b + 1], im);
      }
      re = fmadd(-ui, h[2 * b + 1], re);
      im = fmadd(ui, h[2 * b], im);
    }
    chi[2 * a] = re;
    chi[2 * a + 1] = im;
  }
}

// chi = U h - c  or  U^dag h - c: the chains of su3_mul started from -c.
template <bool DAG, typename Tm>
__device__ __forceinline__ void su3_mul_sub(const Tm (&u)[18], const Tm* h, const Tm* c, Tm* chi) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    Tm re = -c[2 * a], im = -c[2 * a + 1];
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const int k = DAG ? (b * 3 + a) * 2 : (a * 3 + b) * 2;
      const Tm ur = u[k];
      const Tm ui = DAG ? -u[k + 1] : u[k + 1];
      re = fmadd(ur, h[2 * b], re);
      im = fmadd(ur, h[2 * b + 1], im);
      re = fmadd(-ui, h[2 * b + 1], re);
      im = fmadd(ui, h[2 * b], im);
    }
    chi[2 * a] = re;
    chi[2 * a + 1] = im;
  }
}

// Spin projection h = (1 + S gamma_mu) psi on the upper two spins (the lower two follow
// from them), S = -1 forward, +1 backward. psi index: spin s, colour c, re/im ->
// psi[6 s + 2 c + {0, 1}]; h[0..5] spin 0, h[6..11] spin 1.
template <int MU, int S, typename Tm>
__device__ __forceinline__ void project(const Tm (&psi)[24], Tm (&h)[12]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const Tm p0r = psi[2 * c], p0i = psi[2 * c + 1];
    const Tm p1r = psi[6 + 2 * c], p1i = psi[6 + 2 * c + 1];
    const Tm p2r = psi[12 + 2 * c], p2i = psi[12 + 2 * c + 1];
    const Tm p3r = psi[18 + 2 * c], p3i = psi[18 + 2 * c + 1];
    Tm g0r, g0i, g1r, g1i;  // G psi_dn
    if (MU == 0) {          // G1 = [[0, i], [i, 0]]
      g0r = -p3i; g0i = p3r; g1r = -p2i; g1i = p2r;
    } else if (MU == 1) {   // G2 = [[0, -1], [1, 0]]
      g0r = -p3r; g0i = -p3i; g1r = p2r; g1i = p2i;
    } else if (MU == 2) {   // G3 = diag(i, -i)
      g0r = -p2i; g0i = p2r; g1r = p3i; g1i = -p3r;
    } else {                // G4 = 1
      g0r = p2r; g0i = p2i; g1r = p3r; g1i = p3i;
    }
    h[2 * c] = p0r + S * g0r; h[2 * c + 1] = p0i + S * g0i;
    h[6 + 2 * c] = p1r + S * g1r; h[6 + 2 * c + 1] = p1i + S * g1i;
  }
}

// The antiperiodic boundary phase ph = +-1 of a t hop. In FP64 it is a sign flip done on
// the integer units (identical to the product, and off the FP64 pipe).
template <typename Tm>
__device__ __forceinline__ void apply_phase(Tm (&h)[12], Tm ph) {
  if constexpr (std::is_same<Tm, double>::value) {
    const unsigned long long m = ph < 0 ? 0x8000000000000000ull : 0ull;
#pragma unroll
    for (int k = 0; k < 12; k++) h[k] = __longlong_as_double(__double_as_longlong(h[k]) ^ m);
  } else {
#pragma unroll
    for (int k = 0; k < 12; k++) h[k] *= ph;
  }
}

// The two hops of direction mu are formed as a pair. Forward, (1 - gamma_mu) U_mu(x)
// psi(x + mu): its upper-spin product xf = U h_f (hop_fwd). Backward, (1 + gamma_mu)
// U_mu(x - mu)^dag psi(x - mu): z = U^dag h_b - xf in one chain per entry, then
//   upper spins  += xf + xb = 2 xf + z,
//   lower spins  += G^dag (xb - xf) = G^dag z
// (the lower spins of a hop are -S G^dag of its upper product). The pair costs twelve
// operations fewer than two separate accumulations.
template <int MU, typename Tm>
__device__ __forceinline__ void fwd_core(Tm (&xf)[12], Tm (&h)[12], const Tm (&u)[18], Tm ph) {
  if (MU == 3) apply_phase(h, ph);
  su3_mul<false>(u, h, xf);
  su3_mul<false>(u, h + 6, xf + 6);
}

template <int MU, typename Tm>
__device__ __forceinline__ void hop_fwd(Tm (&xf)[12], const Tm (&psi)[24], const Tm (&u)[18], Tm ph) {
  Tm h[12];
  project<MU, -1>(psi, h);
  fwd_core<MU>(xf, h, u, ph);
}

template <int MU, typename Tm>
__device__ __forceinline__ void bwd_core(Tm (&acc)[24], const Tm (&xf)[12], Tm (&h)[12], const Tm (&u)[18], Tm ph) {
  if (MU == 3) apply_phase(h, ph);
  Tm z[12];
  su3_mul_sub<true>(u, h, xf, z);
  su3_mul_sub<true>(u, h + 6, xf + 6, z + 6);
#pragma unroll
  for (int c = 0; c < 3; c++) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
      acc[2 * c + q] = fmadd((Tm)2, xf[2 * c + q], acc[2 * c + q]) + z[2 * c + q];
      acc[6 + 2 * c + q] = fmadd((Tm)2, xf[6 + 2 * c + q], acc[6 + 2 * c + q]) + z[6 + 2 * c + q];
    }
    const Tm z0r = z[2 * c], z0i = z[2 * c + 1], z1r = z[6 + 2 * c], z1i = z[6 + 2 * c + 1];
    Tm d0r, d0i, d1r, d1i;  // G^dag z
    if (MU == 0) {          // G1^dag = [[0, -i], [-i, 0]]
      d0r = z1i; d0i = -z1r; d1r = z0i; d1i = -z0r;
    } else if (MU == 1) {   // G2^dag = [[0, 1], [-1, 0]]
      d0r = z1r; d0i = z1i; d1r = -z0r; d1i = -z0i;
    } else if (MU == 2) {   // G3^dag = diag(-i, i)
      d0r = z0i; d0i = -z0r; d1r = -z1i; d1i = z1r;
    } else {
      d0r = z0r; d0i = z0i; d1r = z1r; d1i = z1i;
    }
    acc[12 + 2 * c] += d0r; acc[12 + 2 * c + 1] += d0i;
    acc[18 + 2 * c] += d1r; acc[18 + 2 * c + 1] += d1i;
  }
}

template <int MU, typename Tm>
__device__ __forceinline__ void hop_bwd(Tm (&acc)[24], const Tm (&xf)[12], const Tm (&psi)[24], const Tm (&u)[18],
                                        Tm ph) {
  Tm h[12];
  project<MU, +1>(psi, h);
  bwd_core<MU>(acc, xf, h, u, ph);
}

// Mixed-precision adds (sm_100 and later): an FP16 operand enters an FP32 add directly,
// a + c or a - c rounded once to FP32 -- the value of converting a first, since the
// conversion is exact.
__device__ __forceinline__ float add_h(unsigned short a, float c) {
  float d;
  asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
  return d;
}
__device__ __forceinline__ float sub_h(unsigned short a, float c) {
  float d;
  asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
  return d;
}
__device__ __forceinline__ float h2f(unsigned short a) { return __half2float(__ushort_as_half(a)); }

// project<MU, S> on FP16 input: only the lower-spin entries are converted, the upper-spin
// ones enter the adds directly. Gives exactly the values of project() on converted input.
template <int MU, int S>
__device__ __forceinline__ void project_h(const unsigned short (&p)[24], float (&h)[12]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const float p2r = h2f(p[12 + 2 * c]), p2i = h2f(p[12 + 2 * c + 1]);
    const float p3r = h2f(p[18 + 2 * c]), p3i = h2f(p[18 + 2 * c + 1]);
    float g0r, g0i, g1r, g1i;  // G psi_dn, as in project()
    if (MU == 0) {
      g0r = -p3i; g0i = p3r; g1r = -p2i; g1i = p2r;
    } else if (MU == 1) {
      g0r = -p3r; g0i = -p3i; g1r = p2r; g1i = p2i;
    } else if (MU == 2) {
      g0r = -p2i; g0i = p2r; g1r = p3i; g1i = -p3r;
    } else {
      g0r = p2r; g0i = p2i; g1r = p3r; g1i = p3i;
    }
    if (S > 0) {
      h[2 * c] = add_h(p[2 * c], g0r); h[2 * c + 1] = add_h(p[2 * c + 1], g0i);
      h[6 + 2 * c] = add_h(p[6 + 2 * c], g1r); h[6 + 2 * c + 1] = add_h(p[6 + 2 * c + 1], g1i);
    } else {
      h[2 * c] = sub_h(p[2 * c], g0r); h[2 * c + 1] = sub_h(p[2 * c + 1], g0i);
      h[6 + 2 * c] = sub_h(p[6 + 2 * c], g1r); h[6 + 2 * c + 1] = sub_h(p[6 + 2 * c + 1], g1i);
    }
  }
}

template <typename Ts, typename Tg, typename Tm, int NR, int MU>
__device__ __forceinline__ void hop_mu(Tm (&acc)[24], const Field<Ts>& in, const Tg* gauge, const Geom& g,
                                       int p_out, int site, int sys, const int (&x)[4]) {
  Tm xf[12];
  // forward: (1 - g_mu) U_mu(x) psi(x + mu)
  {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[MU] += 1;
    Tm ph = 1;
    if (y[MU] == g.L[MU]) { y[MU] = 0; if (MU == 3) ph = (Tm)g.bc_t; }
    Tm psi[24], u[18];
    in.load(cb_index(g, y), sys, psi);
    load_link<Tg, Tm, NR>((const Tg*)gauge, g.Vh, p_out, MU, site, u);
    hop_fwd<MU>(xf, psi, u, ph);
  }
  // backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)
  {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[MU] -= 1;
    Tm ph = 1;
    if (y[MU] < 0) { y[MU] = g.L[MU] - 1; if (MU == 3) ph = (Tm)g.bc_t; }
    const int nb = cb_index(g, y);
    Tm psi[24], u[18];
    in.load(nb, sys, psi);
    load_link<Tg, Tm, NR>((const Tg*)gauge, g.Vh, 1 - p_out, MU, nb, u);
    hop_bwd<MU>(acc, xf, psi, u, ph);
  }
}

// Write per-thread values into per-(8-site group, system) partial sums, in fixed order.
// Ta: the type the 8 site values are summed in (the kernel's arithmetic type: FP32
// values are summed in FP32, as every FP32 hop variant does).
template <int K, typename Ta = double>
__device__ __forceinline__ void group_partials(const double (&vals)[K], int lsite, int lsys, int sys_base,
                                               const Shape& sh, int Vh, int chunk, double* smem,
                                               double* partial) {
  const int NB = sh.NB;
#pragma unroll
  for (int k = 0; k < K; k++) smem[(lsite * NB + lsys) * K + k] = vals[k];
  __syncthreads();
  const int ngb = sh.SB / 8;
  const int ngroups = Vh / 8;
  if (lsite < ngb) {
    const int grp = chunk * ngb + lsite;
    const int sys = sys_base + lsys;
    if (grp < ngroups && sys < sh.N) {
      Ta s[K];
#pragma unroll
      for (int k = 0; k < K; k++) s[k] = 0;
      for (int j = 0; j < 8; j++) {
#pragma unroll
        for (int k = 0; k < K; k++) s[k] += (Ta)smem[((lsite * 8 + j) * NB + lsys) * K + k];
      }
#pragma unroll
      for (int k = 0; k < K; k++) partial[((size_t)sys * K + k) * ngroups + grp] = (double)s[k];
    }
  }
  __syncthreads();
}

// Selected systems of a system-major launch (one system per block row, N <= 64), in
// ascending order, listed by every block itself: work items are then (k-th selected
// system, chunk), so a launch costs nothing for the systems it skips. Needs >= 64 threads.
__device__ __forceinline__ int selected_list(const SysState* st, int N, int mask, int* list) {
  __shared__ unsigned bal[2];
  const int t = threadIdx.x;
  const bool s = t < N && t < 64 && selected(st, t, mask);
  if (t < 64) {
    const unsigned b = __ballot_sync(0xffffffffu, s);
    if ((t & 31) == 0) bal[t >> 5] = b;
  }
  __syncthreads();
  if (s) list[__popc(bal[t >> 5] & ((1u << (t & 31)) - 1u)) + (t >= 32 ? __popc(bal[0]) : 0)] = t;
  const int n = __popc(bal[0]) + __popc(bal[1]);
  __syncthreads();
  return n;
}

// Half-precision storage is held to 3 resident blocks (<= 80 registers, no spills
// with 18-real links) for latency hiding; FP32 storage needs ~128 registers for its
// float4 spinors and keeps 2 blocks; FP64 is ALU bound.
// WL: system-major work-list launch (a.sysmajor); else the tile shape.
// WL launches (system-major work lists) use 128-thread blocks: bounds for three of them per
// SM leave the FP64 hop 168 registers; tile-shaped launches use 256-thread blocks.
// CLV: the Wilson-clover M-hat / D_sw epilogue, out = Y + A X + cb (H in) with Y = C X from a
// clover pass (the other coefficient changes of the clover operator follow a.clover at run time).
template <typename Ts, typename Tg, typename Tm, int NR, int COEF, int DOT, bool WL = false, bool CLV = false>
__global__ void __launch_bounds__(WL ? 128 : 256, WL ? 3 : (sizeof(Tm) == 8 ? 2 : (sizeof(Ts) == 2 ? 3 : 2)))
    hop_kernel(HopArgs a) {
  if (a.gate != nullptr && *a.gate == 0) return;
  constexpr int K = DotK<DOT>::K;
  __shared__ double smem[256 * (K > 0 ? K : 1)];
  const Shape sh = a.sh;
  const Geom g = a.g;
  const int lsys = threadIdx.x % sh.NB;
  const int lsite = threadIdx.x / sh.NB;
  constexpr bool smj = WL;
  const Field<Ts> in = make_field<Ts>(const_cast<void*>(a.in), g.Vh, sh.N, smj);
  const Field<Ts> out = make_field<Ts>(a.out, g.Vh, sh.N, smj);

  // one chunk of sites for system `sys` (sel: the system takes part), block rows sys_base..
  auto chunk_body = [&](const int sys, const int chunk, const bool sel, const int sys_base) {
    Tm ca = 0, cb = 1;
    if (sel) {
      const SysState& s = a.st[sys];
      // with the clover term the site factors A^-1 come from clover passes on the operands
      // (in = A_oo^-1 H x, z_o pre-inverted, x_o inverted afterwards) and C x enters through Y
      const bool cl = a.clover != 0;
      if (COEF == COEF_MHAT) { ca = coef<Tm>(s, C_A); cb = cl ? (Tm)-0.25 : coef<Tm>(s, C_MINV4A); }
      else if (COEF == COEF_DSLASH) { ca = coef<Tm>(s, C_A); cb = (Tm)-0.5; }
      else if (COEF == COEF_PREP) { ca = 1; cb = cl ? (Tm)0.5 : coef<Tm>(s, C_INV2A); }
      else if (COEF == COEF_RECON) { ca = cl ? (Tm)1 : coef<Tm>(s, C_INVA); cb = cl ? (Tm)0.5 : coef<Tm>(s, C_INV2A); }
      else if (COEF == COEF_TRUERES) { ca = coef<Tm>(s, C_MINVA); cb = cl ? (Tm)0.25 : coef<Tm>(s, C_INV4A); }
      else if (COEF == COEF_FULLRES) { ca = coef<Tm>(s, C_MINVA); cb = (Tm)0.5; }
      else if (COEF == COEF_KAPPA) { cb = cl ? (Tm)0.5 : coef<Tm>(s, C_INV2A); }  // clover: then A(x)^-1
    }
    const int site = chunk * sh.SB + lsite;
    const bool act = sel && site < g.Vh;
    if (a.work != nullptr) {  // profiling: (site, system) pairs computed, one atomic per warp
      const unsigned m = __ballot_sync(__activemask(), act);  // blocks may end in a partial warp
      if ((threadIdx.x & 31) == 0 && m) atomicAdd(a.work, (unsigned long long)__popc(m));
    }
    double dv[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < (K > 0 ? K : 1); k++) dv[k] = 0.0;
    if (act) {
      int x[4];
      cb_coords(g, a.p_out, site, x);
      Tm acc[24];
#pragma unroll
      for (int k = 0; k < 24; k++) acc[k] = 0;
      hop_mu<Ts, Tg, Tm, NR, 0>(acc, in, (const Tg*)a.gauge, g, a.p_out, site, sys, x);
      hop_mu<Ts, Tg, Tm, NR, 1>(acc, in, (const Tg*)a.gauge, g, a.p_out, site, sys, x);
      hop_mu<Ts, Tg, Tm, NR, 2>(acc, in, (const Tg*)a.gauge, g, a.p_out, site, sys, x);
      hop_mu<Ts, Tg, Tm, NR, 3>(acc, in, (const Tg*)a.gauge, g, a.p_out, site, sys, x);
      Tm o[24];
      if (COEF == COEF_PLAIN) {
#pragma unroll
        for (int k = 0; k < 24; k++) o[k] = acc[k];
      } else if (COEF == COEF_KAPPA) {
#pragma unroll
        for (int k = 0; k < 24; k++) o[k] = cb * acc[k];
      } else {
        Tm xv[24];
        make_field<Ts>(const_cast<void*>(a.X), g.Vh, sh.N, smj).load(site, sys, xv);
        if constexpr (CLV) {
          // Wilson-clover M-hat / D_sw: out = ca X + (cb (H in) + Y), Y = C X, in this rounding
          // order (the persistent kernel consumes Y before X)
          Tm yv[24];
          make_field<Ts>(const_cast<void*>(a.Y), g.Vh, sh.N, smj).load(site, sys, yv);
#pragma unroll
          for (int k = 0; k < 24; k++) o[k] = fmadd(ca, xv[k], fmadd(cb, acc[k], yv[k]));
        } else if constexpr (COEF == COEF_TRUERES || COEF == COEF_FULLRES) {
          // out = Y + ca X + cb (H in): two multiply-adds per entry
          Tm yv[24];
          make_field<Ts>(const_cast<void*>(a.Y), g.Vh, sh.N, smj).load(site, sys, yv);
#pragma unroll
          for (int k = 0; k < 24; k++) o[k] = fmadd(cb, acc[k], fmadd(ca, xv[k], yv[k]));
        } else {
#pragma unroll
          for (int k = 0; k < 24; k++) o[k] = axpby(ca, xv[k], cb, acc[k]);
        }
        if constexpr (DOT == DOT_TS) {
          Tm rv[24];
          make_field<Ts>(const_cast<void*>(a.R), g.Vh, sh.N, smj).load(site, sys, rv);
          ts_dots(dv, o, xv, rv);
        }
      }
      if (DOT == DOT_R) {
        Tm rv[24];
        make_field<Ts>(const_cast<void*>(a.R), g.Vh, sh.N, smj).load(site, sys, rv);
        Tm sr = 0, si = 0;
#pragma unroll
        for (int k = 0; k < 24; k += 2) dot_acc(sr, si, rv[k], rv[k + 1], o[k], o[k + 1]);
        dv[0] = (double)sr; dv[1] = (double)si;
      }
      if (DOT == DOT_NORM) {
        Tm nn = 0;
#pragma unroll
        for (int k = 0; k < 24; k += 2) norm_acc(nn, o[k], o[k + 1]);
        dv[0] = (double)nn;
      }
      out.store(site, sys, o);
    }
    if constexpr (K > 0) {
      group_partials<K, Tm>(dv, lsite, lsys, sys_base, sh, g.Vh, chunk, smem, a.partial);
    }
  };

  if constexpr (!WL) {
    const int sys = blockIdx.y * sh.NB + lsys;
    const bool sel = sys < sh.N && selected(a.st, sys, a.mask);
    for (int chunk = blockIdx.x; chunk < sh.nchunk; chunk += gridDim.x) chunk_body(sys, chunk, sel, blockIdx.y * sh.NB);
  } else {
    // system-major (NB = 1, grid.y = 1): items (k-th selected system, chunk)
    __shared__ int slist[64];
    const int nsel = selected_list(a.st, sh.N, a.mask, slist);
    for (int item = blockIdx.x; item < nsel * sh.nchunk; item += gridDim.x) {
      const int sys = slist[item / sh.nchunk];
      chunk_body(sys, item - (item / sh.nchunk) * sh.nchunk, true, sys);
    }
  }
}

}  // namespace fs

namespace fs {

// ---- prefetching variant --------------------------------------------------------
// The eight neighbour spinors of a (site, system) are fetched with per-thread
// asynchronous copies (cp.async.cg, 16 B each, L2 only) into a ring of PF shared
// memory slots, PF directions ahead of the arithmetic; the epilogue operands X
// and R follow the directions through the same ring. This keeps ~PF x 24 reals
// of every thread in flight without holding them in registers. Each thread reads
// back only what it copied, so the ring needs no block barrier.
// Ring layout: [slot][16-byte chunk][thread] (conflict-free 128-bit LDS/STS).

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename Ts>
__host__ __device__ constexpr int chunks16() { return 24 * (int)sizeof(Ts) / 16; }

template <typename Ts, int PF>
__host__ __device__ constexpr size_t hop_pf_smem(int block) {
  return (size_t)PF * chunks16<Ts>() * block * 16;
}

// Links of a block's sites staged in shared memory as FP32 (reconstructed once per
// link instead of once per thread) when a block covers few sites, i.e. many systems
// per site: [site][direction][20 floats] (18 used, padded to 16-byte multiples).
constexpr int LINK_STAGE_MAX_SITES = 32;
constexpr int LINK_F32 = 20;

template <typename Ts, typename Tg, typename Tm, int NR, int COEF, int DOT, int PF>
__global__ void __launch_bounds__(256, 2) hop_kernel_pf(HopArgs a) {
  constexpr int K = DotK<DOT>::K;
  constexpr int CV = chunks16<Ts>();
  constexpr int VW = Store<Ts>::VW;
  // items: 0..7 neighbour spinors, 8 = X (epilogue axpy operand), 9 = R (dot partner)
  constexpr bool HAS_X = COEF != COEF_PLAIN;
  constexpr bool HAS_R = DOT == DOT_R || DOT == DOT_TS;
  constexpr int NITEM = 8 + (HAS_X ? 1 : 0) + (HAS_R ? 1 : 0);
  extern __shared__ uint4 ring[];
  __shared__ double smem[256 * (K > 0 ? K : 1)];
  __shared__ __align__(16) float lsm[LINK_STAGE_MAX_SITES * 8 * LINK_F32];
  __shared__ unsigned grp_arrivals;
  if (a.gate != nullptr && *a.gate == 0) return;
  const Shape sh = a.sh;
  const Geom g = a.g;
  const int T = blockDim.x;
  // With 32 systems per warp a warp is one site: links are staged per warp and the
  // 8-site dot partials are combined by the last warp to arrive (no block barrier).
  const bool warp_mode = sh.NB == 32 && gridDim.x >= sh.nchunk;  // uniform per launch
  const bool stage = !warp_mode && sh.SB <= LINK_STAGE_MAX_SITES;  // block-cooperative staging
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lsys = threadIdx.x % sh.NB;
  const int lsite = threadIdx.x / sh.NB;
  const int sys = blockIdx.y * sh.NB + lsys;
  const bool sel = sys < sh.N && selected(a.st, sys, a.mask);
  if (warp_mode && K > 0) {
    if (threadIdx.x == 0) grp_arrivals = 0;
    __syncthreads();
  }

  Tm ca = 0, cb = 1;
  if (sel) {
    const SysState& s = a.st[sys];
    if (COEF == COEF_MHAT) { ca = coef<Tm>(s, C_A); cb = coef<Tm>(s, C_MINV4A); }
    else if (COEF == COEF_DSLASH) { ca = coef<Tm>(s, C_A); cb = (Tm)-0.5; }
  }
  const size_t cstride = (size_t)g.Vh * sh.N * VW;  // elements between 16-byte chunks c and c+1
  const size_t rowstride = (size_t)sh.N * VW;        // elements between consecutive sites

  for (int chunk = blockIdx.x; chunk < sh.nchunk; chunk += gridDim.x) {
    const int site = chunk * sh.SB + lsite;
    const bool live = site < g.Vh;
    const bool act = sel && live;
    if (a.work != nullptr) {  // profiling: (site, system) pairs computed, one atomic per warp
      const unsigned m = __ballot_sync(__activemask(), act);  // blocks may end in a partial warp
      if ((threadIdx.x & 31) == 0 && m) atomicAdd(a.work, (unsigned long long)__popc(m));
    }
    int nb[8];
    Tm ph[2] = {1, 1};  // t forward / backward boundary phase
    if (live) {
      int x[4];
      cb_coords(g, a.p_out, site, x);
#pragma unroll
      for (int mu = 0; mu < 4; mu++) {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = x[mu] + 1;
        if (y[mu] == g.L[mu]) { y[mu] = 0; if (mu == 3) ph[0] = (Tm)g.bc_t; }
        nb[2 * mu] = cb_index(g, y);
        y[mu] = x[mu] - 1;
        if (y[mu] < 0) { y[mu] = g.L[mu] - 1; if (mu == 3) ph[1] = (Tm)g.bc_t; }
        nb[2 * mu + 1] = cb_index(g, y);
      }
    }
    const Ts* in_base = (const Ts*)a.in + (size_t)sys * VW;
    const size_t myoff = (size_t)site * rowstride + (size_t)sys * VW;
    auto issue = [&](int item) {
      if (act && item < NITEM) {
        const Ts* src;
        if (item < 8) src = in_base + (size_t)nb[item] * rowstride;
        else if (HAS_X && item == 8) src = (const Ts*)a.X + myoff;
        else src = (const Ts*)a.R + myoff;
        uint4* dst = ring + (size_t)(item % PF) * CV * T + threadIdx.x;
#pragma unroll
        for (int c = 0; c < CV; c++) cp_async16(dst + c * T, src + c * cstride);
      }
      cp_async_commit();  // one group per item (empty when idle) keeps the wait counts uniform
    };
    auto fetch = [&](int item, Tm (&v)[24]) {
      const uint4* srcv = ring + (size_t)(item % PF) * CV * T + threadIdx.x;
#pragma unroll
      for (int c = 0; c < CV; c++) {
        const uint4 w = srcv[c * T];
        load_vec<Ts, Tm>(reinterpret_cast<const Ts*>(&w), v + c * VW);
      }
    };
#pragma unroll
    for (int i = 0; i < PF; i++) issue(i);
    // links of this chunk's sites, reconstructed once, while the first spinors are in flight
    float* my_links = lsm + (warp_mode ? warp : lsite) * 8 * LINK_F32;
    if (warp_mode) {
      if (lane < 8 && live) {
        const int d = lane, mu = d >> 1;
        int nbd = nb[1];
#pragma unroll
        for (int k = 3; k < 8; k += 2)
          if (d == k) nbd = nb[k];
        Tm u[18];
        if ((d & 1) == 0) load_link<Tg, Tm, NR>((const Tg*)a.gauge, g.Vh, a.p_out, mu, site, u);
        else load_link<Tg, Tm, NR>((const Tg*)a.gauge, g.Vh, 1 - a.p_out, mu, nbd, u);
        float* dst = my_links + d * LINK_F32;
#pragma unroll
        for (int q = 0; q < 18; q++) dst[q] = (float)u[q];
      }
      __syncwarp();
    } else if (stage) {
      // thread k < 8 SB stages link k: site chunk*SB + k/8, direction k%8
      __syncthreads();  // the previous chunk's readers are done with lsm
      for (int k = threadIdx.x; k < 8 * sh.SB; k += T) {
        const int ls = k >> 3, d = k & 7, mu = d >> 1;
        const int s2 = chunk * sh.SB + ls;
        if (s2 < g.Vh) {
          Tm u[18];
          if ((d & 1) == 0) {
            load_link<Tg, Tm, NR>((const Tg*)a.gauge, g.Vh, a.p_out, mu, s2, u);
          } else {
            int x[4];
            cb_coords(g, a.p_out, s2, x);
            x[mu] = x[mu] == 0 ? g.L[mu] - 1 : x[mu] - 1;
            load_link<Tg, Tm, NR>((const Tg*)a.gauge, g.Vh, 1 - a.p_out, mu, cb_index(g, x), u);
          }
          float* dst = lsm + (ls * 8 + d) * LINK_F32;
#pragma unroll
          for (int q = 0; q < 18; q++) dst[q] = (float)u[q];
        }
      }
      __syncthreads();
    }
    const bool staged = warp_mode || stage;
    Tm acc[24], xf[12];
#pragma unroll
    for (int k = 0; k < 24; k++) acc[k] = 0;
#pragma unroll
    for (int d = 0; d < 8; d++) {
      cp_async_wait<PF - 1>();
      Tm psi[24], u[18];
      if (act) {
        fetch(d, psi);
        const int mu = d >> 1;
        if (staged) {
          const float4* src4 = reinterpret_cast<const float4*>(my_links + d * LINK_F32);
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const float4 w = src4[q];
            u[4 * q] = (Tm)w.x; u[4 * q + 1] = (Tm)w.y; u[4 * q + 2] = (Tm)w.z; u[4 * q + 3] = (Tm)w.w;
          }
          const float2 w2 = *reinterpret_cast<const float2*>(my_links + d * LINK_F32 + 16);
          u[16] = (Tm)w2.x; u[17] = (Tm)w2.y;
        } else if ((d & 1) == 0) {
          load_link<Tg, Tm, NR>((const Tg*)a.gauge, g.Vh, a.p_out, mu, site, u);
        } else {
          load_link<Tg, Tm, NR>((const Tg*)a.gauge, g.Vh, 1 - a.p_out, mu, nb[d], u);
        }
      }
      issue(d + PF);  // the slot just read is refilled
      if (act) {
        switch (d) {
          case 0: hop_fwd<0>(xf, psi, u, (Tm)1); break;
          case 1: hop_bwd<0>(acc, xf, psi, u, (Tm)1); break;
          case 2: hop_fwd<1>(xf, psi, u, (Tm)1); break;
          case 3: hop_bwd<1>(acc, xf, psi, u, (Tm)1); break;
          case 4: hop_fwd<2>(xf, psi, u, (Tm)1); break;
          case 5: hop_bwd<2>(acc, xf, psi, u, (Tm)1); break;
          case 6: hop_fwd<3>(xf, psi, u, ph[0]); break;
          default: hop_bwd<3>(acc, xf, psi, u, ph[1]); break;
        }
      }
    }
    // remaining items (X, R) were issued in the last steps; wait for all
    for (int i = 8 + PF; i < NITEM; i++) issue(i);
    cp_async_wait<0>();
    double dv[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < (K > 0 ? K : 1); k++) dv[k] = 0.0;
    if (act) {
      Tm o[24], xv[24];
      if constexpr (!HAS_X) {
#pragma unroll
        for (int k = 0; k < 24; k++) o[k] = acc[k];
      } else {
        fetch(8, xv);
#pragma unroll
        for (int k = 0; k < 24; k++) o[k] = axpby(ca, xv[k], cb, acc[k]);
      }
      if constexpr (HAS_R) {
        Tm rv[24];
        fetch(8 + (HAS_X ? 1 : 0), rv);
        if constexpr (DOT == DOT_TS) {
          ts_dots(dv, o, xv, rv);
        } else {
          Tm sr = 0, si = 0;
#pragma unroll
          for (int k = 0; k < 24; k += 2) dot_acc(sr, si, rv[k], rv[k + 1], o[k], o[k + 1]);
          dv[0] = (double)sr; dv[1] = (double)si;
        }
      }
      make_field<Ts>(a.out, g.Vh, sh.N).store(site, sys, o);
    }
    if constexpr (K > 0) {
      if (warp_mode) {
        // warp = site `warp` of the chunk's single 8-site group; lane = system
#pragma unroll
        for (int k = 0; k < K; k++) smem[(warp * 32 + lane) * K + k] = dv[k];
        __syncwarp();
        __threadfence_block();
        unsigned ticket = 0;
        if (lane == 0) ticket = atomicAdd(&grp_arrivals, 1u);
        ticket = __shfl_sync(0xffffffffu, ticket, 0);
        if ((ticket & 7u) == 7u) {  // the last of the 8 warps sums the group in site order
          __threadfence_block();
          const int ngroups = g.Vh / 8;
          const int grp = chunk;
          const int sysg = blockIdx.y * 32 + lane;
          if (grp < ngroups && sysg < sh.N) {
            Tm sacc[K > 0 ? K : 1];
#pragma unroll
            for (int k = 0; k < K; k++) sacc[k] = 0;
            for (int j = 0; j < 8; j++) {
#pragma unroll
              for (int k = 0; k < K; k++) sacc[k] += (Tm)smem[(j * 32 + lane) * K + k];
            }
#pragma unroll
            for (int k = 0; k < K; k++) a.partial[((size_t)sysg * K + k) * ngroups + grp] = (double)sacc[k];
          }
        }
      } else {
        group_partials<K, Tm>(dv, lsite, lsys, blockIdx.y * sh.NB, sh, g.Vh, chunk, smem, a.partial);
      }
    }
  }
}

}  // namespace fs

namespace fs {

// ---- persistent paired variant: two systems per thread in packed FP32 arithmetic -----
// A 32-system tile chunk at one site is held by 16 lanes: lane q computes systems q and
// q + 16 in the two halves of packed FP32 instructions (fma/add/mul .f32x2: one issue slot
// for two systems, each half rounded exactly as the scalar instruction), so every system
// goes through the same sequence of roundings as in the scalar hop kernels. A warp holds
// two sites, a 128-thread block the 8 sites of one 8-site dot group, and the persistent
// grid (resident blocks x SMs) sweeps the site chunks blockIdx.x, blockIdx.x + gridDim.x, ...
//
// Operands stream through a per-thread ring of PF shared-memory slots (cp.async, 16 B per
// copy), item n = j NITEM + i of chunk j (the 8 neighbour spinors, then X and R), PF items
// ahead of the arithmetic and across chunk boundaries. The raw links of a chunk travel with
// its item 0; lane d < 8 of each half-warp rebuilds link d of its site once and stores it as
// (s u_r, u_i) per entry, s = -1 for the forward links, with the t boundary phase folded in.
// The forward hop therefore forms -U h directly and the backward chain starts from it; the
// packed operands (s u_r, s u_r), (u_i, u_i) and (-u_i, -u_i) are formed in registers
// (measured faster than storing them pre-paired: half the shared-memory link reads).
namespace pk {
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// -a (a sign flip, which the packed instructions take as an operand modifier) and a - b
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }

constexpr int LINK_PK = 18;              // floats per link: 9 entries (s u_r, u_i)
constexpr int SITE_PK = 8 * LINK_PK + 4;  // per site; the 4 pad floats put the two sites of a
                                          // warp on different banks

// nxf = -U h_f, the forward hop's upper-spin product negated (links stored with s = -1): row
// by row, both spin halves together (four independent chains), in su3_mul's multiply-add order.
__device__ __forceinline__ void fwd_pk(float2 (&nxf)[12], const float2 (&h)[12], const float* L) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float2 r0, i0, r1, i1;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const float2 w = *reinterpret_cast<const float2*>(L + 2 * (a * 3 + b));
      const float2 ur = make_float2(w.x, w.x), up = make_float2(w.y, w.y), um = make_float2(-w.y, -w.y);
      if (b == 0) {
        r0 = mul2(ur, h[0]); i0 = mul2(ur, h[1]); r1 = mul2(ur, h[6]); i1 = mul2(ur, h[7]);
      } else {
        r0 = fma2(ur, h[2 * b], r0); i0 = fma2(ur, h[2 * b + 1], i0);
        r1 = fma2(ur, h[6 + 2 * b], r1); i1 = fma2(ur, h[6 + 2 * b + 1], i1);
      }
      r0 = fma2(up, h[2 * b + 1], r0); i0 = fma2(um, h[2 * b], i0);
      r1 = fma2(up, h[6 + 2 * b + 1], r1); i1 = fma2(um, h[6 + 2 * b], i1);
    }
    nxf[2 * a] = r0; nxf[2 * a + 1] = i0; nxf[6 + 2 * a] = r1; nxf[6 + 2 * a + 1] = i1;
  }
}

// Backward hop of direction MU (bwd_core, packed): row c of z = U^dag h_b - xf for both spin
// halves (the chains of su3_mul_sub, started from nxf = -xf), then at once
//   upper spins += 2 xf + z,   lower spins += G^dag z.
template <int MU>
__device__ __forceinline__ void bwd_pk(float2 (&acc)[24], const float2 (&nxf)[12], const float2 (&h)[12],
                                       const float* L) {
  const float2 m2 = make_float2(-2.f, -2.f);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float2 z0r, z0i, z1r, z1i;
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const float2 w = *reinterpret_cast<const float2*>(L + 2 * (b * 3 + c));
      const float2 ur = make_float2(w.x, w.x), up = make_float2(w.y, w.y), um = make_float2(-w.y, -w.y);
      if (b == 0) {
        z0r = fma2(ur, h[0], nxf[2 * c]); z0i = fma2(ur, h[1], nxf[2 * c + 1]);
        z1r = fma2(ur, h[6], nxf[6 + 2 * c]); z1i = fma2(ur, h[7], nxf[6 + 2 * c + 1]);
      } else {
        z0r = fma2(ur, h[2 * b], z0r); z0i = fma2(ur, h[2 * b + 1], z0i);
        z1r = fma2(ur, h[6 + 2 * b], z1r); z1i = fma2(ur, h[6 + 2 * b + 1], z1i);
      }
      z0r = fma2(up, h[2 * b + 1], z0r); z0i = fma2(um, h[2 * b], z0i);
      z1r = fma2(up, h[6 + 2 * b + 1], z1r); z1i = fma2(um, h[6 + 2 * b], z1i);
    }
    acc[2 * c] = add2(fma2(m2, nxf[2 * c], acc[2 * c]), z0r);
    acc[2 * c + 1] = add2(fma2(m2, nxf[2 * c + 1], acc[2 * c + 1]), z0i);
    acc[6 + 2 * c] = add2(fma2(m2, nxf[6 + 2 * c], acc[6 + 2 * c]), z1r);
    acc[6 + 2 * c + 1] = add2(fma2(m2, nxf[6 + 2 * c + 1], acc[6 + 2 * c + 1]), z1i);
    float2& a0r = acc[12 + 2 * c];
    float2& a0i = acc[12 + 2 * c + 1];
    float2& a1r = acc[18 + 2 * c];
    float2& a1i = acc[18 + 2 * c + 1];
    if (MU == 0) {         // G1^dag = [[0, -i], [-i, 0]]
      a0r = add2(a0r, z1i); a0i = sub2(a0i, z1r); a1r = add2(a1r, z0i); a1i = sub2(a1i, z0r);
    } else if (MU == 1) {  // G2^dag = [[0, 1], [-1, 0]]
      a0r = add2(a0r, z1r); a0i = add2(a0i, z1i); a1r = sub2(a1r, z0r); a1i = sub2(a1i, z0i);
    } else if (MU == 2) {  // G3^dag = diag(-i, i)
      a0r = add2(a0r, z0i); a0i = sub2(a0i, z0r); a1r = sub2(a1r, z1i); a1i = add2(a1i, z1r);
    } else {
      a0r = add2(a0r, z0r); a0i = add2(a0i, z0i); a1r = add2(a1r, z1r); a1i = add2(a1i, z1i);
    }
  }
}

// Spin projection of both systems (scalar: the destination registers of the two halves are
// free, so the pairs cost no moves). FP16 input takes the mixed-precision adds of project_h.
template <int MU, int S, typename Ts, int CV>
__device__ __forceinline__ void project_pk(const uint4 (&wa)[CV], const uint4 (&wb)[CV], float2 (&h)[12]) {
  float ha[12], hb[12];
  if constexpr (std::is_same<Ts, __half>::value) {
    unsigned short pa[24], pb[24];
#pragma unroll
    for (int c = 0; c < CV; c++) {
      const unsigned short* qa = reinterpret_cast<const unsigned short*>(&wa[c]);
      const unsigned short* qb = reinterpret_cast<const unsigned short*>(&wb[c]);
#pragma unroll
      for (int e = 0; e < 8; e++) { pa[c * 8 + e] = qa[e]; pb[c * 8 + e] = qb[e]; }
    }
    project_h<MU, S>(pa, ha);
    project_h<MU, S>(pb, hb);
  } else {
    constexpr int VW = Store<Ts>::VW;
    float psa[24], psb[24];
#pragma unroll
    for (int c = 0; c < CV; c++) {
      load_vec<Ts, float>(reinterpret_cast<const Ts*>(&wa[c]), psa + c * VW);
      load_vec<Ts, float>(reinterpret_cast<const Ts*>(&wb[c]), psb + c * VW);
    }
    project<MU, S>(psa, ha);
    project<MU, S>(psb, hb);
  }
#pragma unroll
  for (int k = 0; k < 12; k++) h[k] = make_float2(ha[k], hb[k]);
}
}  // namespace pk

template <typename Ts, int PF, int K>
__host__ __device__ constexpr size_t hop_pk_smem() {
  // ring [PF][CV][2 systems][128 threads] x 16 B
  return (size_t)PF * chunks16<Ts>() * 2 * 128 * 16;
}

template <bool COND> struct BoolC { static constexpr bool value = COND; };
template <int I> struct IntC { static constexpr int value = I; };

template <typename Tg>
__host__ __device__ constexpr int link_chunks16(int nr) {
  return link_pad<Tg>(nr) * (int)sizeof(Tg) / 16;
}

// CLV: the Wilson-clover M-hat, out = ca X + (cb (H in) + Y) with Y = C X from a clover pass
// (an operand item of its own, consumed before X).
template <typename Ts, typename Tg, int NR, int COEF, int DOT, int PF, bool CLV = false>
__global__ void __launch_bounds__(128, 3) hop_kernel_pk(HopArgs a) {
  using namespace pk;
  constexpr int K = DotK<DOT>::K;
  constexpr int KK = K > 0 ? K : 1;
  constexpr int CV = chunks16<Ts>();
  constexpr int VW = Store<Ts>::VW;
  constexpr bool HAS_X = COEF != COEF_PLAIN;
  constexpr bool HAS_Y = CLV;
  constexpr bool HAS_R = DOT == DOT_R || DOT == DOT_TS;
  static_assert(!CLV || COEF == COEF_MHAT, "the clover operand belongs to M-hat");
  constexpr int NITEM = 8 + (HAS_X ? 1 : 0) + (HAS_Y ? 1 : 0) + (HAS_R ? 1 : 0);
  constexpr int IY = 8;                    // Y, when present
  constexpr int IX = 8 + (HAS_Y ? 1 : 0);  // X
  constexpr int IR = NITEM - 1;            // R
  static_assert(PF >= 1 && PF < NITEM && PF <= 6, "ring depth");
  static_assert(DOT != DOT_TS || (HAS_X && PF >= 2), "DOT_TS consumes X and R together");
  constexpr int RPC = link_chunks16<Tg>(NR);  // 16-byte chunks per stored link
  constexpr int RP = link_pad<Tg>(NR);
  constexpr int GVW = Store<Tg>::VW;
  extern __shared__ uint4 ring[];             // [PF][CV][2][128]
  // dot values of chunk parity j & 1: [site][value][system]; FP32 sums, so held exactly as float
  __shared__ float dsm[2][8][KK][32];
  __shared__ __align__(16) float lsm[4 * 2 * SITE_PK];   // [warp][half][direction][LINK_PK]
  __shared__ uint4 lraw[2 * 4 * 2 * 8 * RPC];            // raw links, double buffered by chunk parity
  if (a.gate != nullptr && *a.gate == 0) return;
  const Shape sh = a.sh;
  const Geom g = a.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int half = lane >> 4, q = lane & 15;
  const int ls = 2 * warp + half;              // site of the chunk
  const int sa = blockIdx.y * 32 + q, sb = sa + 16;
  const bool sel_a = sa < sh.N && selected(a.st, sa, a.mask);
  const bool sel_b = sb < sh.N && selected(a.st, sb, a.mask);
  float2 ca = make_float2(0.f, 0.f), cb = make_float2(1.f, 1.f);
  if (COEF == COEF_MHAT || COEF == COEF_DSLASH) {
    // Wilson-clover: the site factors come from clover passes, H_eo A_oo^-1 H_oe p / 4
    if (sel_a) { ca.x = coef<float>(a.st[sa], C_A); cb.x = COEF == COEF_MHAT ? (CLV ? -0.25f : coef<float>(a.st[sa], C_MINV4A)) : -0.5f; }
    if (sel_b) { ca.y = coef<float>(a.st[sb], C_A); cb.y = COEF == COEF_MHAT ? (CLV ? -0.25f : coef<float>(a.st[sb], C_MINV4A)) : -0.5f; }
  }
  const size_t cstride = (size_t)g.Vh * sh.N * VW;  // elements between 16-byte chunks c and c+1
  const size_t rowstride = (size_t)sh.N * VW;        // elements between consecutive sites
  const Ts* in_a = (const Ts*)a.in + (size_t)sa * VW;
  const int G = gridDim.x;
  const int nmine = (sh.nchunk - (int)blockIdx.x + G - 1) / G;  // chunks of this block (uniform)
  if (a.work != nullptr) {  // profiling: (site, system) pairs computed, one atomic per warp
    const int m = __popc(__ballot_sync(0xffffffffu, sel_a)) + __popc(__ballot_sync(0xffffffffu, sel_b));
    if (lane == 0 && m && nmine > 0) atomicAdd(a.work, (unsigned long long)m * (unsigned long long)nmine);
  }
  const int dl = q & 7, mul = dl >> 1;  // the direction this lane computes neighbours for
  auto site_of = [&](int j) { return ((int)blockIdx.x + j * G) * 8 + ls; };
  // neighbour of site in direction dl, and the boundary phase of that hop (unrolled over mu
  // with selects: a lane-dependent array index would put the geometry in local memory)
  auto neighbour = [&](int site, int& nb, float& ph) {
    int x[4];
    cb_coords(g, a.p_out, site, x);
    ph = 1.f;
#pragma unroll
    for (int m = 0; m < 4; m++) {
      if (m == mul) {
        int y = x[m];
        if ((dl & 1) == 0) {
          y += 1;
          if (y == g.L[m]) { y = 0; if (m == 3) ph = (float)g.bc_t; }
        } else {
          y -= 1;
          if (y < 0) { y = g.L[m] - 1; if (m == 3) ph = (float)g.bc_t; }
        }
        x[m] = y;
      }
    }
    nb = cb_index(g, x);
  };
  int nbc = 0, nbn = 0;
  float phc = 1.f, phn = 1.f;
  if (nmine > 0) neighbour(site_of(0), nbc, phc);
  if (nmine > 1) neighbour(site_of(1), nbn, phn);

  auto slot_of = [&](int j, int i) {  // compile-time where PF divides the items per chunk
    if constexpr (NITEM % PF == 0) return i % PF;
    else return (int)(((unsigned)j * NITEM + i) % PF);
  };
  auto ring_at = [&](int slot, int c, int s) -> uint4* { return ring + (((size_t)slot * CV + c) * 2 + s) * 128 + tid; };
  // issue operand I of chunk j (NEXT: j is the chunk after the current one)
  auto issue = [&](auto Ic, auto NEXTc, int j) {
    constexpr int I = decltype(Ic)::value;
    constexpr bool NEXT = decltype(NEXTc)::value;
    if (j < nmine) {
      const int nbl = NEXT ? nbn : nbc;
      const int site = site_of(j);
      if (I == 0 && q < 8) {
        // raw link of direction d = q: U_mu(x) forward, U_mu(x - mu) backward
        const int lsite = (dl & 1) ? nbl : site;
        const int par = (dl & 1) ? 1 - a.p_out : a.p_out;
        const Tg* src = (const Tg*)a.gauge + ((size_t)(par * 4 + mul) * g.Vh + lsite) * RP;
        uint4* dst = lraw + ((((j & 1) * 4 + warp) * 2 + half) * 8 + dl) * RPC;
#pragma unroll
        for (int c = 0; c < RPC; c++) cp_async16(dst + c, src + c * (16 / sizeof(Tg)));
      }
      const Ts* src;
      if constexpr (I < 8) {
        const int nbi = __shfl_sync(0xffffffffu, nbl, (lane & 16) | I);
        src = in_a + (size_t)nbi * rowstride;
      } else {
        const Ts* base = (HAS_Y && I == IY) ? (const Ts*)a.Y : (HAS_X && I == IX) ? (const Ts*)a.X : (const Ts*)a.R;
        src = base + (size_t)site * rowstride + (size_t)sa * VW;
      }
      const int slot = slot_of(j, I);
      if (sel_a) {
#pragma unroll
        for (int c = 0; c < CV; c++) cp_async16(ring_at(slot, c, 0), src + c * cstride);
      }
      if (sel_b) {
#pragma unroll
        for (int c = 0; c < CV; c++) cp_async16(ring_at(slot, c, 1), src + c * cstride + 16 * VW);
      }
    }
    cp_async_commit();  // one group per item (empty when idle) keeps the wait counts uniform
  };
  // item I of chunk j, PF items ahead of item D being consumed
  auto issue_ahead = [&](auto Dc, int j) {
    constexpr int N2 = decltype(Dc)::value + PF;
    if constexpr (N2 < NITEM) issue(IntC<N2>{}, BoolC<false>{}, j);
    else issue(IntC<N2 - NITEM>{}, BoolC<true>{}, j + 1);
  };
  // 16-byte chunk c of both systems' operand in `slot`, converted to FP32 pairs
  auto fetch_pk = [&](int slot, int c, float2* v) {
    float xa[VW], xb[VW];
    const uint4 wa = *ring_at(slot, c, 0), wb = *ring_at(slot, c, 1);
    load_vec<Ts, float>(reinterpret_cast<const Ts*>(&wa), xa);
    load_vec<Ts, float>(reinterpret_cast<const Ts*>(&wb), xb);
#pragma unroll
    for (int k = 0; k < VW; k++) v[k] = make_float2(xa[k], xb[k]);
  };

  // prologue: the first PF operands of chunk 0
  issue(IntC<0>{}, BoolC<false>{}, 0);
  if constexpr (PF > 1) issue(IntC<1>{}, BoolC<false>{}, 0);
  if constexpr (PF > 2) issue(IntC<2>{}, BoolC<false>{}, 0);
  if constexpr (PF > 3) issue(IntC<3>{}, BoolC<false>{}, 0);
  if constexpr (PF > 4) issue(IntC<4>{}, BoolC<false>{}, 0);
  if constexpr (PF > 5) issue(IntC<5>{}, BoolC<false>{}, 0);

  const float* wl = lsm + (warp * 2 + half) * SITE_PK;
  for (int j = 0; j < nmine; j++) {
    const int site = site_of(j);
    float2 acc[24], nxf[12];
#pragma unroll
    for (int k = 0; k < 24; k++) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 8; d++) {
      cp_async_wait<PF - 1>();
      if (d == 0) {
        // this chunk's raw links arrived with its item 0: lane d < 8 of each half rebuilds
        // link d of its site, folds in the t boundary phase and stores it sign-paired
        __syncwarp();  // every lane is done with the previous chunk's links
        if (q < 8) {
          const Tg* rawp = reinterpret_cast<const Tg*>(lraw + ((((j & 1) * 4 + warp) * 2 + half) * 8 + q) * RPC);
          float tmp[RP];
#pragma unroll
          for (int c = 0; c < RP / GVW; c++) load_vec<Tg, float>(rawp + c * GVW, tmp + c * GVW);
          float u[18];
#pragma unroll
          for (int k = 0; k < NR; k++) u[k] = tmp[k];
          if constexpr (NR == 12) link_row3(u);
          const float sr = (q & 1) ? phc : -phc;  // forward links negated
          float* dst = lsm + (warp * 2 + half) * SITE_PK + q * LINK_PK;
#pragma unroll
          for (int k = 0; k < 9; k++)
            *reinterpret_cast<float2*>(dst + 2 * k) = make_float2(u[2 * k] * sr, u[2 * k + 1] * phc);
        }
        __syncwarp();
      }
      // every lane computes (no per-lane branches); a system that sits out reads a stale
      // ring slot, and its results are neither stored nor summed
      uint4 wa[CV], wb[CV];
      {
        const int slot = slot_of(j, d);
#pragma unroll
        for (int c = 0; c < CV; c++) { wa[c] = *ring_at(slot, c, 0); wb[c] = *ring_at(slot, c, 1); }
      }
      switch (d) {  // the slot just read is refilled (d is a constant after unrolling)
        case 0: issue_ahead(IntC<0>{}, j); break;
        case 1: issue_ahead(IntC<1>{}, j); break;
        case 2: issue_ahead(IntC<2>{}, j); break;
        case 3: issue_ahead(IntC<3>{}, j); break;
        case 4: issue_ahead(IntC<4>{}, j); break;
        case 5: issue_ahead(IntC<5>{}, j); break;
        case 6: issue_ahead(IntC<6>{}, j); break;
        default: issue_ahead(IntC<7>{}, j); break;
      }
      float2 h[12];
      const float* L = wl + d * LINK_PK;
      switch (d) {
        case 0: project_pk<0, -1, Ts, CV>(wa, wb, h); fwd_pk(nxf, h, L); break;
        case 1: project_pk<0, +1, Ts, CV>(wa, wb, h); bwd_pk<0>(acc, nxf, h, L); break;
        case 2: project_pk<1, -1, Ts, CV>(wa, wb, h); fwd_pk(nxf, h, L); break;
        case 3: project_pk<1, +1, Ts, CV>(wa, wb, h); bwd_pk<1>(acc, nxf, h, L); break;
        case 4: project_pk<2, -1, Ts, CV>(wa, wb, h); fwd_pk(nxf, h, L); break;
        case 5: project_pk<2, +1, Ts, CV>(wa, wb, h); bwd_pk<2>(acc, nxf, h, L); break;
        case 6: project_pk<3, -1, Ts, CV>(wa, wb, h); fwd_pk(nxf, h, L); break;
        default: project_pk<3, +1, Ts, CV>(wa, wb, h); bwd_pk<3>(acc, nxf, h, L); break;
      }
    }
    float2 dv[KK];
#pragma unroll
    for (int k = 0; k < KK; k++) dv[k] = make_float2(0.f, 0.f);
    if constexpr (HAS_Y) {
      // cb (H in) + Y in place of acc, one 16-byte chunk of Y at a time
      cp_async_wait<PF - 1>();
      const int slot = slot_of(j, IY);
#pragma unroll
      for (int c = 0; c < CV; c++) {
        float2 yv[VW];
        fetch_pk(slot, c, yv);
#pragma unroll
        for (int k = 0; k < VW; k++) acc[c * VW + k] = fma2(cb, acc[c * VW + k], yv[k]);
      }
      issue_ahead(IntC<IY>{}, j);
    }
    if constexpr (DOT == DOT_TS) {
      // X (= s) and R (= rhat) together, one 16-byte chunk of each at a time:
      // t = ca s + cb (H in) in place of acc, and <t, s>, ||t||^2, ||s||^2, <rhat, s>, <rhat, t>
      cp_async_wait<PF - 2>();
      float2 sr = dv[0], si = dv[0], tt = dv[0], ss = dv[0], qr = dv[0], qi = dv[0], tr = dv[0], ti = dv[0];
      {
        const int xslot = slot_of(j, IX), rslot = slot_of(j, IR);
#pragma unroll
        for (int c = 0; c < CV; c++) {
          float2 xv[VW], rv[VW];
          fetch_pk(xslot, c, xv);
          fetch_pk(rslot, c, rv);
#pragma unroll
          for (int k = 0; k < VW; k++)
            acc[c * VW + k] = HAS_Y ? fma2(ca, xv[k], acc[c * VW + k]) : fma2(cb, acc[c * VW + k], mul2(ca, xv[k]));
#pragma unroll
          for (int k = 0; k < VW; k += 2) {
            const float2 t0 = acc[c * VW + k], t1 = acc[c * VW + k + 1];
            const float2 nt1 = neg2(t1), nr1 = neg2(rv[k + 1]);
            sr = fma2(t0, xv[k], sr); sr = fma2(t1, xv[k + 1], sr);
            si = fma2(t0, xv[k + 1], si); si = fma2(nt1, xv[k], si);
            tt = fma2(t0, t0, tt); tt = fma2(t1, t1, tt);
            ss = fma2(xv[k], xv[k], ss); ss = fma2(xv[k + 1], xv[k + 1], ss);
            qr = fma2(rv[k], xv[k], qr); qr = fma2(rv[k + 1], xv[k + 1], qr);
            qi = fma2(rv[k], xv[k + 1], qi); qi = fma2(nr1, xv[k], qi);
            tr = fma2(rv[k], t0, tr); tr = fma2(rv[k + 1], t1, tr);
            ti = fma2(rv[k], t1, ti); ti = fma2(nr1, t0, ti);
          }
        }
      }
      issue_ahead(IntC<IX>{}, j);
      issue_ahead(IntC<IR>{}, j);
      dv[0] = sr; dv[1] = si; dv[2] = tt; dv[3] = ss; dv[4] = qr; dv[5] = qi; dv[6] = tr; dv[7] = ti;
    } else {
      if constexpr (HAS_X) {
        // out = ca X + cb (H in), in place of acc, one 16-byte chunk of X at a time
        cp_async_wait<PF - 1>();
        const int slot = slot_of(j, IX);
#pragma unroll
        for (int c = 0; c < CV; c++) {
          float2 xv[VW];
          fetch_pk(slot, c, xv);
#pragma unroll
          for (int k = 0; k < VW; k++)
            acc[c * VW + k] = HAS_Y ? fma2(ca, xv[k], acc[c * VW + k]) : fma2(cb, acc[c * VW + k], mul2(ca, xv[k]));
        }
        issue_ahead(IntC<IX>{}, j);
      }
      if constexpr (HAS_R) {
        // <rhat, v>, out = v
        cp_async_wait<PF - 1>();
        float2 sr = dv[0], si = dv[0];
        const int slot = slot_of(j, IR);
#pragma unroll
        for (int c = 0; c < CV; c++) {
          float2 rv[VW];
          fetch_pk(slot, c, rv);
#pragma unroll
          for (int k = 0; k < VW; k += 2) {
            const float2 o0 = acc[c * VW + k], o1 = acc[c * VW + k + 1];
            sr = fma2(rv[k], o0, sr); sr = fma2(rv[k + 1], o1, sr);
            si = fma2(rv[k], o1, si); si = fma2(neg2(rv[k + 1]), o0, si);
          }
        }
        issue_ahead(IntC<IR>{}, j);
        dv[0] = sr; dv[1] = si;
      }
    }
    {
      // store both systems
      Ts* ob = (Ts*)a.out + (size_t)site * rowstride + (size_t)sa * VW;
#pragma unroll
      for (int c = 0; c < CV; c++) {
        float va[VW], vb[VW];
#pragma unroll
        for (int k = 0; k < VW; k++) { va[k] = acc[c * VW + k].x; vb[k] = acc[c * VW + k].y; }
        if (sel_a) store_vec<Ts, float>(ob + c * cstride, va);
        if (sel_b) store_vec<Ts, float>(ob + c * cstride + 16 * VW, vb);
      }
    }
    if constexpr (K > 0) {
      // the block's 8 sites form the 8-site group `chunk`; each value summed in site order
      const int par = j & 1;
#pragma unroll
      for (int k = 0; k < K; k++) {
        dsm[par][ls][k][q] = sel_a ? dv[k].x : 0.f;
        dsm[par][ls][k][q + 16] = sel_b ? dv[k].y : 0.f;
      }
      __syncthreads();
      const int chunk = (int)blockIdx.x + j * G;
#pragma unroll
      for (int r = 0; r < (K * 32 + 127) / 128; r++) {
        const int idx = r * 128 + tid;  // (value k, system) of the group
        const int k = idx >> 5, s = idx & 31;
        const int sys = blockIdx.y * 32 + s;
        if (k < K && sys < sh.N) {
          float acc1 = 0.f;
#pragma unroll
          for (int w = 0; w < 8; w++) acc1 += dsm[par][w][k][s];
          a.partial[((size_t)sys * K + k) * (g.Vh / 8) + chunk] = (double)acc1;
        }
      }
      // dsm[par] is rewritten two chunks later, after the next barrier: no second barrier
    }
    // the next chunk becomes current
    nbc = nbn;
    phc = phn;
    if (j + 2 < nmine) neighbour(site_of(j + 2), nbn, phn);
  }
  cp_async_wait<0>();
}

}  // namespace fs
