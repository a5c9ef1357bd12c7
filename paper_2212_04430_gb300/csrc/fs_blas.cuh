// Per-site BiCGStab vector updates over a tile of systems, the per-system
// finalize kernels that turn group partials into the BiCGStab scalars, and the
// reliable-update and initialisation steps.
//
// Mixed precision: vectors r, rhat, p, v, s, t live in the storage type Ts and
// are combined in Tm (FP32 for FP32/FP16/BF16 storage); the iterate x is split
// into x_hi (FP64) + x_lo / scale (Tx). A reliable update folds x_lo into x_hi,
// recomputes r_hi = bhat - M x_hi entirely in FP64 and restarts the sloppy
// residual from it (the search direction p is kept).
//
// One BiCGStab iteration is: v = M p, alpha; s = r - alpha v; t = M s together
// with <t, s>, ||t||^2, ||s||^2, <rhat, s>, <rhat, t>; then omega = <t, s> / ||t||^2
// and, by linearity of r = s - omega t, rho' = <rhat, s> - omega <rhat, t> and
// ||r||^2 = ||s||^2 - 2 Re(conj(omega) <t, s>) + |omega|^2 ||t||^2, so beta is known
// before r exists and one pass updates x, r and p together.
#pragma once

#include "fs_hop.cuh"

namespace fs {

enum BlasOp {
  OP_S = 1,       // s = r - alpha v
  OP_XRP = 2,     // x_lo += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v)
  OP_ACCX = 3,    // x_hi += x_lo / scale ; x_lo = 0 ; with src: src = x_lo / scale for the
                  // systems at an even update k >= 2 (the change the correction residual needs)
  OP_ZEROX = 4,   // x_hi = 0 ; x_lo = 0
  OP_SETR = 5,    // r = scale * src ; on restart/init rhat = p = r, v = 0, else p rescaled ;
                  // <rhat, r>, ||r||^2
  OP_NORM64 = 6,  // ||src||^2 of an FP64 field
  OP_RECON = 7,   // x_hi <- src2 / A + src / (2A): the odd sites x_o = A^-1 (z_o - D_oe x_e) from
                  // src = H_oe x_e of the final FP64 residual (x_hi: the x_o field, src2: z_o)
};

struct BlasArgs {
  void* x_lo;
  void* r;
  void* rhat;
  void* p;
  void* v;
  void* s;
  void* t;
  double* x_hi;
  const double* src;
  const double* src2;
  const SysState* st;
  double* partial;
  const int* gate;
  int Vh;
  Shape sh;
  int mask;
  int sysmajor;  // 1: one system per block row, work items over the selected systems
};

template <typename Tm>
__device__ __forceinline__ void cmul_acc(Tm (&o)[24], const Tm (&a)[24], Tm cr, Tm ci) {
  // o += (cr + i ci) * a
#pragma unroll
  for (int k = 0; k < 24; k += 2) {
    o[k] += cr * a[k] - ci * a[k + 1];
    o[k + 1] += cr * a[k + 1] + ci * a[k];
  }
}

// WL: system-major work-list launch (a.sysmajor); else the tile shape.
template <typename Ts, typename Tx, typename Tm, int OP, bool WL>
__global__ void __launch_bounds__(256) blas_kernel(BlasArgs a) {
  if (a.gate != nullptr && *a.gate == 0) return;
  constexpr int K = OP == OP_SETR ? 3 : (OP == OP_NORM64 ? 1 : 0);
  __shared__ double smem[256 * (K > 0 ? K : 1)];
  const Shape sh = a.sh;
  const int Vh = a.Vh;
  const int lsys = threadIdx.x % sh.NB;
  const int lsite = threadIdx.x / sh.NB;
  const Field<Ts> r = make_field<Ts>(a.r, Vh, sh.N);
  const Field<Ts> rh = make_field<Ts>(a.rhat, Vh, sh.N);
  const Field<Ts> p = make_field<Ts>(a.p, Vh, sh.N);
  const Field<Ts> v = make_field<Ts>(a.v, Vh, sh.N);
  const Field<Ts> s = make_field<Ts>(a.s, Vh, sh.N);
  const Field<Ts> t = make_field<Ts>(a.t, Vh, sh.N);
  const Field<Tx> xl = make_field<Tx>(a.x_lo, Vh, sh.N);
  // x_hi and src (r_hi, bhat, z) are FP64 reliable-update fields: system-major layout
  const Field<double> xh = make_field<double>(a.x_hi, Vh, sh.N, true);
  const Field<double> src = make_field<double>(const_cast<double*>(a.src), Vh, sh.N, true);
  const Field<double> src2 = make_field<double>(const_cast<double*>(a.src2), Vh, sh.N, true);

  // one chunk of sites for system `sys` (sel: the system takes part), block rows sys_base..
  auto chunk_body = [&](const int sys, const int chunk, const bool sel, const int sys_base) {
    Tm c0r = 0, c0i = 0, c1r = 0, c1i = 0, c2r = 0, c2i = 0;
    bool reset = false;
    if (sel) {
      const SysState& st = a.st[sys];
      if (OP == OP_S) { c0r = coef<Tm>(st, C_ALPHA); c0i = coef<Tm>(st, C_ALPHA + 1); }
      if (OP == OP_XRP) { c0r = coef<Tm>(st, C_ALPHA); c0i = coef<Tm>(st, C_ALPHA + 1);
                          c1r = coef<Tm>(st, C_OMEGA); c1i = coef<Tm>(st, C_OMEGA + 1);
                          c2r = coef<Tm>(st, C_BETA); c2i = coef<Tm>(st, C_BETA + 1); }
      if (OP == OP_SETR) { reset = (st.flags & (FLAG_RESTART | FLAG_INIT)) != 0; c0r = coef<Tm>(st, C_RATIO); }
    }
    const int site = chunk * sh.SB + lsite;
    const bool act = sel && site < Vh;
    double dv[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < (K > 0 ? K : 1); k++) dv[k] = 0.0;
    if (act) {
      if constexpr (OP == OP_S) {
        Tm rv[24], vv[24];
        r.load(site, sys, rv); v.load(site, sys, vv);
        cmul_acc(rv, vv, -c0r, -c0i);
        s.store(site, sys, rv);
      } else if constexpr (OP == OP_XRP) {
        Tm xv[24], pv[24], sv[24], tv[24], vv[24];
        xl.load(site, sys, xv); p.load(site, sys, pv); s.load(site, sys, sv);
        t.load(site, sys, tv); v.load(site, sys, vv);
        cmul_acc(xv, pv, c0r, c0i);
        cmul_acc(xv, sv, c1r, c1i);
        xl.store(site, sys, xv);
        cmul_acc(sv, tv, -c1r, -c1i);  // r = s - omega t
        r.store(site, sys, sv);
        Tm rv[24];
        r.load(site, sys, rv);         // the stored (rounded) r, as the next iteration sees it
        cmul_acc(pv, vv, -c1r, -c1i);  // p - omega v
        cmul_acc(rv, pv, c2r, c2i);    // r + beta (p - omega v)
        p.store(site, sys, rv);
      } else if constexpr (OP == OP_ACCX) {
        // on a breakdown the sloppy correction is discarded, never folded into x_hi
        const bool keep = !(a.st[sys].flags & FLAG_RESTART);
        const double isc = a.st[sys].cd[C_INVSCALE];
        const int ku = a.st[sys].updates;
        double hv[24], lv[24];
        xh.load(site, sys, hv); xl.load(site, sys, lv);
        if (a.src != nullptr && ku >= 2 && !(ku & 1) && !(a.st[sys].flags & FLAG_CHECK)) {
          double dx[24];
#pragma unroll
          for (int k = 0; k < 24; k++) dx[k] = keep ? isc * lv[k] : 0.0;
          src.store(site, sys, dx);
        }
#pragma unroll
        for (int k = 0; k < 24; k++) { if (keep) hv[k] += isc * lv[k]; lv[k] = 0.0; }
        xh.store(site, sys, hv); xl.store(site, sys, lv);
      } else if constexpr (OP == OP_RECON) {
        // the epilogue of the reconstruction hop, fma(1/(2A), H_oe x_e, z_o / A), on the stored
        // H_oe x_e: the same rounding, so the same x_o bit for bit
        const double ca = a.st[sys].cd[C_INVA], cb = a.st[sys].cd[C_INV2A];
        double hv[24], zv[24], ov[24];
        src.load(site, sys, hv); src2.load(site, sys, zv);
#pragma unroll
        for (int k = 0; k < 24; k++) ov[k] = fmadd(cb, hv[k], ca * zv[k]);
        xh.store(site, sys, ov);
      } else if constexpr (OP == OP_ZEROX) {
        double z[24];
#pragma unroll
        for (int k = 0; k < 24; k++) z[k] = 0.0;
        xh.store(site, sys, z); xl.store(site, sys, z);
      } else if constexpr (OP == OP_SETR) {
        const double sc = a.st[sys].cd[C_SCALE];
        double sv[24];
        src.load(site, sys, sv);
        Tm iv[24];
        if (!reset) r.load(site, sys, iv);  // the iterated residual, replaced below
        Tm o[24];
#pragma unroll
        for (int k = 0; k < 24; k++) o[k] = (Tm)(sc * sv[k]);
        r.store(site, sys, o);
        // re-read what was stored so the dots see the rounded vector
        Tm ov[24];
        r.load(site, sys, ov);
        Tm hv[24];
        if (reset) {
          // fresh start: rhat = p = r (the first direction), v = 0
          rh.store(site, sys, o);
          p.store(site, sys, o);
#pragma unroll
          for (int k = 0; k < 24; k++) hv[k] = ov[k];
          Tm z[24];
#pragma unroll
          for (int k = 0; k < 24; k++) z[k] = 0;
          v.store(site, sys, z);
        } else {
          // p was formed from the iterated residual r_it in the old scale:
          // p' = ratio (p - r_it) + r' keeps the direction, rescaled, around the new r'
          rh.load(site, sys, hv);
          Tm pv[24];
          p.load(site, sys, pv);
#pragma unroll
          for (int k = 0; k < 24; k++) pv[k] = fmadd(c0r, pv[k] - iv[k], ov[k]);
          p.store(site, sys, pv);
        }
        Tm dr = 0, di = 0, nn = 0;
#pragma unroll
        for (int k = 0; k < 24; k += 2) {
          dr += hv[k] * ov[k] + hv[k + 1] * ov[k + 1];
          di += hv[k] * ov[k + 1] - hv[k + 1] * ov[k];
          nn += ov[k] * ov[k] + ov[k + 1] * ov[k + 1];
        }
        dv[0] = (double)dr; dv[1] = (double)di; dv[2] = (double)nn;
      } else if constexpr (OP == OP_NORM64) {
        double sv[24];
        src.load(site, sys, sv);
        double nn = 0;
#pragma unroll
        for (int k = 0; k < 24; k++) nn += sv[k] * sv[k];
        dv[0] = nn;
      }
    }
    if constexpr (K > 0) {
      group_partials<K>(dv, lsite, lsys, sys_base, sh, Vh, chunk, smem, a.partial);
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

// ---- CGNR fallback (FP64) ------------------------------------------------------
// A system BiCGStab could not solve (breakdowns past the restart limit, or
// max_iter) is re-solved by conjugate gradients on the normal equations
// M^dag M x = M^dag bhat, with M^dag = gamma5 M gamma5 (gamma5-hermiticity of the
// Wilson operator carries over to the even-odd Schur complement). CG on a
// Hermitian positive definite operator cannot break down. The residual of the
// original system, s = bhat - M x, is carried along (s -= alpha q) to decide
// convergence, and replaced by the true FP64 residual every 64 iterations and at
// apparent convergence.
enum CgOp {
  CG_XS = 0,  // x += alpha p ; s -= alpha q ; ||s||^2
  CG_G5 = 1,  // g = gamma5 s
  CG_R = 2,   // r = gamma5 w ; ||r||^2
  CG_P = 3,   // p = r + beta p
  CG_P0 = 4,  // p = r
};

struct CgArgs {
  double *x, *s, *p, *q, *g, *w, *r;
  const SysState* st;
  double* partial;
  int Vh;
  Shape sh;
  int mask;
};

template <int OP>
__global__ void __launch_bounds__(256) cg_kernel(CgArgs a) {
  constexpr int K = (OP == CG_XS || OP == CG_R) ? 1 : 0;
  __shared__ double smem[256];
  const Shape sh = a.sh;
  const int lsite = threadIdx.x;  // system-major: NB = 1
  const Field<double> fx = make_field<double>(a.x, a.Vh, sh.N, true), fs = make_field<double>(a.s, a.Vh, sh.N, true);
  const Field<double> fp = make_field<double>(a.p, a.Vh, sh.N, true), fq = make_field<double>(a.q, a.Vh, sh.N, true);
  const Field<double> fg = make_field<double>(a.g, a.Vh, sh.N, true), fw = make_field<double>(a.w, a.Vh, sh.N, true);
  const Field<double> fr = make_field<double>(a.r, a.Vh, sh.N, true);
  // work items (k-th system in the fallback, chunk)
  __shared__ int slist[64];
  const int nsel = selected_list(a.st, sh.N, a.mask, slist);
  for (int item = blockIdx.x; item < nsel * sh.nchunk; item += gridDim.x) {
    const int sys = slist[item / sh.nchunk];
    const int chunk = item - (item / sh.nchunk) * sh.nchunk;
    const double alpha = a.st[sys].cd[C_ALPHA];
    const double beta = a.st[sys].cd[C_BETA];
    const int site = chunk * sh.SB + lsite;
    const bool act = site < a.Vh;
    double dv[1] = {0.0};
    if (act) {
      double u[24], v[24];
      if constexpr (OP == CG_XS) {
        fx.load(site, sys, u); fp.load(site, sys, v);
#pragma unroll
        for (int k = 0; k < 24; k++) u[k] = fma(alpha, v[k], u[k]);
        fx.store(site, sys, u);
        fs.load(site, sys, u); fq.load(site, sys, v);
#pragma unroll
        for (int k = 0; k < 24; k++) u[k] = fma(-alpha, v[k], u[k]);
        fs.store(site, sys, u);
#pragma unroll
        for (int k = 0; k < 24; k++) dv[0] = fma(u[k], u[k], dv[0]);
      } else if constexpr (OP == CG_G5 || OP == CG_R) {
        // gamma5 = diag(1, 1, -1, -1) in spin (DeGrand-Rossi): negate spin components 2, 3
        (OP == CG_G5 ? fs : fw).load(site, sys, u);
#pragma unroll
        for (int k = 12; k < 24; k++) u[k] = -u[k];
        (OP == CG_G5 ? fg : fr).store(site, sys, u);
        if constexpr (OP == CG_R) {
#pragma unroll
          for (int k = 0; k < 24; k++) dv[0] = fma(u[k], u[k], dv[0]);
        }
      } else if constexpr (OP == CG_P) {
        fr.load(site, sys, u); fp.load(site, sys, v);
#pragma unroll
        for (int k = 0; k < 24; k++) u[k] = fma(beta, v[k], u[k]);
        fp.store(site, sys, u);
      } else {
        fr.load(site, sys, u);
        fp.store(site, sys, u);
      }
    }
    if constexpr (K > 0) group_partials<K>(dv, lsite, 0, sys, sh, a.Vh, chunk, smem, a.partial);
  }
}

// ---- finalize: one block per system sums its group partials in fixed order ----
enum FinOp { FIN_ALPHA = 0, FIN_OMEGA = 1, FIN_TRUE = 3, FIN_UPDATE = 4, FIN_INIT = 5,
             FIN_NORM = 6, FIN_VERIFY = 7, FIN_CG_INIT = 8, FIN_CG_ALPHA = 9, FIN_CG_BETA = 10,
             FIN_CG_TRUE = 11 };

constexpr int FIN_SPLIT = 8;  // blocks per system in a finalize
constexpr int FIN_MAXV = 8;   // summed values per system, at most

struct FinArgs {
  SysState* st;
  double* slice;     // [N][FIN_SPLIT][FIN_MAXV] slice sums
  unsigned* count;   // [N] arrival tickets, zero between finalizes
  const double* pa;  // partials [N][K][ngroups]
  const double* pb;
  const double* pc;
  int* gate;
  int N;
  int ngroups;
  int mask;
  double target;     // rms target of the scaled residual entries
  double nreal;      // 24 * Vh
  int max_restarts;
  int first_approx;  // a system's first reliable update took its true residual in FP32
  int hx_kept;       // the FP64 scratch of a converged system is kept until its harvest
};

__device__ __forceinline__ void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
  const double d = br * br + bi * bi;
  cr = (ar * br + ai * bi) / d;
  ci = (ai * br - ar * bi) / d;
}

__device__ __forceinline__ void set_coef(SysState& s, int k, double val) {
  s.cd[k] = val;
  s.cf[k] = (float)val;
}

__device__ __forceinline__ void set_beta(SysState& s) {
  // beta = (rho / rho_old) (alpha / omega)
  double q1r, q1i, q2r, q2i;
  if (s.omega[0] == 0.0 && s.omega[1] == 0.0) {
    set_coef(s, C_BETA, 0.0); set_coef(s, C_BETA + 1, 0.0);
    return;
  }
  cdiv(s.rho[0], s.rho[1], s.rho_old[0], s.rho_old[1], q1r, q1i);
  cdiv(s.alpha[0], s.alpha[1], s.omega[0], s.omega[1], q2r, q2i);
  set_coef(s, C_BETA, q1r * q2r - q1i * q2i);
  set_coef(s, C_BETA + 1, q1r * q2i + q1i * q2r);
}

// Values a finalize op sums per system (all its sources together).
__host__ __device__ constexpr int fin_values(int op) {
  return op == FIN_ALPHA ? 2
       : op == FIN_OMEGA ? 8
       : (op == FIN_UPDATE || op == FIN_INIT || op == FIN_NORM) ? 3
       : (op == FIN_VERIFY || op == FIN_CG_INIT || op == FIN_CG_BETA) ? 2
       : 1;
}

// Operands summed by each finalize op, in the order its logic consumes them.
__device__ __forceinline__ int fin_sources(int op, const FinArgs& a, const double* (&p)[3], int (&k)[3]) {
  switch (op) {
    case FIN_ALPHA: p[0] = a.pa; k[0] = 2; return 1;
    case FIN_OMEGA: p[0] = a.pa; k[0] = 8; return 1;
    case FIN_UPDATE: case FIN_INIT: p[0] = a.pa; k[0] = 3; return 1;
    case FIN_NORM: p[0] = a.pa; p[1] = a.pb; p[2] = a.pc; k[0] = k[1] = k[2] = 1; return 3;
    case FIN_VERIFY: case FIN_CG_INIT: case FIN_CG_BETA: p[0] = a.pa; p[1] = a.pb; k[0] = k[1] = 1; return 2;
    default: p[0] = a.pa; k[0] = 1; return 1;  // FIN_TRUE, FIN_CG_ALPHA, FIN_CG_TRUE
  }
}

template <int K>
__device__ __forceinline__ void take(double (&v)[K], const double* tot, int& off) {
#pragma unroll
  for (int k = 0; k < K; k++) v[k] = tot[off + k];
  off += K;
}

// The per-system scalar step of the solver (one thread) from the summed operands.
__device__ __forceinline__ void fin_logic(const FinArgs& a, int op, SysState& s, const double* tot) {
  int off = 0;
  if (op == FIN_ALPHA) {
    double rv[2];
    take<2>(rv, tot, off);
    if (threadIdx.x == 0) {
      double ar = 0, ai = 0;
      if (rv[0] == 0.0 && rv[1] == 0.0) {
        s.flags |= FLAG_UPDATE | FLAG_RESTART;
      } else {
        cdiv(s.rho[0], s.rho[1], rv[0], rv[1], ar, ai);
        if (!isfinite(ar) || !isfinite(ai)) { ar = ai = 0; s.flags |= FLAG_UPDATE | FLAG_RESTART; }
      }
      if ((s.flags & FLAG_RESTART) && a.gate) atomicExch(a.gate, 1);
      s.alpha[0] = ar; s.alpha[1] = ai;
      set_coef(s, C_ALPHA, ar); set_coef(s, C_ALPHA + 1, ai);
    }
  } else if (op == FIN_OMEGA) {
    // v = <t, s>, ||t||^2, ||s||^2, <rhat, s>, <rhat, t>
    double v[8];
    take<8>(v, tot, off);
    if (threadIdx.x == 0) {
      double wr = 0, wi = 0;
      if (v[2] > 0.0 && isfinite(v[2])) { wr = v[0] / v[2]; wi = v[1] / v[2]; }
      else s.flags |= FLAG_UPDATE | FLAG_RESTART;
      s.omega[0] = wr; s.omega[1] = wi;
      set_coef(s, C_OMEGA, wr); set_coef(s, C_OMEGA + 1, wi);
      if (!(s.flags & FLAG_RESTART)) {
        // r = s - omega t: rho' = <rhat, s> - omega <rhat, t>,
        // ||r||^2 = ||s||^2 - 2 Re(conj(omega) <t, s>) + |omega|^2 ||t||^2
        s.iters += 1;
        s.rho_old[0] = s.rho[0]; s.rho_old[1] = s.rho[1];
        s.rho[0] = v[4] - (wr * v[6] - wi * v[7]);
        s.rho[1] = v[5] - (wr * v[7] + wi * v[6]);
        const double r2 = v[3] - 2.0 * (wr * v[0] + wi * v[1]) + (wr * wr + wi * wi) * v[2];
        s.r2 = r2 > 0.0 ? r2 : 0.0;
        set_beta(s);
        const double isc = s.cd[C_INVSCALE];
        const double r2hi = s.r2 * isc * isc;
        if (!isfinite(r2) || !isfinite(s.rho[0]) || !isfinite(s.rho[1])) s.flags |= FLAG_UPDATE | FLAG_RESTART;
        // below this the recurrence for ||r||^2 has lost most of its digits: ask FP64
        if (!(r2 > 1e-5 * v[3])) s.flags |= FLAG_UPDATE | FLAG_CHECK;
        if (r2hi <= s.tol2) s.flags |= FLAG_UPDATE | FLAG_CHECK;
        if (s.r2 < s.delta2 * s.r2_max) s.flags |= FLAG_UPDATE;
        if (s.iters >= s.max_iter) s.flags |= FLAG_UPDATE | FLAG_FINAL | FLAG_CHECK;
        if (s.r2 > s.r2_max) s.r2_max = s.r2;
      }
      if ((s.flags & FLAG_UPDATE) && a.gate) atomicExch(a.gate, 1);
    }
  } else if (op == FIN_TRUE) {
    double v[1];
    take<1>(v, tot, off);
    if (threadIdx.x == 0) {
      // an FP32-arithmetic residual (update 0, or a correction at an even update k >= 2) restarts
      // the iteration but never decides convergence: a system below tol goes on and its next
      // update, a full FP64 residual, checks it
      const bool approx = a.first_approx && !(s.updates & 1) && !(s.flags & FLAG_CHECK);
      s.r2_true = v[0];
      s.updates += 1;
      if (v[0] <= s.tol2 && !approx) {
        s.status = SYS_CONVERGED;
        s.flags = a.hx_kept ? FLAG_HX : 0;  // the FP64 hop just left H_oe x_e in the scratch
      } else if ((s.flags & FLAG_FINAL) || !isfinite(v[0]) ||
                 ((s.flags & FLAG_RESTART) && s.restarts >= a.max_restarts)) {
        s.status = SYS_NOCONV;
        s.flags = 0;
      } else {
        const double sc = a.target * sqrt(a.nreal / fmax(v[0], 1e-300));
        set_coef(s, C_RATIO, sc * s.cd[C_INVSCALE]);
        set_coef(s, C_SCALE, sc);
        set_coef(s, C_INVSCALE, 1.0 / sc);
      }
    }
  } else if (op == FIN_UPDATE || op == FIN_INIT) {
    double v[3];
    take<3>(v, tot, off);
    if (threadIdx.x == 0) {
      s.rho[0] = v[0]; s.rho[1] = v[1];
      s.r2 = v[2];
      s.r2_max = v[2];
      if (s.flags & (FLAG_RESTART | FLAG_INIT)) {
        if (s.flags & FLAG_RESTART) s.restarts += 1;
        s.rho_old[0] = 1.0; s.rho_old[1] = 0.0;
        s.alpha[0] = 1.0; s.alpha[1] = 0.0;
        s.omega[0] = 1.0; s.omega[1] = 0.0;
        set_coef(s, C_BETA, 0.0); set_coef(s, C_BETA + 1, 0.0);
        set_coef(s, C_OMEGA, 1.0); set_coef(s, C_OMEGA + 1, 0.0);
      }
      // (beta of the next iteration comes from FIN_OMEGA; p was rescaled by OP_SETR)
      s.flags = 0;
    }
  } else if (op == FIN_NORM) {
    // initial norms: pa = ||bhat||^2, pb = ||z_e||^2, pc = ||z_o||^2
    double bh[1], ze[1], zo[1];
    take<1>(bh, tot, off);
    take<1>(ze, tot, off);
    take<1>(zo, tot, off);
    if (threadIdx.x == 0) {
      s.b2 = ze[0] + zo[0];
      s.r2_true = bh[0];
      s.iters = 0; s.updates = 0; s.restarts = 0;
      if (s.b2 == 0.0 || bh[0] <= s.tol2 * s.b2) {
        // zero right-hand side (or already solved by x = 0)
        s.tol2 = s.tol2 * s.b2;
        s.status = SYS_CONVERGED;
        s.flags = 0;
      } else {
        s.tol2 = s.tol2 * s.b2;  // host stored tol^2; make it absolute
        s.status = SYS_ACTIVE;
        const double sc = a.target * sqrt(a.nreal / bh[0]);
        set_coef(s, C_SCALE, sc);
        set_coef(s, C_INVSCALE, 1.0 / sc);
      }
    }
  } else if (op == FIN_VERIFY) {
    double e[1], o[1];
    take<1>(e, tot, off);
    take<1>(o, tot, off);
    if (threadIdx.x == 0) s.r2_full = e[0] + o[0];
  } else if (op == FIN_CG_INIT) {
    // pa = ||s||^2 (s = bhat - M x), pb = ||r||^2 (r = M^dag s)
    double sv[1], rv[1];
    take<1>(sv, tot, off);
    take<1>(rv, tot, off);
    if (threadIdx.x == 0) {
      s.r2_true = sv[0];
      s.r2 = sv[0];
      s.rho[0] = rv[0]; s.rho[1] = 0.0;
      s.cg_iters = 0;
      if (sv[0] <= s.tol2) { s.status = SYS_CONVERGED; s.flags = 0; }
      else if (!(rv[0] > 0.0) || !isfinite(rv[0]) || !isfinite(sv[0])) { s.status = SYS_NOCONV; s.flags = 0; }
      else s.flags = FLAG_CG;
    }
  } else if (op == FIN_CG_ALPHA) {
    double qv[1];
    take<1>(qv, tot, off);  // ||M p||^2
    if (threadIdx.x == 0) {
      const double al = s.rho[0] / qv[0];
      if (!(qv[0] > 0.0) || !isfinite(al)) { s.status = SYS_NOCONV; s.flags = 0; }
      s.alpha[0] = al; s.alpha[1] = 0.0;
      set_coef(s, C_ALPHA, al); set_coef(s, C_ALPHA + 1, 0.0);
    }
  } else if (op == FIN_CG_BETA) {
    // pa = ||s||^2 after the step, pb = ||r||^2 of the new normal residual
    double sv[1], rv[1];
    take<1>(sv, tot, off);
    take<1>(rv, tot, off);
    if (threadIdx.x == 0) {
      s.cg_iters += 1;
      s.r2 = sv[0];
      const double be = rv[0] / s.rho[0];
      s.rho_old[0] = s.rho[0];
      s.rho[0] = rv[0];
      set_coef(s, C_BETA, be); set_coef(s, C_BETA + 1, 0.0);
      if (!isfinite(be) || !isfinite(sv[0])) { s.status = SYS_NOCONV; s.flags = 0; }
      else {
        if (sv[0] <= s.tol2 || (s.cg_iters & 63) == 0 || s.cg_iters >= s.cg_max_iter) s.flags |= FLAG_UPDATE;
        if (s.cg_iters >= s.cg_max_iter) s.flags |= FLAG_FINAL;
      }
    }
  } else if (op == FIN_CG_TRUE) {
    double tv[1];
    take<1>(tv, tot, off);  // ||bhat - M x||^2 in FP64; s now holds that residual
    if (threadIdx.x == 0) {
      s.r2_true = tv[0];
      s.r2 = tv[0];
      s.updates += 1;
      if (tv[0] <= s.tol2) { s.status = SYS_CONVERGED; s.flags = 0; }
      else if ((s.flags & FLAG_FINAL) || !isfinite(tv[0])) { s.status = SYS_NOCONV; s.flags = 0; }
      else s.flags &= ~FLAG_UPDATE;
    }
  }
}

#ifdef FS_ENGINE_KERNELS
// Grid (N, FIN_SPLIT): block (sys, y) sums slice y of the system's group partials
// (fixed slices, fixed in-slice tree) into a.slice; the last block of the system to
// finish (an atomic ticket; no block ever waits) adds the FIN_SPLIT slice sums in slice
// order and runs the scalar step. The result depends only on the partials, not on
// which block finishes last. NV = fin_values(op).
template <int NV>
__global__ void __launch_bounds__(256) fin_kernel(FinArgs a, int op) {
  __shared__ double sm[256 * NV];
  __shared__ unsigned ticket;
  const int sys = blockIdx.x, y = blockIdx.y;
  if (op == FIN_UPDATE && sys == 0 && y == 0 && threadIdx.x == 0 && a.gate) {
    // every gated update kernel of this iteration has run (stream order); re-arm
    *a.gate = 0;
  }
  if (sys >= a.N || !selected(a.st, sys, a.mask)) return;
  const double* src[3];
  int kk[3] = {0, 0, 0};
  fin_sources(op, a, src, kk);
  const int g0 = (int)((long long)a.ngroups * y / FIN_SPLIT), g1 = (int)((long long)a.ngroups * (y + 1) / FIN_SPLIT);
  double acc[NV];
  const double* base[NV];
#pragma unroll
  for (int v = 0; v < NV; v++) {
    // value v: entry kidx of source q (sources in order, kk[q] entries each)
    int q = 0, kidx = v;
    if (kidx >= kk[0]) { kidx -= kk[0]; q = 1; if (kidx >= kk[1]) { kidx -= kk[1]; q = 2; } }
    const double* sp = q == 0 ? src[0] : (q == 1 ? src[1] : src[2]);
    const int kq = q == 0 ? kk[0] : (q == 1 ? kk[1] : kk[2]);
    base[v] = sp + ((size_t)sys * kq + kidx) * a.ngroups;
    acc[v] = 0.0;
  }
  // each value summed over this thread's groups in ascending order, the NV loads of a group
  // issued together
  for (int g = g0 + (int)threadIdx.x; g < g1; g += blockDim.x) {
#pragma unroll
    for (int v = 0; v < NV; v++) acc[v] += base[v][g];
  }
#pragma unroll
  for (int v = 0; v < NV; v++) sm[threadIdx.x * NV + v] = acc[v];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int v = 0; v < NV; v++) sm[threadIdx.x * NV + v] += sm[(threadIdx.x + w) * NV + v];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; v++) a.slice[((size_t)sys * FIN_SPLIT + y) * FIN_MAXV + v] = sm[v];
    __threadfence();
    ticket = atomicAdd(&a.count[sys], 1u);
  }
  __syncthreads();
  if (ticket != FIN_SPLIT - 1) return;
  // the last block: thread v adds value v's FIN_SPLIT slice sums in slice order
  __shared__ double tsum[FIN_MAXV];
  __threadfence();
  if (threadIdx.x < NV) {
    const int v = threadIdx.x;
    double t = 0.0;
#pragma unroll
    for (int yy = 0; yy < FIN_SPLIT; yy++)
      t += __ldcg(&a.slice[((size_t)sys * FIN_SPLIT + yy) * FIN_MAXV + v]);  // L2: other SMs wrote them
    tsum[v] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  a.count[sys] = 0;  // re-armed for the next finalize of this system
  double tot[FIN_MAXV];
#pragma unroll
  for (int v = 0; v < FIN_MAXV; v++) tot[v] = v < NV ? tsum[v] : 0.0;
  fin_logic(a, op, a.st[sys], tot);
}
#endif  // FS_ENGINE_KERNELS

}  // namespace fs
