// The clover (Sheikholeslami-Wohlert) term of the Wilson-clover operator on the device: the
// per-site table and the site-local passes that apply it to a tile of systems.
//
// Operator: D_sw + sigma = (a + C(x)) - H/2, a = 4 + m + sigma, with the clover term
//   C(x) = (c_sw / 2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
//   sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu],  F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / (8 i),
// Q_{mu nu}(x) the four counter-clockwise plaquettes of the (mu, nu) plane at x. C(x) commutes with
// gamma_5 (DeGrand-Rossi basis, gamma_5 = diag(1, 1, -1, -1)): two Hermitian 6x6 blocks, spins
// {0, 1} and {2, 3}.
//
// Table: each block is eigen-decomposed once per gauge field, C_b = V_b diag(lambda_b) V_b^dag, so
// that for every shift of every system (a + C)^-1 = V diag(1 / (a + lambda)) V^dag and C itself
// are two 6x6 products and a diagonal per block: one table serves all the shifts of a tile.
// Layout: [parity 2][Vh][block 2][CLV_REALS], per block V row-major (36 complex: V[i][j], column j
// the j-th eigenvector) then the 6 eigenvalues.
#pragma once

#include "fs_hop.cuh"

namespace fs {

constexpr int CLV_REALS = 78;  // 72 (V) + 6 (lambda) per chirality block

enum ClovMode {
  CLV_MUL = 0,  // out = C in
  CLV_SUB = 1,  // out = Y - C in
  CLV_INV = 2,  // out = (a + C)^-1 in, a = the system's A = 4 + m + sigma
};

struct ClovArgs {
  void* out;
  const void* in;
  const void* Y;
  const void* table;   // [2][Vh][2][CLV_REALS] in the pass's table type
  const SysState* st;
  const int* gate;     // returns at once if *gate == 0 (nullptr: always run)
  Geom g;
  Shape sh;
  int parity;          // of the sites the fields hold
  int mask;
  int sysmajor;
};

// One site of one system: the two chirality blocks of the spinor v (index 6 spin + 2 colour + re/im).
template <int MODE, typename Tc, typename Tm>
__device__ __forceinline__ void clover_site(const Tc* __restrict__ tab, Tm a, const Tm (&v)[24], Tm (&o)[24]) {
#pragma unroll
  for (int b = 0; b < 2; b++) {
    const Tc* t = tab + b * CLV_REALS;
    // w_j = sum_i conj(V_ij) psi_i, psi_i = spinor entry (spin 2b + i / 3, colour i % 3)
    Tm wr[6], wi[6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
      Tm re = 0, im = 0;
#pragma unroll
      for (int i = 0; i < 6; i++) {
        const Tm vr = (Tm)t[2 * (i * 6 + j)], vi = (Tm)t[2 * (i * 6 + j) + 1];
        const Tm pr = v[12 * b + 2 * i], pi = v[12 * b + 2 * i + 1];
        re = fmadd(vr, pr, re);
        re = fmadd(vi, pi, re);
        im = fmadd(vr, pi, im);
        im = fmadd(-vi, pr, im);
      }
      const Tm lam = (Tm)t[72 + j];
      const Tm f = MODE == CLV_INV ? (Tm)1 / (a + lam) : lam;
      wr[j] = f * re;
      wi[j] = f * im;
    }
    // out_i = sum_j V_ij w_j
#pragma unroll
    for (int i = 0; i < 6; i++) {
      Tm re = 0, im = 0;
#pragma unroll
      for (int j = 0; j < 6; j++) {
        const Tm vr = (Tm)t[2 * (i * 6 + j)], vi = (Tm)t[2 * (i * 6 + j) + 1];
        re = fmadd(vr, wr[j], re);
        re = fmadd(-vi, wi[j], re);
        im = fmadd(vr, wi[j], im);
        im = fmadd(vi, wr[j], im);
      }
      o[12 * b + 2 * i] = re;
      o[12 * b + 2 * i + 1] = im;
    }
  }
}

// The site-local pass over a tile of systems (tile layout) or the selected systems of a
// system-major work list (WL), one parity.
template <typename Ts, typename Tc, typename Tm, int MODE, bool WL>
__global__ void __launch_bounds__(WL ? 128 : 256) clover_kernel(ClovArgs a) {
  if (a.gate != nullptr && *a.gate == 0) return;
  const Shape sh = a.sh;
  const Geom g = a.g;
  const int lsys = threadIdx.x % sh.NB;
  const int lsite = threadIdx.x / sh.NB;
  const Field<Ts> in = make_field<Ts>(const_cast<void*>(a.in), g.Vh, sh.N, WL);
  const Field<Ts> out = make_field<Ts>(a.out, g.Vh, sh.N, WL);
  const Field<Ts> Y = make_field<Ts>(const_cast<void*>(a.Y), g.Vh, sh.N, WL);
  const Tc* table = (const Tc*)a.table;
  auto body = [&](int sys, int chunk) {
    const int site = chunk * sh.SB + lsite;
    if (site >= g.Vh) return;
    Tm v[24], o[24];
    in.load(site, sys, v);
    const Tm A = coef<Tm>(a.st[sys], C_A);
    clover_site<MODE, Tc, Tm>(table + ((size_t)a.parity * g.Vh + site) * 2 * CLV_REALS, A, v, o);
    if constexpr (MODE == CLV_SUB) {
      Tm y[24];
      Y.load(site, sys, y);
#pragma unroll
      for (int k = 0; k < 24; k++) o[k] = y[k] - o[k];
    }
    out.store(site, sys, o);
  };
  if constexpr (!WL) {
    const int sys = blockIdx.y * sh.NB + lsys;
    if (sys >= sh.N || !selected(a.st, sys, a.mask)) return;
    for (int chunk = blockIdx.x; chunk < sh.nchunk; chunk += gridDim.x) body(sys, chunk);
  } else {
    __shared__ int slist[64];
    const int nsel = selected_list(a.st, sh.N, a.mask, slist);
    for (int item = blockIdx.x; item < nsel * sh.nchunk; item += gridDim.x)
      body(slist[item / sh.nchunk], item - (item / sh.nchunk) * sh.nchunk);
  }
}

}  // namespace fs
