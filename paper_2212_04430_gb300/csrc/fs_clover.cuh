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
// that for every shift of every system (a + C)^-1 = V diag(1 / (a + lambda)) V^dag is two 6x6
// products and a diagonal per block: one table serves all the shifts of a tile. C itself is
// applied from its packed Hermitian form (one 6x6 product, 132 multiply-adds per block instead of
// 288). Layout: [parity 2][Vh][block 2][CLV_REALS], per block V row-major (36 complex: V[i][j],
// column j the j-th eigenvector), the 6 eigenvalues, then C_b packed: its 6 (real) diagonal
// entries and its 15 entries above the diagonal, (0,1), (0,2), ..., (0,5), (1,2), ..., (4,5).
#pragma once

#include "fs_hop.cuh"

namespace fs {

constexpr int CLV_REALS = 114;  // 72 (V) + 6 (lambda) + 36 (C packed) per chirality block
constexpr int CLV_C = 78;       // offset of the packed C in a block
constexpr int CLV_PACKED = 36;  // a packed Hermitian 6x6 block (the per-shift inverses)

// index of the upper-triangle entry (i < j) in the packed C (complex entries after the diagonal)
__host__ __device__ constexpr int clv_upper(int i, int j) { return i * 5 - i * (i - 1) / 2 + (j - i - 1); }

enum ClovMode {
  CLV_MUL = 0,      // out = C in
  CLV_SUB = 1,      // out = Y - C in
  CLV_INV = 2,      // out = (a + C)^-1 in, a = the system's A = 4 + m + sigma
  CLV_INV_MUL = 3,  // both site factors of one M-hat in one launch: out = (a + C)^-1 in on `parity`,
                    // out2 = C in2 on the other parity (tile layout)
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
  void* out2;          // CLV_INV_MUL: the C pass's output and input, on the other parity
  const void* in2;
};

// products rounded on their own (never contracted into a neighbouring add), so that the paired
// pass below rounds every lane exactly as this scalar one
__device__ __forceinline__ float mulrn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulrn(double a, double b) { return __dmul_rn(a, b); }

// o = P v for one chirality block (12 reals of v and o), P Hermitian and packed (its 6 real
// diagonal entries, then the 15 above the diagonal): row i is d_i v_i + sum_{j != i} P_ij v_j with
// P_ji = conj(P_ij). C itself, or the packed inverse of one shift.
template <typename Tc, typename Tm>
__device__ __forceinline__ void herm6(const Tc* __restrict__ t, const Tm* v, Tm* o) {
#pragma unroll
  for (int i = 0; i < 6; i++) {
    const Tm d = (Tm)t[i];
    Tm re = mulrn(d, v[2 * i]), im = mulrn(d, v[2 * i + 1]);
#pragma unroll
    for (int j = 0; j < 6; j++) {
      if (j == i) continue;
      const int u = 6 + 2 * (i < j ? clv_upper(i, j) : clv_upper(j, i));
      const Tm cr = (Tm)t[u], ci = i < j ? (Tm)t[u + 1] : -(Tm)t[u + 1];
      const Tm pr = v[2 * j], pi = v[2 * j + 1];
      re = fmadd(cr, pr, re);
      re = fmadd(-ci, pi, re);
      im = fmadd(cr, pi, im);
      im = fmadd(ci, pr, im);
    }
    o[2 * i] = re;
    o[2 * i + 1] = im;
  }
}

// (A + C(x))^-1 v from the packed inverse of the system's shift (the site's two blocks)
template <typename Tc, typename Tm>
__device__ __forceinline__ void clover_site_packed(const Tc* __restrict__ inv, const Tm (&v)[24], Tm (&o)[24]) {
  herm6<Tc, Tm>(inv, v, o);
  herm6<Tc, Tm>(inv + CLV_PACKED, v + 12, o + 12);
}

// One site of one system: the two chirality blocks of the spinor v (index 6 spin + 2 colour + re/im).
template <int MODE, typename Tc, typename Tm>
__device__ __forceinline__ void clover_site(const Tc* __restrict__ tab, Tm a, const Tm (&v)[24], Tm (&o)[24]) {
  if constexpr (MODE != CLV_INV) {
    // o = C v from the packed blocks
    herm6<Tc, Tm>(tab + CLV_C, v, o);
    herm6<Tc, Tm>(tab + CLV_REALS + CLV_C, v + 12, o + 12);
    return;
  }
  // (a + C)^-1 v = V diag(1 / (a + lambda)) V^dag v, one eigenvector (column j of V) at a time:
  // w_j = sum_i conj(V_ij) psi_i, w_j /= a + lambda_j, o_i += V_ij w_j (psi_i: spin 2b + i / 3,
  // colour i % 3), so only one column is live
#pragma unroll
  for (int b = 0; b < 2; b++) {
    const Tc* t = tab + b * CLV_REALS;
    Tm orr[6], oi[6];
#pragma unroll
    for (int i = 0; i < 6; i++) orr[i] = oi[i] = 0;
#pragma unroll
    for (int j = 0; j < 6; j++) {
      Tm vr[6], vi[6];
#pragma unroll
      for (int i = 0; i < 6; i++) {
        vr[i] = (Tm)t[2 * (i * 6 + j)];
        vi[i] = (Tm)t[2 * (i * 6 + j) + 1];
      }
      Tm re = 0, im = 0;
#pragma unroll
      for (int i = 0; i < 6; i++) {
        const Tm pr = v[12 * b + 2 * i], pi = v[12 * b + 2 * i + 1];
        re = fmadd(vr[i], pr, re);
        re = fmadd(vi[i], pi, re);
        im = fmadd(vr[i], pi, im);
        im = fmadd(-vi[i], pr, im);
      }
      const Tm f = (Tm)1 / (a + (Tm)t[72 + j]);
      const Tm wr = mulrn(f, re), wi = mulrn(f, im);
#pragma unroll
      for (int i = 0; i < 6; i++) {
        orr[i] = fmadd(vr[i], wr, orr[i]);
        orr[i] = fmadd(-vi[i], wi, orr[i]);
        oi[i] = fmadd(vr[i], wi, oi[i]);
        oi[i] = fmadd(vi[i], wr, oi[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
      o[12 * b + 2 * i] = orr[i];
      o[12 * b + 2 * i + 1] = oi[i];
    }
  }
}

// herm6 for two systems at once, each lane with its own packed block (t0, t1; the per-shift
// inverses of two shifts): per lane the same operations in the same order as herm6.
__device__ __forceinline__ void herm6_pk2(const float* __restrict__ t0, const float* __restrict__ t1, const float2* v,
                                          float2* o) {
  using namespace pk;
#pragma unroll
  for (int i = 0; i < 6; i++) {
    const float2 d = make_float2(t0[i], t1[i]);
    float2 re = mul2(d, v[2 * i]), im = mul2(d, v[2 * i + 1]);
#pragma unroll
    for (int j = 0; j < 6; j++) {
      if (j == i) continue;
      const int u = 6 + 2 * (i < j ? clv_upper(i, j) : clv_upper(j, i));
      const float2 c2 = make_float2(t0[u], t1[u]);
      const float2 i2 = i < j ? make_float2(t0[u + 1], t1[u + 1]) : make_float2(-t0[u + 1], -t1[u + 1]);
      re = fma2(c2, v[2 * j], re);
      re = fma2(neg2(i2), v[2 * j + 1], re);
      im = fma2(c2, v[2 * j + 1], im);
      im = fma2(i2, v[2 * j], im);
    }
    o[2 * i] = re;
    o[2 * i + 1] = im;
  }
}

// clover_site for two systems of one site at once (the lanes of packed FP32 instructions, the
// table entries broadcast to both): per lane the same operations in the same order as the scalar
// form, so the results are bit-identical to it.
template <int MODE>
__device__ __forceinline__ void clover_site_pk(const float* __restrict__ tab, float2 a, const float2 (&v)[24],
                                               float2 (&o)[24]) {
  using namespace pk;
  if constexpr (MODE != CLV_INV) {
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const float* t = tab + b * CLV_REALS + CLV_C;
#pragma unroll
      for (int i = 0; i < 6; i++) {
        const float2 d = make_float2(t[i], t[i]);
        float2 re = mul2(d, v[12 * b + 2 * i]), im = mul2(d, v[12 * b + 2 * i + 1]);
#pragma unroll
        for (int j = 0; j < 6; j++) {
          if (j == i) continue;
          const int u = 6 + 2 * (i < j ? clv_upper(i, j) : clv_upper(j, i));
          const float cr = t[u], ci = i < j ? t[u + 1] : -t[u + 1];
          const float2 c2 = make_float2(cr, cr), i2 = make_float2(ci, ci), ni2 = make_float2(-ci, -ci);
          const float2 pr = v[12 * b + 2 * j], pi = v[12 * b + 2 * j + 1];
          re = fma2(c2, pr, re);
          re = fma2(ni2, pi, re);
          im = fma2(c2, pi, im);
          im = fma2(i2, pr, im);
        }
        o[12 * b + 2 * i] = re;
        o[12 * b + 2 * i + 1] = im;
      }
    }
    return;
  }
#pragma unroll
  for (int b = 0; b < 2; b++) {
    const float* t = tab + b * CLV_REALS;
    float2 orr[6], oi[6];
#pragma unroll
    for (int i = 0; i < 6; i++) orr[i] = oi[i] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 6; j++) {
      float vr[6], vi[6];
#pragma unroll
      for (int i = 0; i < 6; i++) {
        vr[i] = t[2 * (i * 6 + j)];
        vi[i] = t[2 * (i * 6 + j) + 1];
      }
      float2 re = make_float2(0.f, 0.f), im = re;
#pragma unroll
      for (int i = 0; i < 6; i++) {
        const float2 pr = v[12 * b + 2 * i], pi = v[12 * b + 2 * i + 1];
        re = fma2(make_float2(vr[i], vr[i]), pr, re);
        re = fma2(make_float2(vi[i], vi[i]), pi, re);
        im = fma2(make_float2(vr[i], vr[i]), pi, im);
        im = fma2(make_float2(-vi[i], -vi[i]), pr, im);
      }
      const float lam = t[72 + j];
      const float2 f = make_float2(1.f / (a.x + lam), 1.f / (a.y + lam));
      const float2 wr = mul2(f, re), wi = mul2(f, im);
#pragma unroll
      for (int i = 0; i < 6; i++) {
        orr[i] = fma2(make_float2(vr[i], vr[i]), wr, orr[i]);
        orr[i] = fma2(make_float2(-vi[i], -vi[i]), wi, orr[i]);
        oi[i] = fma2(make_float2(vr[i], vr[i]), wi, oi[i]);
        oi[i] = fma2(make_float2(vi[i], vi[i]), wr, oi[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
      o[12 * b + 2 * i] = orr[i];
      o[12 * b + 2 * i + 1] = oi[i];
    }
  }
}

// The paired pass over a tile of an even number of systems per block row (NB): NB / 2 threads per
// site, each holding systems (2k, 2k + 1) of its row; blockDim.x / (NB / 2) sites per block.
// One site of the paired pass: systems s0, s0 + 1 of fields in / out (MODE != CLV_INV_MUL).
template <typename Ts, int MODE>
__device__ __forceinline__ void clover_pair_site(const ClovArgs& a, const Field<Ts>& in, const Field<Ts>& out,
                                                 const Field<Ts>& Y, int parity, int site, int s0, bool sel0,
                                                 bool sel1, float2 A, const float* inv0, const float* inv1) {
  const Geom& g = a.g;
  float v0[24], v1[24];
  in.load(site, s0, v0);
  in.load(site, s0 + 1, v1);
  float2 v[24], o[24];
#pragma unroll
  for (int k = 0; k < 24; k++) v[k] = make_float2(v0[k], v1[k]);
  if (MODE == CLV_INV && inv0 != nullptr) {
    const size_t off = ((size_t)parity * g.Vh + site) * 2 * CLV_PACKED;
    herm6_pk2(inv0 + off, inv1 + off, v, o);
    herm6_pk2(inv0 + off + CLV_PACKED, inv1 + off + CLV_PACKED, v + 12, o + 12);
  } else {
    clover_site_pk<MODE>((const float*)a.table + ((size_t)parity * g.Vh + site) * 2 * CLV_REALS, A, v, o);
  }
  if constexpr (MODE == CLV_SUB) {
    Y.load(site, s0, v0);
    Y.load(site, s0 + 1, v1);
#pragma unroll
    for (int k = 0; k < 24; k++) o[k] = make_float2(v0[k] - o[k].x, v1[k] - o[k].y);
  }
#pragma unroll
  for (int k = 0; k < 24; k++) { v0[k] = o[k].x; v1[k] = o[k].y; }
  if (sel0) out.store(site, s0, v0);
  if (sel1) out.store(site, s0 + 1, v1);
}

template <typename Ts, int MODE>
__global__ void __launch_bounds__(256, 2) clover_kernel_pk(ClovArgs a) {
  if (a.gate != nullptr && *a.gate == 0) return;
  const Shape sh = a.sh;
  const Geom g = a.g;
  const int P = sh.NB / 2;
  const int pi = threadIdx.x % P, ls = threadIdx.x / P;
  const int S2 = blockDim.x / P;
  const int s0 = blockIdx.y * sh.NB + 2 * pi, s1 = s0 + 1;
  const bool sel0 = selected(a.st, s0, a.mask), sel1 = selected(a.st, s1, a.mask);
  if (!sel0 && !sel1) return;  // no barriers below
  const float2 A = make_float2(sel0 ? coef<float>(a.st[s0], C_A) : 1.f, sel1 ? coef<float>(a.st[s1], C_A) : 1.f);
  const Field<Ts> in = make_field<Ts>(const_cast<void*>(a.in), g.Vh, sh.N, false);
  const Field<Ts> out = make_field<Ts>(a.out, g.Vh, sh.N, false);
  const Field<Ts> Y = make_field<Ts>(const_cast<void*>(a.Y), g.Vh, sh.N, false);
  const Field<Ts> in2 = make_field<Ts>(const_cast<void*>(a.in2), g.Vh, sh.N, false);
  const Field<Ts> out2 = make_field<Ts>(a.out2, g.Vh, sh.N, false);
  // the packed inverses of the two systems' shifts: the systems of one call all have theirs (the
  // autotuner's trial systems none), so where only one is set its partner sits idle and takes
  // the same table, its result discarded
  constexpr bool INV = MODE == CLV_INV || MODE == CLV_INV_MUL;
  const float* inv0 = INV ? a.st[s0].clv_inv32 : nullptr;
  const float* inv1 = INV ? a.st[s1].clv_inv32 : nullptr;
  if (inv0 == nullptr) inv0 = inv1;
  if (inv1 == nullptr) inv1 = inv0;
  const int nchunk2 = (g.Vh + S2 - 1) / S2;
  for (int chunk = blockIdx.x; chunk < nchunk2; chunk += gridDim.x) {
    const int site = chunk * S2 + ls;
    if (site >= g.Vh) continue;
    if constexpr (MODE == CLV_INV_MUL) {
      clover_pair_site<Ts, CLV_INV>(a, in, out, Y, a.parity, site, s0, sel0, sel1, A, inv0, inv1);
      clover_pair_site<Ts, CLV_MUL>(a, in2, out2, Y, 1 - a.parity, site, s0, sel0, sel1, A, nullptr, nullptr);
    } else {
      clover_pair_site<Ts, MODE>(a, in, out, Y, a.parity, site, s0, sel0, sel1, A, inv0, inv1);
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
  const Field<Ts> in2 = make_field<Ts>(const_cast<void*>(a.in2), g.Vh, sh.N, WL);
  const Field<Ts> out2 = make_field<Ts>(a.out2, g.Vh, sh.N, WL);
  const Tc* table = (const Tc*)a.table;
  // one site of one system in mode M (a single-pass mode) on fields fi -> fo of parity par
  auto pass = [&](auto Mc, int sys, int site, const Field<Ts>& fi, const Field<Ts>& fo, int par) {
    constexpr int M = decltype(Mc)::value;
    Tm v[24], o[24];
    fi.load(site, sys, v);
    const Tm A = coef<Tm>(a.st[sys], C_A);
    const Tc* inv = nullptr;  // the packed inverse of the system's shift, where the call built one
    if constexpr (M == CLV_INV) {
      if constexpr (std::is_same<Tc, double>::value) inv = a.st[sys].clv_inv64;
      else inv = a.st[sys].clv_inv32;
    }
    if (inv != nullptr) clover_site_packed<Tc, Tm>(inv + ((size_t)par * g.Vh + site) * 2 * CLV_PACKED, v, o);
    else clover_site<M, Tc, Tm>(table + ((size_t)par * g.Vh + site) * 2 * CLV_REALS, A, v, o);
    if constexpr (M == CLV_SUB) {
      Tm y[24];
      Y.load(site, sys, y);
#pragma unroll
      for (int k = 0; k < 24; k++) o[k] = y[k] - o[k];
    }
    fo.store(site, sys, o);
  };
  auto body = [&](int sys, int chunk) {
    const int site = chunk * sh.SB + lsite;
    if (site >= g.Vh) return;
    if constexpr (MODE == CLV_INV_MUL) {
      pass(IntC<CLV_INV>{}, sys, site, in, out, a.parity);
      pass(IntC<CLV_MUL>{}, sys, site, in2, out2, 1 - a.parity);
    } else {
      pass(IntC<MODE>{}, sys, site, in, out, a.parity);
    }
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
