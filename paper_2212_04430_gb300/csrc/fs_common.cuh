// Shared device-side definitions for the FS-MLMC CUDA path: lattice geometry in
// even-odd (checkerboard) order, storage precisions with 16-byte vector access,
// complex arithmetic, and the per-system solver state.
//
// Field layout on the device (one parity, a tile of N systems):
//   real index = ((c * Vh + site) * N + sys) * VW + v,   c in [0, 24/VW), v in [0, VW)
// where VW = 16 / sizeof(storage real) reals form one 16-byte vector. Consecutive
// threads take consecutive (site, sys) pairs with sys fastest, so every vector load
// of a warp is contiguous for any N, and with N >= 32 a warp covers one site.
// The 24 reals of a spinor are ordered [spin 4][colour 3][re, im].
//
// Gauge layout: [parity 2][mu 4][Vh][RP] reals, RP = 18 (or 12 compressed)
// rounded up to whole 16-byte vectors; U_mu(x) of a site is stored with that site.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace fs {

enum Prec { PREC_F64 = 0, PREC_F32 = 1, PREC_F16 = 2, PREC_BF16 = 3 };

// Unsigned division by a runtime constant d >= 1 through a multiply-high and a shift
// (Granlund & Montgomery, PLDI'94): q = (hi32(n * mul) + n) >> shift with
// shift = ceil(log2 d) and mul = floor(2^32 (2^shift - d) / d) + 1, exact for n < 2^31.
struct FastDiv {
  uint32_t d, mul, shift;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t s = 0;
  while ((1ull << s) < d) s++;
  f.shift = s;
  f.mul = (uint32_t)(((1ull << 32) * ((1ull << s) - d)) / d + 1);
  return f;
}
__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const uint32_t hi = __umulhi(n, f.mul);
#else
  const uint32_t hi = (uint32_t)(((uint64_t)n * f.mul) >> 32);
#endif
  return (uint32_t)(((uint64_t)hi + n) >> f.shift);
}

struct Geom {
  int L[4];  // Lx, Ly, Lz, Lt
  int Lh0;   // Lx / 2
  int Vh;    // sites per parity
  int V;     // all sites
  int bc_t;  // +1 periodic, -1 antiperiodic in t
  FastDiv dLh0, dL1, dL2;  // reciprocals of Lx/2, Ly, Lz for the checkerboard coordinates
};

inline void geom_init_div(Geom& g) {
  g.dLh0 = make_fastdiv((uint32_t)g.Lh0);
  g.dL1 = make_fastdiv((uint32_t)g.L[1]);
  g.dL2 = make_fastdiv((uint32_t)g.L[2]);
}

// Coordinates of checkerboard site i of parity p (parity = (x+y+z+t) & 1).
__device__ __forceinline__ void cb_coords(const Geom& g, int p, int i, int x[4]) {
  const uint32_t r0 = fdiv((uint32_t)i, g.dLh0);
  const int xh = i - (int)r0 * g.Lh0;
  const uint32_t r1 = fdiv(r0, g.dL1);
  x[1] = (int)r0 - (int)r1 * g.L[1];
  const uint32_t r2 = fdiv(r1, g.dL2);
  x[2] = (int)r1 - (int)r2 * g.L[2];
  x[3] = (int)r2;
  x[0] = 2 * xh + ((x[1] + x[2] + x[3] + p) & 1);
}

__device__ __forceinline__ int cb_index(const Geom& g, const int x[4]) {
  return (x[0] >> 1) + g.Lh0 * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
}

__device__ __forceinline__ int lex_index(const Geom& g, const int x[4]) {
  return x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
}

// ---- storage precisions --------------------------------------------------
template <typename T> struct Store;
template <> struct Store<double> { static constexpr int VW = 2; using vec = double2; };
template <> struct Store<float> { static constexpr int VW = 4; using vec = float4; };
template <> struct Store<__half> { static constexpr int VW = 8; using vec = uint4; };
template <> struct Store<__nv_bfloat16> { static constexpr int VW = 8; using vec = uint4; };

template <typename Tm> __device__ __forceinline__ void unpack(const double2& w, Tm* o) {
  o[0] = (Tm)w.x; o[1] = (Tm)w.y;
}
template <typename Tm> __device__ __forceinline__ void unpack(const float4& w, Tm* o) {
  o[0] = (Tm)w.x; o[1] = (Tm)w.y; o[2] = (Tm)w.z; o[3] = (Tm)w.w;
}
template <typename Ts, typename Tm> struct Unpack16;
template <typename Tm> struct Unpack16<__half, Tm> {
  static __device__ __forceinline__ void run(const uint4& w, Tm* o) {
    const __half2* h = reinterpret_cast<const __half2*>(&w);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float2 f = __half22float2(h[k]);
      o[2 * k] = (Tm)f.x; o[2 * k + 1] = (Tm)f.y;
    }
  }
};
template <typename Tm> struct Unpack16<__nv_bfloat16, Tm> {
  static __device__ __forceinline__ void run(const uint4& w, Tm* o) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      float2 f = __bfloat1622float2(h[k]);
      o[2 * k] = (Tm)f.x; o[2 * k + 1] = (Tm)f.y;
    }
  }
};

template <typename Ts, typename Tm>
__device__ __forceinline__ void load_vec(const Ts* p, Tm* o) {
  if constexpr (sizeof(Ts) == 2) {
    Unpack16<Ts, Tm>::run(*reinterpret_cast<const uint4*>(p), o);
  } else {
    unpack<Tm>(*reinterpret_cast<const typename Store<Ts>::vec*>(p), o);
  }
}

template <typename Ts, typename Tm>
__device__ __forceinline__ void store_vec(Ts* p, const Tm* o) {
  if constexpr (sizeof(Ts) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2((double)o[0], (double)o[1]);
  } else if constexpr (sizeof(Ts) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
  } else {
    uint4 w;
    if constexpr (std::is_same<Ts, __half>::value) {
      __half2* h = reinterpret_cast<__half2*>(&w);
#pragma unroll
      for (int k = 0; k < 4; k++) h[k] = __floats2half2_rn((float)o[2 * k], (float)o[2 * k + 1]);
    } else {
      __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
      for (int k = 0; k < 4; k++) h[k] = __floats2bfloat162_rn((float)o[2 * k], (float)o[2 * k + 1]);
    }
    *reinterpret_cast<uint4*>(p) = w;
  }
}

// A field view: one parity of a tile of N systems. Two layouts:
//  tile         ((c Vh + site) N + sys) VW + v : a warp's consecutive (site, sys) pairs,
//               system fastest, read 128-bit contiguous; for kernels that work on all
//               systems of a site together (the inner-precision solver);
//  system-major ((sys 24/VW + c) Vh + site) VW + v : one system's parity is contiguous;
//               for kernels that run one system per block (the FP64 reliable-update,
//               preparation, reconstruction and contraction fields), where a few flagged
//               systems must not drag the other systems' interleaved data through DRAM.
template <typename Ts>
struct Field {
  Ts* ptr;
  size_t cstride;    // reals between vector slots c and c+1
  size_t sitestride; // reals between consecutive sites
  size_t sysstride;  // reals between consecutive systems
  int N;
  __device__ __forceinline__ size_t off(int site, int sys) const {
    return (size_t)site * sitestride + (size_t)sys * sysstride;
  }
  template <typename Tm>
  __device__ __forceinline__ void load(int site, int sys, Tm (&v)[24]) const {
    constexpr int VW = Store<Ts>::VW;
    const Ts* b = ptr + off(site, sys);
#pragma unroll
    for (int c = 0; c < 24 / VW; c++) load_vec<Ts, Tm>(b + c * cstride, v + c * VW);
  }
  template <typename Tm>
  __device__ __forceinline__ void store(int site, int sys, const Tm (&v)[24]) const {
    constexpr int VW = Store<Ts>::VW;
    Ts* b = ptr + off(site, sys);
#pragma unroll
    for (int c = 0; c < 24 / VW; c++) store_vec<Ts, Tm>(b + c * cstride, v + c * VW);
  }
};

template <typename Ts>
__host__ __device__ inline Field<Ts> make_field(void* p, int Vh, int N, bool sysmajor = false) {
  constexpr int VW = Store<Ts>::VW;
  Field<Ts> f;
  f.ptr = reinterpret_cast<Ts*>(p);
  f.N = N;
  if (sysmajor) {
    f.cstride = (size_t)Vh * VW;
    f.sitestride = VW;
    f.sysstride = (size_t)24 * Vh;
  } else {
    f.cstride = (size_t)Vh * N * VW;
    f.sitestride = (size_t)N * VW;
    f.sysstride = VW;
  }
  return f;
}

// Reals per stored link, padded to whole 16-byte vectors.
template <typename Tg> __host__ __device__ constexpr int link_pad(int nr) {
  return ((nr + Store<Tg>::VW - 1) / Store<Tg>::VW) * Store<Tg>::VW;
}

// ---- per-system solver state (device resident, one entry per tile slot) ----
enum SysStatus { SYS_IDLE = 0, SYS_ACTIVE = 1, SYS_CONVERGED = 2, SYS_NOCONV = 3 };
// FLAG_CG: the system is in the CGNR fallback; FLAG_HPE: a finished system whose solution takes
// the hopping parameter expansion's kappa H applications before its contraction; FLAG_CHECK: the
// update may end the solve (sloppy residual at tol, or max_iter), so its residual is full FP64;
// FLAG_HX: a converged system whose FP64 scratch still holds H_oe x_e of its final residual, so the
// odd sites follow from it without another hop
enum SysFlags { FLAG_UPDATE = 1, FLAG_RESTART = 2, FLAG_FINAL = 4, FLAG_INIT = 8, FLAG_HARVEST = 16,
                FLAG_CG = 32, FLAG_HPE = 64, FLAG_CHECK = 128, FLAG_HX = 256 };

// Indices into SysState::cd / cf.
enum CoefIdx {
  C_A = 0,        // A = 4 + m + sigma
  C_MINV4A = 1,   // -1 / (4A)
  C_INV2A = 2,    // 1 / (2A)
  C_INVA = 3,     // 1 / A
  C_INV4A = 4,    // 1 / (4A)
  C_ALPHA = 5,    // alpha (re, im)
  C_BETA = 7,     // beta (re, im)
  C_OMEGA = 9,    // omega (re, im)
  C_SCALE = 11,   // r_lo = scale * r_hi
  C_INVSCALE = 12,
  C_MINVA = 13,   // -A
  C_RATIO = 14    // new scale / old scale of the last reliable update
};

struct SysState {
  double sigma, A, inv4A;     // shift, A = 4 + m + sigma, 1 / (4 A)
  double rho[2];              // <rhat, r> of the current residual (complex)
  double rho_old[2];          // rho of the previous iteration
  double alpha[2], omega[2];  // BiCGStab step sizes (complex)
  double r2;                  // ||r_lo||^2 (scaled units)
  double r2_max;              // max ||r_lo||^2 since the last reliable update
  double scale;               // r_lo = scale * r_hi
  double b2;                  // ||z||^2 of the full right-hand side
  double tol2;                // tol^2 * b2
  double r2_true;             // last FP64 ||bhat - M x_hi||^2
  double delta2;              // reliable update when ||r||^2 < delta2 * r2_max
  double r2_full;             // ||z - (D + sigma) x||^2 over the full lattice (verification)
  // Coefficients read by the per-site kernels, in both precisions (kernels never
  // do per-thread FP64 scalar arithmetic: FP64 issues at a small fraction of FP32).
  double cd[15];
  float cf[15];
  int status;
  int flags;
  int iters;
  int updates;
  int restarts;
  int max_iter;
  int cg_iters;               // CGNR fallback iterations
  int cg_max_iter;
  // Wilson-clover: the packed (A + C(x))^-1 of this system's shift, [2][Vh][2][36] in FP64 and
  // FP32 (nullptr: the clover passes take the shift-independent eigen-decomposed table)
  const double* clv_inv64;
  const float* clv_inv32;
};

template <typename Tm>
__device__ __forceinline__ Tm coef(const SysState& s, int k) {
  if constexpr (std::is_same<Tm, double>::value) return s.cd[k];
  else return s.cf[k];
}

}  // namespace fs
