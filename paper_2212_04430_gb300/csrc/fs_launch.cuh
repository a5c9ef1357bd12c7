// Kernel launchers, instantiated once per storage precision (fs_kern_*.cu).
#pragma once

#include <algorithm>

#include "fs_engine.h"

namespace fs {

template <typename Ts>
using MathOf = typename std::conditional<std::is_same<Ts, double>::value, double, float>::type;

// Directions kept in flight by the prefetching hop kernel (shared-memory ring slots).
template <typename Ts> constexpr int hop_pf() { return sizeof(Ts) == 2 ? 4 : 3; }

// Ring depth of the persistent paired kernel: four operands in flight for 16-bit storage
// (measured on the 16^3x32 hop: 2 or 3 slots leave the 10-operand launches waiting on L2), which
// keeps three 128-thread blocks resident per SM; FP32 storage has twice the bytes per operand.
// The autotuner may pick the other depth of hop_pk_depths for a tile.
template <typename Ts>
constexpr int hop_pk_depth() {
  return sizeof(Ts) <= 2 ? 4 : 2;
}
template <typename Ts>
constexpr int hop_pk_alt_depth() {
  return 3;
}

struct PersistentGrid {
  cudaError_t err = cudaSuccess;
  int blocks_per_sm = 0, nsm = 0;
};

// The persistent paired hop for 32-system chunks (hop_kernel_pk) at ring depth PF: 128-thread
// blocks of 8 sites, as many as are resident (capped at l.pk_blocks per SM when set), never more
// blocks than site chunks.
template <typename Ts, typename Tg, int R, int C, int D, int PF, bool CLV = false>
cudaError_t launch_hop_pk_at(const HopArgs& a, const Launch& l) {
  auto kern = hop_kernel_pk<Ts, Tg, R, C, D, PF, CLV>;
  const size_t smem = hop_pk_smem<Ts, PF, DotK<D>::K>();
  // thread-safe one-time set-up: shared-memory opt-in and the resident grid
  static const PersistentGrid pg = [&] {
    PersistentGrid p;
    int dev = 0;
    if ((p.err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return p;
    if ((p.err = cudaGetDevice(&dev))) return p;
    if ((p.err = cudaDeviceGetAttribute(&p.nsm, cudaDevAttrMultiProcessorCount, dev))) return p;
    p.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p.blocks_per_sm, kern, 128, smem);
    if (!p.err && p.blocks_per_sm < 1) p.err = cudaErrorInvalidConfiguration;
    return p;
  }();
  if (pg.err) return pg.err;
  const int per_sm = l.pk_blocks > 0 ? std::min(l.pk_blocks, pg.blocks_per_sm) : pg.blocks_per_sm;
  const int gy = l.grid_y;
  const int gx = std::max(1, std::min(a.sh.nchunk, per_sm * pg.nsm / std::max(gy, 1)));
  kern<<<dim3(gx, gy), 128, smem, l.stream>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <typename Ts, typename Tg, typename Tm, int R, int C, int D, bool CLV = false>
cudaError_t launch_hop_pk(const HopArgs& a, const Launch& l) {
  if (l.pk_depth == hop_pk_alt_depth<Ts>())
    return launch_hop_pk_at<Ts, Tg, R, C, D, hop_pk_alt_depth<Ts>(), CLV>(a, l);
  return launch_hop_pk_at<Ts, Tg, R, C, D, hop_pk_depth<Ts>(), CLV>(a, l);
}

// the shapes the persistent paired kernel serves: 32-system chunks of 8 sites
inline bool pk_shape(const HopArgs& a, const Launch& l) { return a.sh.NB == 32 && a.sh.SB == 8 && l.block == 256; }

template <typename Ts, typename Tg, typename Tm, int R, int C, int D>
cudaError_t launch_hop_pf(const HopArgs& a, const Launch& l) {
  if (a.sysmajor) return cudaErrorInvalidValue;  // inner-precision fields are tile-layout only
  // 32-system chunks, 8 sites per block: the persistent paired kernel
  if (pk_shape(a, l)) return launch_hop_pk<Ts, Tg, Tm, R, C, D>(a, l);
  constexpr int PF = hop_pf<Ts>();
  const size_t smem = hop_pf_smem<Ts, PF>(l.block);
  // thread-safe one-time set-up (several server workers may launch concurrently)
  static const cudaError_t configured = cudaFuncSetAttribute(
      hop_kernel_pf<Ts, Tg, Tm, R, C, D, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)hop_pf_smem<Ts, PF>(256));
  if (configured) return configured;
  hop_kernel_pf<Ts, Tg, Tm, R, C, D, PF><<<dim3(l.grid_x, l.grid_y), l.block, smem, l.stream>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <typename Ts>
cudaError_t launch_hop(int coef, int dot, int nr, const HopArgs& a, const Launch& l) {
  using Tg = typename GaugeOf<Ts>::T;
  using Tm = MathOf<Ts>;
  const dim3 grid(l.grid_x, l.grid_y), block(l.block);
  // Wilson-clover M-hat and D_sw on the tile layout, with the Y operand (C X): the persistent
  // paired kernel for the M-hat of 32-system chunks in the inner precisions, else the generic one
#define FS_HOP_CLV(C, D, R)                                                                  \
  if (coef == C && dot == D && nr == R) {                                                    \
    if constexpr (!std::is_same<Ts, double>::value && C == COEF_MHAT)                        \
      if (pk_shape(a, l)) return launch_hop_pk<Ts, Tg, Tm, R, C, D, true>(a, l);             \
    hop_kernel<Ts, Tg, Tm, R, C, D, false, true><<<grid, block, 0, l.stream>>>(a);           \
    note_launch();                                                                           \
    return cudaGetLastError();                                                               \
  }
  if (a.clover && (coef == COEF_MHAT || coef == COEF_DSLASH)) {
    if (a.sysmajor) {
      // the FP64 work-list M-hat of the CGNR fallback
      if constexpr (std::is_same<Ts, double>::value) {
        if (coef == COEF_MHAT && nr == 18 && (dot == DOT_NONE || dot == DOT_NORM)) {
          if (dot == DOT_NONE) hop_kernel<Ts, Tg, Tm, 18, COEF_MHAT, DOT_NONE, true, true><<<grid, block, 0, l.stream>>>(a);
          else hop_kernel<Ts, Tg, Tm, 18, COEF_MHAT, DOT_NORM, true, true><<<grid, block, 0, l.stream>>>(a);
          note_launch();
          return cudaGetLastError();
        }
      }
      return cudaErrorInvalidValue;
    }
    FS_HOP_CLV(COEF_MHAT, DOT_R, 18)
    FS_HOP_CLV(COEF_MHAT, DOT_TS, 18)
    FS_HOP_CLV(COEF_DSLASH, DOT_NONE, 18)
    if constexpr (!std::is_same<Ts, double>::value) {
      FS_HOP_CLV(COEF_MHAT, DOT_R, 12)
      FS_HOP_CLV(COEF_MHAT, DOT_TS, 12)
      FS_HOP_CLV(COEF_DSLASH, DOT_NONE, 12)
    }
    return cudaErrorInvalidValue;
  }
#undef FS_HOP_CLV
#define FS_HOP(C, D, R)                                                           \
  if (coef == C && dot == D && nr == R) {                                         \
    if (a.sysmajor) hop_kernel<Ts, Tg, Tm, R, C, D, true><<<grid, block, 0, l.stream>>>(a); \
    else hop_kernel<Ts, Tg, Tm, R, C, D, false><<<grid, block, 0, l.stream>>>(a);           \
    note_launch();                                                                \
    return cudaGetLastError();                                                    \
  }
#define FS_HOP_PF(C, D, R) \
  if (coef == C && dot == D && nr == R) return launch_hop_pf<Ts, Tg, Tm, R, C, D>(a, l);
  if constexpr (std::is_same<Ts, double>::value) {
    FS_HOP(COEF_PLAIN, DOT_NONE, 18)
    FS_HOP(COEF_DSLASH, DOT_NONE, 18)
    FS_HOP(COEF_MHAT, DOT_R, 18)
    FS_HOP(COEF_MHAT, DOT_TS, 18)
    FS_HOP(COEF_MHAT, DOT_NORM, 18)   // CGNR fallback: q = M p, ||q||^2
    FS_HOP(COEF_MHAT, DOT_NONE, 18)   // CGNR fallback: M gamma5 s
    FS_HOP(COEF_PREP, DOT_NORM, 18)
    FS_HOP(COEF_RECON, DOT_NONE, 18)
    FS_HOP(COEF_TRUERES, DOT_NORM, 18)
    FS_HOP(COEF_FULLRES, DOT_NORM, 18)
    FS_HOP(COEF_KAPPA, DOT_NONE, 18)  // hopping parameter expansion
  } else {
    FS_HOP_PF(COEF_PLAIN, DOT_NONE, 18)
    FS_HOP_PF(COEF_DSLASH, DOT_NONE, 18)
    FS_HOP_PF(COEF_MHAT, DOT_R, 18)
    FS_HOP_PF(COEF_MHAT, DOT_TS, 18)
    FS_HOP_PF(COEF_PLAIN, DOT_NONE, 12)
    FS_HOP_PF(COEF_DSLASH, DOT_NONE, 12)
    FS_HOP_PF(COEF_MHAT, DOT_R, 12)
    FS_HOP_PF(COEF_MHAT, DOT_TS, 12)
  }
#undef FS_HOP
#undef FS_HOP_PF
  return cudaErrorInvalidValue;
}

template <typename Ts>
cudaError_t launch_blas(int op, const BlasArgs& a, const Launch& l) {
  using Tx = typename XOf<Ts>::T;
  using Tm = MathOf<Ts>;
  const dim3 grid(l.grid_x, l.grid_y), block(l.block);
  // the per-iteration solver updates run on the tile shape; the FP64-field operations
  // (x_hi updates, residual restarts, norms) on the system-major work list
  if ((op == OP_S || op == OP_XRP) == (a.sysmajor != 0)) return cudaErrorInvalidValue;
  switch (op) {
    case OP_S: blas_kernel<Ts, Tx, Tm, OP_S, false><<<grid, block, 0, l.stream>>>(a); break;
    case OP_XRP: blas_kernel<Ts, Tx, Tm, OP_XRP, false><<<grid, block, 0, l.stream>>>(a); break;
    case OP_ACCX: blas_kernel<Ts, Tx, Tm, OP_ACCX, true><<<grid, block, 0, l.stream>>>(a); break;
    case OP_ZEROX: blas_kernel<Ts, Tx, Tm, OP_ZEROX, true><<<grid, block, 0, l.stream>>>(a); break;
    case OP_SETR: blas_kernel<Ts, Tx, Tm, OP_SETR, true><<<grid, block, 0, l.stream>>>(a); break;
    case OP_NORM64: blas_kernel<Ts, Tx, Tm, OP_NORM64, true><<<grid, block, 0, l.stream>>>(a); break;
    case OP_RECON: blas_kernel<Ts, Tx, Tm, OP_RECON, true><<<grid, block, 0, l.stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename Ts>
cudaError_t launch_clover(int mode, const ClovArgs& a, const Launch& l) {
  using Tm = MathOf<Ts>;
  using Tc = typename std::conditional<std::is_same<Ts, double>::value, double, float>::type;
  const dim3 grid(l.grid_x, l.grid_y), block(l.block);
  if (a.sysmajor && !std::is_same<Ts, double>::value) return cudaErrorInvalidValue;  // FP64 fields only
  // the paired pass where the block rows hold an even number of systems that divides 512
  const bool paired = !std::is_same<Ts, double>::value && !a.sysmajor && a.sh.NB % 2 == 0 && 256 % (a.sh.NB / 2) == 0;
#define FS_CLV(M)                                                                                         \
  if (mode == M) {                                                                                        \
    if constexpr (!std::is_same<Ts, double>::value)                                                       \
      if (paired) {                                                                                       \
        clover_kernel_pk<Ts, M><<<grid, 256, 0, l.stream>>>(a);                                           \
        note_launch();                                                                                    \
        return cudaGetLastError();                                                                        \
      }                                                                                                   \
    if (a.sysmajor) clover_kernel<Ts, Tc, Tm, M, true><<<grid, block, 0, l.stream>>>(a);                 \
    else clover_kernel<Ts, Tc, Tm, M, false><<<grid, block, 0, l.stream>>>(a);                           \
    note_launch();                                                                                        \
    return cudaGetLastError();                                                                            \
  }
  FS_CLV(CLV_MUL)
  FS_CLV(CLV_SUB)
  FS_CLV(CLV_INV)
  if (mode == CLV_INV_MUL) {  // tile layout only
    if (a.sysmajor) return cudaErrorInvalidValue;
    if constexpr (!std::is_same<Ts, double>::value)
      if (paired) {
        clover_kernel_pk<Ts, CLV_INV_MUL><<<grid, 256, 0, l.stream>>>(a);
        note_launch();
        return cudaGetLastError();
      }
    clover_kernel<Ts, Tc, Tm, CLV_INV_MUL, false><<<grid, block, 0, l.stream>>>(a);
    note_launch();
    return cudaGetLastError();
  }
#undef FS_CLV
  return cudaErrorInvalidValue;
}

template <typename Ts>
cudaError_t launch_pack(void* fe, void* fo, const double* canon, const int* vec, const Geom& g, const Shape& sh,
                        const Launch& l, bool sysmajor) {
  pack_kernel<Ts><<<dim3(l.grid_x, l.grid_y), l.block, 0, l.stream>>>(fe, fo, canon, vec, g, sh, sysmajor);
  note_launch();
  return cudaGetLastError();
}

template <typename Ts>
cudaError_t launch_unpack(double* canon, const void* fe, const void* fo, const int* vec, const Geom& g,
                          const Shape& sh, const Launch& l, bool sysmajor) {
  unpack_kernel<Ts><<<dim3(l.grid_x, l.grid_y), l.block, 0, l.stream>>>(canon, fe, fo, vec, g, sh, sysmajor);
  note_launch();
  return cudaGetLastError();
}

template <typename Tg>
cudaError_t launch_gauge_pack(void* out, const double* canon, const Geom& g, int nr, cudaStream_t s) {
  const int n = 8 * g.Vh;
  const int blocks = (n + 255) / 256;
  if (nr == 18) gauge_pack_kernel<Tg, 18><<<blocks, 256, 0, s>>>(out, canon, g);
  else if (nr == 12) gauge_pack_kernel<Tg, 12><<<blocks, 256, 0, s>>>(out, canon, g);
  else return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

#define FS_INSTANTIATE(TS)                                                                                   \
  template cudaError_t launch_hop<TS>(int, int, int, const HopArgs&, const Launch&);                        \
  template cudaError_t launch_blas<TS>(int, const BlasArgs&, const Launch&);                                \
  template cudaError_t launch_clover<TS>(int, const ClovArgs&, const Launch&);                              \
  template cudaError_t launch_pack<TS>(void*, void*, const double*, const int*, const Geom&, const Shape&,   \
                                       const Launch&, bool);                                                \
  template cudaError_t launch_unpack<TS>(double*, const void*, const void*, const int*, const Geom&,         \
                                         const Shape&, const Launch&, bool);

}  // namespace fs
