// Kernel instantiations for float storage.
#include "fs_launch.cuh"

namespace fs {
FS_INSTANTIATE(float)
template cudaError_t launch_gauge_pack<float>(void*, const double*, const Geom&, int, cudaStream_t);

cudaError_t launch_hop64_f32(int coef, int dot, const HopArgs& a, const Launch& l) {
  const dim3 grid(l.grid_x, l.grid_y), block(l.block);
  if (!a.sysmajor) return cudaErrorInvalidValue;  // the FP64 fields are system-major
  if (coef == COEF_PLAIN && dot == DOT_NONE)
    hop_kernel<double, float, float, 18, COEF_PLAIN, DOT_NONE, true><<<grid, block, 0, l.stream>>>(a);
  else if (coef == COEF_TRUERES && dot == DOT_NORM)
    hop_kernel<double, float, float, 18, COEF_TRUERES, DOT_NORM, true><<<grid, block, 0, l.stream>>>(a);
  else
    return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_clover64_f32(int mode, const ClovArgs& a, const Launch& l) {
  const dim3 grid(l.grid_x, l.grid_y), block(l.block);
  if (!a.sysmajor) return cudaErrorInvalidValue;
  if (mode == CLV_SUB) clover_kernel<double, float, float, CLV_SUB, true><<<grid, block, 0, l.stream>>>(a);
  else if (mode == CLV_INV) clover_kernel<double, float, float, CLV_INV, true><<<grid, block, 0, l.stream>>>(a);
  else return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}
}  // namespace fs
