// Kernel instantiations for float storage.
#include "fs_launch.cuh"

namespace fs {
FS_INSTANTIATE(float)
template cudaError_t launch_gauge_pack<float>(void*, const double*, const Geom&, int, cudaStream_t);
}  // namespace fs
