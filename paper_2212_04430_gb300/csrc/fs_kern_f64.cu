// Kernel instantiations for double storage.
#include "fs_launch.cuh"

namespace fs {
FS_INSTANTIATE(double)
template cudaError_t launch_gauge_pack<double>(void*, const double*, const Geom&, int, cudaStream_t);
}  // namespace fs
