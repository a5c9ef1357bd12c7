// Kernel instantiations for __half storage.
#include "fs_launch.cuh"

namespace fs {
FS_INSTANTIATE(__half)
template cudaError_t launch_gauge_pack<__half>(void*, const double*, const Geom&, int, cudaStream_t);
}  // namespace fs
