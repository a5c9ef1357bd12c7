// Kernel instantiations for __nv_bfloat16 storage.
#include "fs_launch.cuh"

namespace fs {
FS_INSTANTIATE(__nv_bfloat16)
}  // namespace fs
