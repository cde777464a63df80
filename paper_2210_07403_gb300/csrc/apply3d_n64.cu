// Kernels of the three-dimensional operator for the 64³ grid (every operator, FP64, FP32 and
// float-float).
#include "apply3d_kernels.cuh"

namespace ibdl {
IBDL_INSTANTIATE_3D(6)
}  // namespace ibdl
