// Kernels of the three-dimensional operator for the 32³ grid (every operator, FP64, FP32 and
// float-float).
#include "apply3d_kernels.cuh"

namespace ibdl {
IBDL_INSTANTIATE_3D(5)
}  // namespace ibdl
