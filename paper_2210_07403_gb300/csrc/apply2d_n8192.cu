// Kernels of the two-dimensional operator for the 8192² grid in FP32 (every operator); the FP64
// kernels of this size are in apply2d_n8192_fp64.cu, so the two compile in parallel.
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D_T(float, 13)
}  // namespace ibdl
