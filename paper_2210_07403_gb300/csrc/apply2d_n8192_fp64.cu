// Kernels of the two-dimensional operator for the 8192² grid in FP64 (every operator).
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D_T(double, 13)
}  // namespace ibdl
