// Kernels of the two-dimensional operator for the 1024² grid (every operator, both precisions).
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D(10)
}  // namespace ibdl
