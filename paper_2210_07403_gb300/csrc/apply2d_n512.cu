// Kernels of the two-dimensional operator for the 512² grid (every operator, both precisions).
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D(9)
}  // namespace ibdl
