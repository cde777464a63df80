// Kernels of the two-dimensional operator for the 8192² grid (every operator, both precisions).
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D(13)
}  // namespace ibdl
