// Kernels of the two-dimensional operator for the 4096² grid (every operator, both precisions).
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D(12)
}  // namespace ibdl
