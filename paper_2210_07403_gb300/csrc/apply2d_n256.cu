// Kernels of the two-dimensional operator for the 256² grid (every operator, both precisions).
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D(8)
}  // namespace ibdl
