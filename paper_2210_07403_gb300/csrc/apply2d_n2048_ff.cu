// Float-float kernels of the two-dimensional operator for the 2048² grid: the forward operators
// (single problems and batched stages) and the transposes.
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D_FWD(ff, 11)
IBDL_INSTANTIATE_2D_TRANS(ff, 11)
}  // namespace ibdl
