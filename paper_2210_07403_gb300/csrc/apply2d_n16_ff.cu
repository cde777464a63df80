// Float-float kernels of the two-dimensional operator for the 16² grid: the forward operators
// (single problems and batched stages) and the transposes.
#include "apply2d_launch.cuh"

namespace ibdl {
IBDL_INSTANTIATE_2D_FWD(ff, 4)
IBDL_INSTANTIATE_2D_TRANS(ff, 4)
}  // namespace ibdl
