// Batched launches of the two-dimensional scalar operator in double (both dipole forms).
#include "apply2d_launch.cuh"

namespace ibdl {
template ibdl_status batch_launch_2d<double, OP_SCALAR_AN>(Batch*, int, const double*, double*, cudaStream_t);
template ibdl_status batch_launch_2d<double, OP_SCALAR_SD>(Batch*, int, const double*, double*, cudaStream_t);
}  // namespace ibdl
