// Batched launches of the two-dimensional stokes operator in float (both dipole forms).
#include "apply2d_launch.cuh"

namespace ibdl {
template ibdl_status batch_launch_2d<float, OP_STOKES_AN>(Batch*, int, const double*, double*, cudaStream_t);
template ibdl_status batch_launch_2d<float, OP_STOKES_SD>(Batch*, int, const double*, double*, cudaStream_t);
}  // namespace ibdl
