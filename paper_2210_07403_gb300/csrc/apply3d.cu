// Three-dimensional IBDL operator (not yet built in this revision: calls report UNSUPPORTED).
#include "ibdl_internal.cuh"

namespace ibdl {

ibdl_status plan_3d(Geometry* g) {
  (void)g;
  return IBDL_OK;
}
ibdl_status apply_3d(Geometry*, int, const double*, double*, cudaStream_t, const int*) {
  return fail(IBDL_ERR_UNSUPPORTED, "3-D operator not available in this build");
}
ibdl_status field_3d(Geometry*, const double*, double*, cudaStream_t) {
  return fail(IBDL_ERR_UNSUPPORTED, "3-D operator not available in this build");
}
ibdl_status apply_3d_indexed(Geometry*, int, double*, const int*, int, cudaStream_t, const int*) {
  return fail(IBDL_ERR_UNSUPPORTED, "3-D operator not available in this build");
}
ibdl_status adjoint_3d(Geometry*, int, const double*, double*, cudaStream_t) {
  return fail(IBDL_ERR_UNSUPPORTED, "3-D operator not available in this build");
}

}  // namespace ibdl
