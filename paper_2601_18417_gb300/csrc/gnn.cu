// gnn.cu -- learned graph-network preconditioner (placeholder until built).
#include "hofv_internal.cuh"

namespace hofv {
int gnn_apply(hofv_ctx* c, const double*, const double*, double*) {
  return fail(c, HOFV_ENOTSUP, "learned preconditioner not available in this build");
}
}  // namespace hofv
