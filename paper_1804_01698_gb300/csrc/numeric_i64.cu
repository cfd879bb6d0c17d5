// Numeric-phase kernels instantiated for int64_t values.
#include "numeric.cuh"

namespace sg {
cudaError_t launch_numeric_i64(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v) {
  return launch_numeric_t<int64_t>(p, c_rp, c_ci, static_cast<int64_t *>(c_v));
}
}  // namespace sg
