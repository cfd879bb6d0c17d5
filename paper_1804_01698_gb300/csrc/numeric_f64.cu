// Numeric-phase kernels instantiated for double values.
#include "numeric.cuh"

namespace sg {
cudaError_t launch_numeric_f64(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v) {
  return launch_numeric_t<double>(p, c_rp, c_ci, static_cast<double *>(c_v));
}
}  // namespace sg
