// Numeric-phase kernels instantiated for float values.
#include "numeric.cuh"

namespace sg {
cudaError_t launch_numeric_f32(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v) {
  return launch_numeric_t<float>(p, c_rp, c_ci, static_cast<float *>(c_v));
}
}  // namespace sg
