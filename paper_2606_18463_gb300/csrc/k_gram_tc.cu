// k_gram_tc.cu -- tcgen05 tensor-core Gram (filled in below).
#include "glm_internal.cuh"

namespace glm {

bool gram_tc_supported(int dt, int64_t ld) {
  (void)dt;
  (void)ld;
  return false;
}

int launch_gram_tc(const GramArgs &a, cudaStream_t st) {
  (void)a;
  (void)st;
  return set_error(GLM_EUNSUPPORTED, "tcgen05 Gram not built");
}

}  // namespace glm
