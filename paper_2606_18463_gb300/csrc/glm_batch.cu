// glm_batch.cu -- batched fits (placeholder until the persistent batch
// kernel lands).
#include "glm_internal.cuh"

using namespace glm;

extern "C" {

void glm_batch_opts_default(glm_batch_opts *o) {
  if (!o) return;
  o->dtype = GLM_BF16;
  o->input_dtype = GLM_F32;
  o->input_on_host = 1;
  o->stream = nullptr;
}

int glm_batch_create(int P, const glm_problem_desc *descs, const glm_batch_opts *opts,
                     glm_batch *out) {
  (void)P; (void)descs; (void)opts;
  if (out) *out = nullptr;
  return set_error(GLM_EUNSUPPORTED, "batched fits not built");
}

int glm_batch_run(glm_batch bt, float *const *xs, int *status) {
  (void)bt; (void)xs; (void)status;
  return set_error(GLM_EUNSUPPORTED, "batched fits not built");
}

int glm_batch_loss(glm_batch bt, float *const *xs, double *out) {
  (void)bt; (void)xs; (void)out;
  return set_error(GLM_EUNSUPPORTED, "batched fits not built");
}

int glm_batch_choice(glm_batch bt, int p, int *s, int64_t *b, int *gram_dtype) {
  (void)bt; (void)p; (void)s; (void)b; (void)gram_dtype;
  return set_error(GLM_EUNSUPPORTED, "batched fits not built");
}

int glm_batch_destroy(glm_batch bt) {
  (void)bt;
  return GLM_OK;
}

}  // extern "C"
