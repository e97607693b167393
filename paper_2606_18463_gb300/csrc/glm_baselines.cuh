// glm_baselines.cuh -- host-side interfaces of the numerical baselines of
// the paper's recipe table, kept apart from the shared header of the CA-SGD
// path: the end-to-end low-precision mini-batch SGD (k_sgd_lowp.cu) and the
// FP16-accumulate Gram (k_gram_simt.cu).
#pragma once

#include "glm_internal.cuh"

namespace glm {

// `iters` steps of b rows each, draws q0, q0 + 1, ... of the (seed, problem)
// stream; x is the FP32[n] iterate, read at the start (rounded to the storage
// type) and written at the end.
struct LowpArgs {
  const void *A; int64_t lda; const float *colscale; const float *y;
  int64_t m, n; int b, loss;
  uint64_t seed, problem, q0;
  int64_t iters;
  float alpha, c;
  float *x;
  unsigned *flag;
};
bool lowp_fits(int64_t n, int b);
int launch_sgd_lowp(const LowpArgs &a, int dt, int acc_f16, cudaStream_t st);

// Strictly block-lower Gram of FP16 operands with FP16 accumulation (Recipe
// F's Gram slot); GLM_EINVAL for other operand types or with row scales.
int launch_gram_simt_f16acc(const GramArgs &a, cudaStream_t st);

}  // namespace glm
