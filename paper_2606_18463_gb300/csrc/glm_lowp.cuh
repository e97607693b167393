// glm_lowp.cuh -- host-side interface of the end-to-end low-precision
// mini-batch SGD baseline (k_sgd_lowp.cu), kept apart from the shared header
// of the CA-SGD path.
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

}  // namespace glm
