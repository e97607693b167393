// glm_slab.cu -- column-partitioned CA-SGD (paper Algorithm 1 on P ranks:
// the 1D block-column partition, one grouped AllReduce of the partial
// margins and the strictly block-lower Gram per outer iteration, then the
// recurrence run redundantly on every rank; Sec. 6's grouped reduction of
// {r, G_L} in one buffer).
//
// A rank holds a column slab A_p (its own dataset handle over those columns;
// every rank draws the same rows from the shared counter-based stream).  One
// outer iteration of sh inner steps is two calls around the caller's sum:
//   glm_slab_partial: gather Y_p = A_p[I], write red = [r_p | G_p] with
//                     r_p = Y_p x_p and G_p the strictly block-lower part of
//                     Y_p Y_p^T in the packed row-block layout;
//   (caller)          red <- sum over ranks of red (an AllReduce; on one GPU
//                     glm_sum_buffers over emulated ranks);
//   glm_slab_finish:  run z_j = c^j r_j - alpha sum_{i<j} c^{j-1-i} G_{j,i} u_i,
//                     u_j = dL/dr(z_j, y_{I_j}) on the summed buffer, then
//                     x_p <- c^sh x_p - alpha sum_j c^{sh-1-j} Y_{j,p}^T u_j.
// The recurrence is the same on every rank (same inputs, same order of
// operations), so the ranks' slabs stay one iterate.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "glm_internal.cuh"
#include "glm_baselines.cuh"

namespace glm {
int resolve_public(Handle *h, int s, int64_t b, float eta, float lambda, int64_t iters,
                   uint64_t seed, float *x, const glm_ca_opts *o, int &gram_dt, int &gemv_dt,
                   int &rec64, int &kahan, int &gram_impl, int64_t &ld_gram, int64_t &ld_gemv,
                   uint32_t &problem);

namespace {

constexpr int kWarps = 8;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// r[row] = Y[row, 0:n] . x (FP32 accumulation, lane-strided then a fixed
// shuffle tree), one warp per row.
template <typename TY>
__global__ void __launch_bounds__(kWarps * 32)
k_slab_margin(const TY *Y, int64_t ldy, int64_t rows, int64_t n, const float *x, float *r) {
  const int lane = threadIdx.x & 31;
  for (int64_t row = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); row < rows;
       row += (int64_t)gridDim.x * kWarps) {
    const TY *y = Y + row * ldy;
    float acc = 0.f;
    for (int64_t c = (int64_t)lane * 8; c < n; c += 256) {
      float v[8];
      Vec8<TY>::load(y + c, v);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (c + i < n) acc = fmaf(v[i], __ldg(x + c + i), acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) r[row] = acc;
  }
}

struct RecArgs {
  const float *r, *G, *lab;   // summed margins, summed packed G, labels
  float *w;                   // out: c^-j u_j per row (the update's weights)
  unsigned *flag;
  int64_t b;
  int sh, loss;
  double alpha;
  double cpow[257], cinv[257];
};

// The recurrence of one outer iteration on one CTA (every rank runs it):
// block j's rows are dealt to warps; each row's correction dot over the
// residual history c^-i u_i (i < j) runs lane-strided with a fixed shuffle
// tree, in the recurrence type TR.  The residual is the IEEE FP32 loss
// derivative of the margin (rounded once from FP64 when TR is double).
template <typename TR>
__global__ void __launch_bounds__(1024)
k_slab_recur(const __grid_constant__ RecArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  TR *uh = reinterpret_cast<TR *>(smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t b = a.b;
  for (int j = 0; j < a.sh; ++j) {
    const int64_t jb = (int64_t)j * b, ldj = gram_ld(j, b);
    const float *Gj = a.G + gram_off(j, b);
    for (int64_t l = warp; l < b; l += nw) {
      const int64_t row = jb + l;
      TR corr = 0;
      if (j > 0) {
        const float *g = Gj + l * ldj;
        for (int64_t c = lane; c < jb; c += 32) corr = fma((TR)__ldg(g + c), uh[c], corr);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) corr += __shfl_xor_sync(0xffffffffu, corr, off);
      }
      if (lane == 0) {
        const TR z = (TR)a.cpow[j] * (TR)a.r[row] -
                     (j > 0 ? (TR)(a.alpha * a.cpow[j - 1]) * corr : (TR)0);
        const float u = dloss<float>(a.loss, (float)z, a.lab[row]);
        if (!isfinite((float)z) || !isfinite(u)) atomicOr(a.flag, FLAG_NONFINITE);
        uh[row] = (TR)u * (TR)a.cinv[j];
        a.w[row] = (float)uh[row];
      }
    }
    __syncthreads();
  }
}

// x[col] <- decay x[col] - stp sum_rows Y[row, col] w[row]: 32 columns x 8 row
// groups per block, Kahan-compensated FP32 per thread, the 8 partials summed
// in order (Kahan) by the first group.
template <typename TY>
__global__ void __launch_bounds__(256)
k_slab_update(const TY *Y, int64_t ldy, int64_t rows, int64_t n, const float *w, float decay,
              float stp, int kahan, float *x, unsigned *flag) {
  __shared__ float part[8][32];
  const int cl = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + cl;
  float acc = 0.f, cmp = 0.f;
  if (col < n) {
    for (int64_t row = g; row < rows; row += 8) {
      const float v = to_f(Y[row * ldy + col]) * __ldg(w + row);
      if (kahan) {
        const float yv = v - cmp;
        const float t = acc + yv;
        cmp = (t - acc) - yv;
        acc = t;
      } else {
        acc += v;
      }
    }
  }
  part[g][cl] = acc - cmp;
  __syncthreads();
  if (g == 0 && col < n) {
    float S = 0.f, cS = 0.f;
    for (int k = 0; k < 8; ++k) {
      const float yv = part[k][cl] - cS;
      const float t = S + yv;
      cS = (t - S) - yv;
      S = t;
    }
    const float xn = fmaf(-stp, S - cS, decay * x[col]);
    if (!isfinite(xn)) atomicOr(flag, FLAG_NONFINITE);
    x[col] = xn;
  }
}

struct SumArgs {
  const float *src[64];
  float *dst;
  int64_t count;
  int P;
};

// dst[i] = src[0][i] + src[1][i] + ... in rank order (FP32 additions).
__global__ void k_sum(const __grid_constant__ SumArgs a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    float v = a.src[0][i];
    for (int p = 1; p < a.P; ++p) v += a.src[p][i];
    a.dst[i] = v;
  }
}

int num_sms() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

struct SlabStep {
  int gram_dt, gemv_dt, rec64, kahan, gram_impl;
  int64_t ld_gram, ld_gemv, sb, sbp;
  uint32_t problem;
};

int check_step(Handle *h, int s, int64_t b, int sh, float eta, float lambda, float *x,
               const glm_ca_opts *o, SlabStep &st) {
  if (!h) return set_error(GLM_EINVAL, "null handle");
  if (sh < 1 || sh > s) return set_error(GLM_EINVAL, "sh must be in [1, s]");
  if ((int64_t)s * b > 8192)
    return set_error(GLM_EINVAL, "slab steps hold s * b <= 8192 rows (the recurrence's history)");
  GLM_TRY(resolve_public(h, s, b, eta, lambda, sh, 0, x, o, st.gram_dt, st.gemv_dt, st.rec64,
                         st.kahan, st.gram_impl, st.ld_gram, st.ld_gemv, st.problem));
  st.sb = (int64_t)s * b;
  st.sbp = round_up(st.sb, 4);
  return GLM_OK;
}

// The step's rows, labels, row scales and update weights live in the
// handle's first chunk buffers; a captured run graph that points at a buffer
// this reallocates is dropped.
int ensure_slab_scratch(Handle *h, const SlabStep &st) {
  void *before[5] = {h->ygram[0].ptr, h->ygemv[0].ptr, h->ylab[0].ptr, h->yscale[0].ptr,
                     h->gbuf[0].ptr};
  int rc = h->ygram[0].ensure((size_t)st.sb * st.ld_gram * elem_bytes(st.gram_dt));
  if (rc == GLM_OK && st.ld_gemv)
    rc = h->ygemv[0].ensure((size_t)st.sb * st.ld_gemv * elem_bytes(st.gemv_dt));
  if (rc == GLM_OK) rc = h->ylab[0].ensure((size_t)st.sbp * 4);
  if (rc == GLM_OK) rc = h->yscale[0].ensure((size_t)st.sb * 4);
  if (rc == GLM_OK) rc = h->gbuf[0].ensure((size_t)st.sb * 4);   // the update weights
  void *after[5] = {h->ygram[0].ptr, h->ygemv[0].ptr, h->ylab[0].ptr, h->yscale[0].ptr,
                    h->gbuf[0].ptr};
  if (memcmp(before, after, sizeof(before)) != 0 && h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return rc;
}

template <typename TY>
int margin_t(const void *Y, int64_t ld, int64_t rows, int64_t n, const float *x, float *r,
             cudaStream_t st) {
  const int64_t want = (rows + kWarps - 1) / kWarps;
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms() * 16);
  k_slab_margin<TY><<<grid, kWarps * 32, 0, st>>>(static_cast<const TY *>(Y), ld, rows, n, x, r);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

template <typename TY>
int update_t(const void *Y, int64_t ld, int64_t rows, int64_t n, const float *w, float decay,
             float stp, int kahan, float *x, unsigned *flag, cudaStream_t st) {
  k_slab_update<TY><<<(unsigned)((n + 31) / 32), 256, 0, st>>>(
      static_cast<const TY *>(Y), ld, rows, n, w, decay, stp, kahan, x, flag);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

template <typename F>
int by_type(int dt, F &&f) {
  switch (dt) {
  case GLM_F32: case GLM_TF32: return f(float());
  case GLM_BF16: return f(__nv_bfloat16());
  case GLM_F16: return f(__half());
  }
  return set_error(GLM_EINVAL, "slab: unsupported GEMV operand type");
}

}  // namespace
}  // namespace glm

using namespace glm;

extern "C" {

int glm_slab_reduce_floats(int s, int64_t b, int64_t *count) {
  set_error(GLM_OK, "");
  if (!count) return set_error(GLM_EINVAL, "count is NULL");
  if (s < 1 || b < 1 || (int64_t)s * b > 8192) return set_error(GLM_EINVAL, "need s, b >= 1, s b <= 8192");
  *count = round_up((int64_t)s * b, 4) + gram_size(s, b);
  return GLM_OK;
}

int glm_slab_partial(glm_handle hh, int s, int64_t b, int sh, uint64_t seed, int64_t first_iter,
                     const float *x, float *red, const glm_ca_opts *opts) {
  set_error(GLM_OK, "");
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!x || !red) return set_error(GLM_EINVAL, "x or red is NULL");
  if (first_iter < 0) return set_error(GLM_EINVAL, "first_iter must be >= 0");
  SlabStep st;
  GLM_TRY(check_step(h, s, b, sh, 1.0f, 0.0f, const_cast<float *>(x), opts, st));
  GLM_TRY(ensure_slab_scratch(h, st));
  cudaStream_t cs = h->stream;
  const int64_t rows = (int64_t)sh * b;
  GatherArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.A = h->A; ga.lda = h->lda; ga.a_dt = h->dtype; ga.colscale = h->colscale;
  ga.A8 = h->A8; ga.rs8 = h->rowscale8; ga.lda8 = h->lda8;
  ga.y = h->y; ga.m = h->m; ga.n = h->n; ga.rows = rows;
  ga.flag = h->dflag;
  ga.q0 = (uint64_t)(first_iter * b); ga.seed = seed; ga.problem = st.problem;
  ga.out1 = h->ygram[0].ptr; ga.dt1 = st.gram_dt; ga.ld1 = st.ld_gram;
  if (st.ld_gemv) {
    ga.out2 = h->ygemv[0].ptr; ga.dt2 = st.gemv_dt; ga.ld2 = st.ld_gemv;
  }
  ga.ylab = static_cast<float *>(h->ylab[0].ptr);
  ga.rscale = static_cast<float *>(h->yscale[0].ptr);
  ga.lab_sb = st.sb;
  ga.lab_sbp = st.sbp;
  GLM_TRY(launch_gather(ga, cs));
  // partial margins into red[0 .. sb), zeros past the step's rows
  GLM_CUDA_TRY(cudaMemsetAsync(red, 0, (size_t)st.sbp * 4, cs));
  const void *Yv = st.ld_gemv ? h->ygemv[0].ptr : h->ygram[0].ptr;
  const int64_t ldv = st.ld_gemv ? st.ld_gemv : st.ld_gram;
  GLM_TRY(by_type(st.gemv_dt, [&](auto t) {
    return margin_t<decltype(t)>(Yv, ldv, rows, h->n, x, red, cs);
  }));
  // partial strictly block-lower Gram into red[sbp ..)
  float *G = red + st.sbp;
  GLM_CUDA_TRY(cudaMemsetAsync(G, 0, (size_t)gram_size(s, b) * 4, cs));
  if (sh >= 2) {
    GramArgs gr;
    memset(&gr, 0, sizeof(gr));
    gr.Y = h->ygram[0].ptr; gr.dt = st.gram_dt; gr.ld = st.ld_gram;
    gr.rs = st.gram_dt == GLM_E4M3 ? static_cast<const float *>(h->yscale[0].ptr) : nullptr;
    gr.nouter = 1; gr.rows = rows; gr.s = s; gr.b = b; gr.n = h->n; gr.G = G;
    gr.flag = h->dflag;
    if (st.gram_impl == 2) GLM_TRY(launch_gram_tc(gr, cs));
    else if (st.gram_impl == 3) GLM_TRY(launch_gram_simt_f16acc(gr, cs));
    else if (st.gram_impl == 4) GLM_TRY(launch_gram_tc_f16acc(gr, cs));
    else GLM_TRY(launch_gram_simt(gr, cs));
  }
  return GLM_OK;
}

int glm_slab_finish(glm_handle hh, int s, int64_t b, int sh, float eta, float lambda,
                    const float *red, float *x, const glm_ca_opts *opts) {
  set_error(GLM_OK, "");
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!x || !red) return set_error(GLM_EINVAL, "x or red is NULL");
  SlabStep st;
  GLM_TRY(check_step(h, s, b, sh, eta, lambda, x, opts, st));
  if (!h->gbuf[0].ptr || h->gbuf[0].bytes < (size_t)st.sb * 4)
    return set_error(GLM_EINVAL, "glm_slab_finish needs a preceding glm_slab_partial of this shape");
  cudaStream_t cs = h->stream;
  const double c = 1.0 - (double)eta * (double)lambda;
  RecArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.r = red;
  ra.G = red + st.sbp;
  ra.lab = static_cast<const float *>(h->ylab[0].ptr);
  ra.w = static_cast<float *>(h->gbuf[0].ptr);
  ra.flag = h->dflag;
  ra.b = b;
  ra.sh = sh;
  ra.loss = h->loss;
  ra.alpha = (double)eta / (double)b;
  double cp = 1.0;
  for (int j = 0; j <= s; ++j) {
    ra.cpow[j] = cp;
    ra.cinv[j] = 1.0 / cp;
    cp *= c;
  }
  const size_t smem = (size_t)st.sb * (st.rec64 ? 8 : 4);
  if (st.rec64) {
    GLM_CUDA_TRY(cudaFuncSetAttribute(k_slab_recur<double>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_slab_recur<double><<<1, 1024, smem, cs>>>(ra);
  } else {
    GLM_CUDA_TRY(cudaFuncSetAttribute(k_slab_recur<float>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_slab_recur<float><<<1, 1024, smem, cs>>>(ra);
  }
  GLM_CUDA_TRY(cudaGetLastError());
  const void *Yv = st.ld_gemv ? h->ygemv[0].ptr : h->ygram[0].ptr;
  const int64_t ldv = st.ld_gemv ? st.ld_gemv : st.ld_gram;
  const float decay = (float)ra.cpow[sh];
  const float stp = (float)(ra.alpha * ra.cpow[sh - 1]);
  return by_type(st.gemv_dt, [&](auto t) {
    return update_t<decltype(t)>(Yv, ldv, (int64_t)sh * b, h->n, ra.w, decay, stp, st.kahan, x,
                                 h->dflag, cs);
  });
}

int glm_sum_buffers(float *dst, const float *const *srcs, int P, int64_t count, void *stream) {
  set_error(GLM_OK, "");
  if (!dst || !srcs) return set_error(GLM_EINVAL, "null argument");
  if (P < 1 || P > 64) return set_error(GLM_EINVAL, "P must be in [1, 64]");
  if (count < 0) return set_error(GLM_EINVAL, "count must be >= 0");
  if (count == 0) return GLM_OK;
  SumArgs a;
  memset(&a, 0, sizeof(a));
  for (int p = 0; p < P; ++p) {
    if (!srcs[p]) return set_error(GLM_EINVAL, "a source buffer is NULL");
    a.src[p] = srcs[p];
  }
  a.dst = dst;
  a.count = count;
  a.P = P;
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)num_sms() * 8);
  k_sum<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // extern "C"
