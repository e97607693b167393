// glm_recipe.cu -- CA-SGD with the narrow precision recipes of the paper's
// recipe table (Sec. 5.3) that the fused chain does not carry:
//   * FP16 accumulation in the margin and gradient GEMVs (Recipe F's h_a
//     slots; with the FP16-accumulate Gram, gram_impl 3 or 4);
//   * end-to-end narrow state (Recipes H, FP16, and I, BF16): the margins,
//     the Gram output, every correction, residual and history entry, the
//     gradient and the weights are rounded to the state type T once each,
//     as the plain mini-batch baseline (glm_sgd_lowp_run) rounds its own.
// Numerical baselines, not fast paths: per outer iteration a gather, a
// margin kernel, the Gram, a one-CTA recurrence and an update kernel, all
// enqueued on the handle's stream.
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

// round once to the state type: 0 none (FP32), 1 BF16, 2 FP16
template <int ST> __device__ __forceinline__ float rnd(float v) {
  if (ST == 1) return __bfloat162float(__float2bfloat16_rn(v));
  if (ST == 2) return __half2float(__float2half_rn(v));
  return v;
}

__device__ __forceinline__ float ldv(const float *p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldv(const __half *p) { return __half2float(*p); }

// Warp sum of one value per lane in FP16 (pairwise, fixed order) or FP32.
template <int ACC16> __device__ __forceinline__ float warp_sum(float v) {
  if (ACC16) {
    __half h = __float2half_rn(v);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) h = __hadd(h, __shfl_xor_sync(0xffffffffu, h, off));
    return __half2float(h);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// r[row] = T(Y[row] . x), one warp per row; FP16 accumulation: x rounded to
// FP16, each lane's columns by fused half FMAs in order, lanes pairwise.
template <typename TY, int ACC16, int ST>
__global__ void __launch_bounds__(256)
k_rc_margin(const TY *Y, int64_t ldy, int64_t rows, int64_t n, const float *x, float *r) {
  const int lane = threadIdx.x & 31;
  for (int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); row < rows;
       row += (int64_t)gridDim.x * 8) {
    const TY *y = Y + row * ldy;
    float acc = 0.f;
    __half acch = __float2half_rn(0.f);
    for (int64_t c = lane; c < n; c += 32) {
      if (ACC16) acch = __hfma(__float2half_rn(ldv(y + c)), __float2half_rn(x[c]), acch);
      else acc = fmaf(ldv(y + c), x[c], acc);
    }
    const float t = warp_sum<ACC16>(ACC16 ? __half2float(acch) : acc);
    if (lane == 0) r[row] = rnd<ST>(t);
  }
}

struct RcArgs {
  const float *r, *G, *lab;
  float *w;
  unsigned *flag;
  int64_t b;
  int sh, loss;
  double alpha;
  double cpow[257], cinv[257];
};

// The recurrence of one outer iteration on one CTA with every quantity it
// produces rounded to the state type (G entries as they are read: the Gram
// output in T); corrections accumulate in FP16 (ACC16) or FP32.
template <int ACC16, int ST>
__global__ void __launch_bounds__(1024)
k_rc_recur(const __grid_constant__ RcArgs a) {
  extern __shared__ __align__(16) float uh[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t b = a.b;
  for (int j = 0; j < a.sh; ++j) {
    const int64_t jb = (int64_t)j * b, ldj = gram_ld(j, b);
    const float *Gj = a.G + gram_off(j, b);
    for (int64_t l = warp; l < b; l += nw) {
      const int64_t row = jb + l;
      float corr = 0.f;
      __half corrh = __float2half_rn(0.f);
      if (j > 0) {
        const float *g = Gj + l * ldj;
        for (int64_t c = lane; c < jb; c += 32) {
          const float gv = rnd<ST>(g[c]);
          if (ACC16) corrh = __hfma(__float2half_rn(gv), __float2half_rn(uh[c]), corrh);
          else corr = fmaf(gv, uh[c], corr);
        }
        corr = rnd<ST>(warp_sum<ACC16>(ACC16 ? __half2float(corrh) : corr));
      }
      if (lane == 0) {
        const float z = rnd<ST>((float)a.cpow[j] * a.r[row] -
                                (j > 0 ? (float)(a.alpha * a.cpow[j - 1]) * corr : 0.f));
        const float u = rnd<ST>(dloss<float>(a.loss, z, a.lab[row]));
        if (!isfinite(z) || !isfinite(u)) atomicOr(a.flag, FLAG_NONFINITE);
        uh[row] = rnd<ST>(u * (float)a.cinv[j]);
        a.w[row] = uh[row];
      }
    }
    __syncthreads();
  }
}

// x[col] <- T(c^sh x[col] - alpha c^{sh-1} T(sum_rows Y[row, col] w[row])),
// one thread per column summing the rows in order (fused half FMAs with
// ACC16, else FP32 FMAs).
template <typename TY, int ACC16, int ST>
__global__ void __launch_bounds__(256)
k_rc_update(const TY *Y, int64_t ldy, int64_t rows, int64_t n, const float *w, float decay,
            float stp, float *x, unsigned *flag) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  float acc = 0.f;
  __half acch = __float2half_rn(0.f);
  for (int64_t row = 0; row < rows; ++row) {
    const float yv = ldv(Y + row * ldy + col);
    if (ACC16) acch = __hfma(__float2half_rn(yv), __float2half_rn(w[row]), acch);
    else acc = fmaf(yv, w[row], acc);
  }
  const float g = rnd<ST>(ACC16 ? __half2float(acch) : acc);
  const float xn = rnd<ST>(fmaf(-stp, g, decay * x[col]));
  if (!isfinite(xn)) atomicOr(flag, FLAG_NONFINITE);
  x[col] = xn;
}

template <int ST>
__global__ void k_rc_round(float *x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = rnd<ST>(x[i]);
}

template <typename TY, int ACC16, int ST>
int step_kernels(const void *Y, int64_t ld, int64_t rows, int64_t n, const float *x, float *r,
                 const RcArgs &ra, size_t smem, float decay, float stp, float *xo,
                 unsigned *flag, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((rows + 7) / 8, 148 * 16);
  k_rc_margin<TY, ACC16, ST><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const TY *>(Y), ld,
                                                               rows, n, x, r);
  GLM_CUDA_TRY(cudaGetLastError());
  // the correction sums accumulate in FP16 only end to end (Recipe H); with
  // an FP32 state (Recipe F) the recurrence stays FP32
  constexpr int kRecAcc16 = ACC16 && ST == 2;
  GLM_CUDA_TRY(cudaFuncSetAttribute(k_rc_recur<kRecAcc16, ST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rc_recur<kRecAcc16, ST><<<1, 1024, smem, st>>>(ra);
  GLM_CUDA_TRY(cudaGetLastError());
  k_rc_update<TY, ACC16, ST><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      static_cast<const TY *>(Y), ld, rows, n, ra.w, decay, stp, xo, flag);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // namespace

// CA-SGD under a narrow recipe (see the file comment).  Called from
// glm_ca_sgd_run_ex when opts->accumulate or opts->state_dtype asks for one.
int run_recipe(Handle *h, int s, int64_t b, float eta, float lambda, int64_t iters,
               uint64_t seed, float *x, const glm_ca_opts *o) {
  int gram_dt, gemv_dt, rec64, kahan, gram_impl;
  int64_t ld_gram, ld_gemv;
  uint32_t problem;
  GLM_TRY(resolve_public(h, s, b, eta, lambda, iters, seed, x, o, gram_dt, gemv_dt, rec64, kahan,
                         gram_impl, ld_gram, ld_gemv, problem));
  const int acc16 = o->accumulate == GLM_F16;
  const int st = o->state_dtype == GLM_BF16 ? 1 : (o->state_dtype == GLM_F16 ? 2 : 0);
  if (o->accumulate != GLM_F32 && o->accumulate != GLM_F16)
    return set_error(GLM_EINVAL, "accumulate must be GLM_F32 or GLM_F16");
  if (o->state_dtype != GLM_F32 && o->state_dtype != GLM_BF16 && o->state_dtype != GLM_F16)
    return set_error(GLM_EINVAL, "state_dtype must be GLM_F32, GLM_BF16 or GLM_F16");
  if (acc16 && gemv_dt != GLM_F16)
    return set_error(GLM_EINVAL, "FP16 accumulation needs FP16 GEMV operands");
  if (acc16 && st == 1) return set_error(GLM_EINVAL, "BF16 state accumulates in FP32");
  if (st && (gram_dt != o->state_dtype || gemv_dt != o->state_dtype))
    return set_error(GLM_EINVAL, "a narrow state needs Gram and GEMV operands of that type");
  if (st && rec64 == 1) return set_error(GLM_EINVAL, "a narrow state has no FP64 recurrence");
  if ((int64_t)s * b > 8192) return set_error(GLM_EINVAL, "narrow recipes hold s b <= 8192");
  if (iters == 0) return GLM_OK;
  const int64_t sb = (int64_t)s * b, sbp = round_up(sb, 4);
  // scratch: the step's rows (Gram and GEMV types), labels, row scales, the
  // margins and packed G, the update weights; a run graph that points at a
  // reallocated buffer is dropped
  void *before[6] = {h->ygram[0].ptr, h->ygemv[0].ptr, h->ylab[0].ptr, h->yscale[0].ptr,
                     h->gbuf[0].ptr, h->gbuf[1].ptr};
  int rc = h->ygram[0].ensure((size_t)sb * ld_gram * elem_bytes(gram_dt));
  if (rc == GLM_OK && ld_gemv) rc = h->ygemv[0].ensure((size_t)sb * ld_gemv * elem_bytes(gemv_dt));
  if (rc == GLM_OK) rc = h->ylab[0].ensure((size_t)sbp * 4);
  if (rc == GLM_OK) rc = h->yscale[0].ensure((size_t)sb * 4);
  if (rc == GLM_OK) rc = h->gbuf[0].ensure((size_t)sb * 4);
  if (rc == GLM_OK) rc = h->gbuf[1].ensure((size_t)(sbp + gram_size(s, b)) * 4);
  void *after[6] = {h->ygram[0].ptr, h->ygemv[0].ptr, h->ylab[0].ptr, h->yscale[0].ptr,
                    h->gbuf[0].ptr, h->gbuf[1].ptr};
  if (memcmp(before, after, sizeof(before)) != 0 && h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (rc != GLM_OK) return rc;
  cudaStream_t cs = h->stream;
  if (st == 1) k_rc_round<1><<<8, 256, 0, cs>>>(x, h->n);
  if (st == 2) k_rc_round<2><<<8, 256, 0, cs>>>(x, h->n);
  GLM_CUDA_TRY(cudaGetLastError());
  const double c = 1.0 - (double)eta * (double)lambda;
  float *rbuf = static_cast<float *>(h->gbuf[1].ptr);
  float *G = rbuf + sbp;
  RcArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.r = rbuf;
  ra.G = G;
  ra.lab = static_cast<const float *>(h->ylab[0].ptr);
  ra.w = static_cast<float *>(h->gbuf[0].ptr);
  ra.flag = h->dflag;
  ra.b = b;
  ra.loss = h->loss;
  ra.alpha = (double)eta / (double)b;
  double cp = 1.0;
  for (int j = 0; j <= s; ++j) {
    ra.cpow[j] = cp;
    ra.cinv[j] = 1.0 / cp;
    cp *= c;
  }
  const void *Yv = ld_gemv ? h->ygemv[0].ptr : h->ygram[0].ptr;
  const int64_t ldv_ = ld_gemv ? ld_gemv : ld_gram;
  const int64_t first = o->first_iter;
  for (int64_t t = 0; t < iters; t += s) {
    const int sh = (int)std::min<int64_t>(s, iters - t);
    const int64_t rows = (int64_t)sh * b;
    GatherArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.A = h->A; ga.lda = h->lda; ga.a_dt = h->dtype; ga.colscale = h->colscale;
    ga.A8 = h->A8; ga.rs8 = h->rowscale8; ga.lda8 = h->lda8;
    ga.y = h->y; ga.m = h->m; ga.n = h->n; ga.rows = rows;
    ga.flag = h->dflag;
    ga.q0 = (uint64_t)((first + t) * b); ga.seed = seed; ga.problem = problem;
    ga.out1 = h->ygram[0].ptr; ga.dt1 = gram_dt; ga.ld1 = ld_gram;
    if (ld_gemv) { ga.out2 = h->ygemv[0].ptr; ga.dt2 = gemv_dt; ga.ld2 = ld_gemv; }
    ga.ylab = const_cast<float *>(ra.lab);
    ga.rscale = static_cast<float *>(h->yscale[0].ptr);
    ga.lab_sb = sb;
    ga.lab_sbp = sbp;
    GLM_TRY(launch_gather(ga, cs));
    if (sh >= 2) {
      GramArgs gr;
      memset(&gr, 0, sizeof(gr));
      gr.Y = h->ygram[0].ptr; gr.dt = gram_dt; gr.ld = ld_gram;
      gr.rs = gram_dt == GLM_E4M3 ? static_cast<const float *>(h->yscale[0].ptr) : nullptr;
      gr.nouter = 1; gr.rows = rows; gr.s = s; gr.b = b; gr.n = h->n; gr.G = G;
      gr.flag = h->dflag;
      if (gram_impl == 2) GLM_TRY(launch_gram_tc(gr, cs));
      else if (gram_impl == 3) GLM_TRY(launch_gram_simt_f16acc(gr, cs));
      else if (gram_impl == 4) GLM_TRY(launch_gram_tc_f16acc(gr, cs));
      else GLM_TRY(launch_gram_simt(gr, cs));
    }
    ra.sh = sh;
    const float decay = (float)ra.cpow[sh];
    const float stp = (float)(ra.alpha * ra.cpow[sh - 1]);
    const size_t smem = (size_t)sb * 4;
    if (acc16 && st == 2)
      GLM_TRY((step_kernels<__half, 1, 2>(Yv, ldv_, rows, h->n, x, rbuf, ra, smem, decay, stp, x,
                                          h->dflag, cs)));
    else if (acc16)
      GLM_TRY((step_kernels<__half, 1, 0>(Yv, ldv_, rows, h->n, x, rbuf, ra, smem, decay, stp, x,
                                          h->dflag, cs)));
    else if (st == 2)
      GLM_TRY((step_kernels<__half, 0, 2>(Yv, ldv_, rows, h->n, x, rbuf, ra, smem, decay, stp, x,
                                          h->dflag, cs)));
    else if (st == 1)
      GLM_TRY((step_kernels<__nv_bfloat16, 0, 1>(Yv, ldv_, rows, h->n, x, rbuf, ra, smem, decay,
                                                 stp, x, h->dflag, cs)));
    else
      return set_error(GLM_EINVAL, "no narrow recipe requested");
  }
  return GLM_OK;
}

}  // namespace glm
