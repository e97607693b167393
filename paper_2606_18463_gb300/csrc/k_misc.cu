// k_misc.cu -- risk evaluation (paper Sec. 2.1), the index stream as a
// standalone kernel (Algorithm 1, sampling step), and the one-time dataset
// conversions done by glm_create (storage type with per-column power-of-two
// scales; FP8-E4M3 copy with per-row power-of-two scales).
#include "glm_internal.cuh"

namespace glm {
namespace {

int num_sms() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// ---------------------------------------------------------------------------
// F(x): warp per row, FP32 margin, Kahan-compensated FP32 per-warp sums,
// FP64 block totals written to partials[blockIdx.x].
// ---------------------------------------------------------------------------
constexpr int kLossWarps = 8;

template <typename TS>
__global__ void __launch_bounds__(kLossWarps * 32)
k_loss(const TS *A, int64_t lda, const float *colscale, const float *y, int64_t m,
       int64_t n, const float *x, int loss, double *partials) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float sum = 0.f, comp = 0.f;
  for (int64_t row = (int64_t)blockIdx.x * kLossWarps + warp; row < m;
       row += (int64_t)gridDim.x * kLossWarps) {
    const TS *a = A + row * lda;
    float acc = 0.f;
    for (int64_t c = (int64_t)lane * 8; c < n; c += 256) {
      float v[8];
      Vec8<TS>::load(a + c, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (c + i < n) {
          const float sc = colscale ? __ldg(colscale + c + i) : 1.f;
          acc = fmaf(v[i] * sc, __ldg(x + c + i), acc);
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      const float term = loss_term(loss, acc, __ldg(y + row));
      const float yv = term - comp;
      const float t = sum + yv;
      comp = (t - sum) - yv;
      sum = t;
    }
  }
  __shared__ double wsum[kLossWarps];
  if (lane == 0) wsum[warp] = (double)sum - (double)comp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kLossWarps; ++w) tot += wsum[w];
    partials[blockIdx.x] = tot;
  }
}

__global__ void k_loss_final(const double *partials, int nb, int64_t m, const float *x,
                             int64_t n, float lambda, double *out) {
  __shared__ double red[256];
  double xx = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) xx += (double)x[k] * (double)x[k];
  red[threadIdx.x] = xx;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double risk = 0.0;
    for (int i = 0; i < nb; ++i) risk += partials[i];
    *out = risk / (double)m + 0.5 * (double)lambda * red[0];
  }
}

// ---------------------------------------------------------------------------
// Index stream
// ---------------------------------------------------------------------------
__global__ void k_sample(uint64_t seed, uint64_t problem, int64_t first, int64_t count,
                         int64_t m, int32_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = draw_row(seed, problem, (uint64_t)(first + i), (uint64_t)m);
}

// ---------------------------------------------------------------------------
// Dataset conversions at create time
// ---------------------------------------------------------------------------
__device__ __forceinline__ float load_src(const void *src, int dt, int64_t i) {
  if (dt == GLM_BF16) {
    const uint16_t bits = static_cast<const uint16_t *>(src)[i];
    return __uint_as_float((uint32_t)bits << 16);
  }
  return static_cast<const float *>(src)[i];
}

// sum over rows of v^2 per column, FP64 (one thread per column).
__global__ void k_colsumsq(const void *src, int dt, int64_t rows, int64_t n,
                           int64_t rows_per_block, double *acc) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(rows, r0 + rows_per_block);
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double v = load_src(src, dt, r * n + col);
    s += v * v;
  }
  atomicAdd(acc + col, s);
}

// storage row = round(v / colscale) in the storage type, zero-padded to lda.
__global__ void k_convert(const void *src, int src_dt, int64_t rows, int64_t n,
                          void *dst, int dst_dt, int64_t lda, const float *colscale) {
  const int64_t total = rows * lda;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / lda, c = i - r * lda;
    float v = 0.f;
    if (c < n) {
      v = load_src(src, src_dt, r * n + c);
      if (colscale) v = v / colscale[c];  // power of two: exact
    }
    if (dst_dt == GLM_F32) static_cast<float *>(dst)[i] = v;
    else if (dst_dt == GLM_BF16) static_cast<__nv_bfloat16 *>(dst)[i] = __float2bfloat16_rn(v);
    else static_cast<__half *>(dst)[i] = __float2half_rn(v);
  }
}

// FP8 copy: rho_i = smallest power of two with max|a_i| <= 448 rho_i,
// a8 = E4M3(a / rho) with round-to-nearest-even and saturation.
constexpr int kF8Warps = 8;
__global__ void __launch_bounds__(kF8Warps * 32)
k_fp8_copy(const void *src, int src_dt, int64_t rows, int64_t n, uint8_t *dst,
           int64_t lda8, float *rowscale) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (int64_t)blockIdx.x * kF8Warps + (threadIdx.x >> 5); r < rows;
       r += (int64_t)gridDim.x * kF8Warps) {
    float amax = 0.f;
    for (int64_t c = lane; c < n; c += 32) amax = fmaxf(amax, fabsf(load_src(src, src_dt, r * n + c)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    int k = 0;
    if (amax > 0.f) {
      int e;
      const float f = frexpf(amax, &e);  // amax = f 2^e, f in [0.5, 1)
      k = (f <= 0.875f) ? e - 9 : e - 8;  // 448 = 0.875 * 2^9
    }
    for (int64_t c = lane; c < lda8; c += 32) {
      uint8_t q = 0;
      if (c < n) {
        const float v = ldexpf(load_src(src, src_dt, r * n + c), -k);
        q = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
      }
      dst[r * lda8 + c] = q;
    }
    if (lane == 0) rowscale[r] = ldexpf(1.f, k);
  }
}

__global__ void k_check_labels(const float *y, int64_t m, int loss, unsigned *flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = y[i];
    if (!isfinite(v) || (loss == GLM_LOGISTIC && v != 1.f && v != -1.f) ||
        (loss == GLM_POISSON && v < 0.f))
      atomicOr(flag, FLAG_BAD_LABEL);
  }
}

}  // namespace

int launch_loss(Handle *h, const float *x, float lambda, cudaStream_t st) {
  const int nb = num_sms() * 4;
  switch (h->dtype) {
  case GLM_F32:
    k_loss<float><<<nb, kLossWarps * 32, 0, st>>>(static_cast<const float *>(h->A), h->lda,
        h->colscale, h->y, h->m, h->n, x, h->loss, h->loss_partials);
    break;
  case GLM_BF16:
    k_loss<__nv_bfloat16><<<nb, kLossWarps * 32, 0, st>>>(
        static_cast<const __nv_bfloat16 *>(h->A), h->lda, h->colscale, h->y, h->m, h->n, x,
        h->loss, h->loss_partials);
    break;
  case GLM_F16:
    k_loss<__half><<<nb, kLossWarps * 32, 0, st>>>(static_cast<const __half *>(h->A), h->lda,
        h->colscale, h->y, h->m, h->n, x, h->loss, h->loss_partials);
    break;
  default:
    return set_error(GLM_EINVAL, "loss: bad storage type");
  }
  k_loss_final<<<1, 256, 0, st>>>(h->loss_partials, nb, h->m, x, h->n, lambda, h->loss_out);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

int loss_partials_needed() { return num_sms() * 4; }

int launch_sample(uint64_t seed, uint64_t problem, int64_t first, int64_t count, int64_t m,
                  int32_t *out, cudaStream_t st) {
  if (count <= 0) return GLM_OK;
  const int64_t blocks = (count + 255) / 256;
  k_sample<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(seed, problem, first, count,
                                                                 m, out);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

int launch_colsumsq(const void *src, int src_dt, int64_t rows, int64_t n, double *acc,
                    cudaStream_t st) {
  const int64_t rpb = 4096;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((rows + rpb - 1) / rpb));
  k_colsumsq<<<grid, 256, 0, st>>>(src, src_dt, rows, n, rpb, acc);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

int launch_create_convert(Handle *h, const void *src, int src_dt, int64_t row0, int64_t rows,
                          cudaStream_t st) {
  const int eb = elem_bytes(h->dtype);
  void *dst = static_cast<char *>(h->A) + row0 * h->lda * eb;
  k_convert<<<num_sms() * 8, 256, 0, st>>>(src, src_dt, rows, h->n, dst, h->dtype, h->lda,
                                          h->colscale);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

int launch_fp8_copy(Handle *h, const void *src, int src_dt, int64_t row0, int64_t rows,
                    cudaStream_t st) {
  k_fp8_copy<<<num_sms() * 8, kF8Warps * 32, 0, st>>>(src, src_dt, rows, h->n,
                                                     h->A8 + row0 * h->lda8, h->lda8,
                                                     h->rowscale8 + row0);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

int launch_check_labels(const float *y, int64_t m, int loss, unsigned *flag, cudaStream_t st) {
  k_check_labels<<<num_sms() * 4, 256, 0, st>>>(y, m, loss, flag);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // namespace glm
