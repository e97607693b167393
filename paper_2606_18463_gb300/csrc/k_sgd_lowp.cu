// k_sgd_lowp.cu -- end-to-end low-precision mini-batch SGD: the paper's
// end-to-end FP16 and BF16 baselines (Recipes H and I of the precision-symbol
// table, Sec. 5.3; the end-to-end mini-batch SGD check of Sec. 7, "Accuracy
// gap").  Every quantity a step produces is held in the storage type T (BF16
// or FP16): the margins z = Y x, the residuals u = dL/dz(z, y), the gradient
// g = Y^T u and the weights x <- c x - alpha g, each rounded to T once.  The
// two inner products accumulate in FP32 (BF16 / FP16 input, FP32
// accumulation) or, for FP16, in FP16 with fused multiply-adds (Recipe H's
// FP16 accumulation).  The residual and the update are evaluated in FP32
// before their rounding.
//
// Storage holds A_ik = kappa_k * At_ik with power-of-two column scales
// kappa_k (1 without scales).  The margin reads At_ik against kappa_k x_k
// (exact in FP32) and the gradient's column sum of At_ik u_i is multiplied by
// kappa_k afterwards (exact), so the scales change no rounding.
//
// One CTA of 1024 threads runs the whole chain of steps: x (T values) and
// kappa x sit in shared memory, the b drawn rows are read straight from the
// storage (each step's rows are read twice, the second time from L2).  This
// path is a numerical baseline of the paper's, not a fast path: it keeps
// nothing on the tensor cores and runs on one SM.
#include "glm_baselines.cuh"

namespace glm {
namespace {

constexpr int kThreads = 1024, kWarps = kThreads / 32;

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// v rounded to T (nearest, ties to even), returned as a float
template <typename T> __device__ __forceinline__ float round_t(float v);
template <> __device__ __forceinline__ float round_t<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ float round_t<__half>(float v) {
  return __half2float(__float2half_rn(v));
}

template <typename T, bool kAccF16>
__global__ void __launch_bounds__(kThreads) k_sgd_lowp(LowpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t n = a.n;
  const int b = a.b;
  const int64_t npad = round_up(n, 4);
  float *xw = reinterpret_cast<float *>(smem);  // x_k (T values)
  float *xs = xw + npad;                         // kappa_k x_k
  float *su = xs + npad;                         // residuals of the step (T values)
  float *sy = su + round_up(b, 4);               // labels of the step
  int32_t *sidx = reinterpret_cast<int32_t *>(sy + round_up(b, 4));  // rows of the step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T *A = static_cast<const T *>(a.A);

  for (int64_t k = tid; k < n; k += kThreads) {
    const float xv = round_t<T>(a.x[k]);
    xw[k] = xv;
    xs[k] = (a.colscale ? a.colscale[k] : 1.f) * xv;
  }
  bool bad = false;
  for (int64_t t = 0; t < a.iters; ++t) {
    if (tid < b) {
      const int32_t r = draw_row(a.seed, a.problem, a.q0 + (uint64_t)(t * b + tid),
                                 (uint64_t)a.m);
      const int32_t rr = in_bounds(r >= 0 && r < a.m, a.flag) ? r : 0;
      sidx[tid] = rr;
      sy[tid] = a.y[rr];
    }
    __syncthreads();
    // margins and residuals: warp w takes rows w, w + 32, ...; lane l sums
    // columns l, l + 32, ... and the warp adds its lanes pairwise
    for (int l = warp; l < b; l += kWarps) {
      const T *row = A + (int64_t)sidx[l] * a.lda;
      float z;
      if constexpr (kAccF16) {
        __half acc = __float2half_rn(0.f);
        for (int64_t k = lane; k < n; k += 32)
          acc = __hfma(row[k], __float2half_rn(xs[k]), acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
          acc = __hadd(acc, __shfl_xor_sync(0xffffffffu, acc, off));
        z = __half2float(acc);
      } else {
        float acc = 0.f;
        for (int64_t k = lane; k < n; k += 32) acc = fmaf(to_f<T>(row[k]), xs[k], acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        z = round_t<T>(acc);
      }
      if (lane == 0) {
        const float u = round_t<T>(dloss<float>(a.loss, z, sy[l]));
        su[l] = u;
        bad |= !isfinite(u);
      }
    }
    __syncthreads();
    // gradient column sums in row order and the update
    for (int64_t k = tid; k < n; k += kThreads) {
      float g;
      if constexpr (kAccF16) {
        __half acc = __float2half_rn(0.f);
        for (int l = 0; l < b; ++l)
          acc = __hfma(A[(int64_t)sidx[l] * a.lda + k], __float2half_rn(su[l]), acc);
        g = __half2float(acc);
      } else {
        float acc = 0.f;
        for (int l = 0; l < b; ++l) acc = fmaf(to_f<T>(A[(int64_t)sidx[l] * a.lda + k]), su[l], acc);
        g = round_t<T>(acc);
      }
      const float kap = a.colscale ? a.colscale[k] : 1.f;
      const float xn = round_t<T>(a.c * xw[k] - a.alpha * (kap * g));
      bad |= !isfinite(xn);
      xw[k] = xn;
      xs[k] = kap * xn;
    }
    __syncthreads();
  }
  for (int64_t k = tid; k < n; k += kThreads) a.x[k] = xw[k];
  if (bad) atomicOr(a.flag, FLAG_NONFINITE);
}

size_t lowp_smem(int64_t n, int b) {
  return (size_t)(2 * round_up(n, 4) + 2 * round_up(b, 4)) * 4 + (size_t)round_up(b, 4) * 4;
}

template <typename T, bool kAccF16>
int launch_t(const LowpArgs &a, cudaStream_t st) {
  const size_t shm = lowp_smem(a.n, a.b);
  auto kern = k_sgd_lowp<T, kAccF16>;
  GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)shm));
  kern<<<1, kThreads, shm, st>>>(a);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // namespace

bool lowp_fits(int64_t n, int b) {
  return n >= 1 && b >= 1 && b <= kThreads && lowp_smem(n, b) <= 227 * 1024;
}

int launch_sgd_lowp(const LowpArgs &a, int dt, int acc_f16, cudaStream_t st) {
  if (!lowp_fits(a.n, a.b)) return set_error(GLM_EUNSUPPORTED, "low-precision SGD: n or b too large");
  if (a.iters <= 0) return GLM_OK;
  if (dt == GLM_BF16 && !acc_f16) return launch_t<__nv_bfloat16, false>(a, st);
  if (dt == GLM_F16) return acc_f16 ? launch_t<__half, true>(a, st) : launch_t<__half, false>(a, st);
  return set_error(GLM_EINVAL, "low-precision SGD: storage must be BF16, or FP16 for FP16 accumulation");
}

}  // namespace glm
