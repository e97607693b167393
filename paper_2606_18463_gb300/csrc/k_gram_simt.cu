// k_gram_simt.cu -- strictly block-lower Gram G_{j,i} = Y_j Y_i^T, i < j
// (paper Algorithm 1, Gram step; only G_{j,<j} is ever read), with true FP32
// FMA accumulation on the CUDA cores.  It is the FP32 (Recipe A) Gram, which
// must not fall back to TF32, and the reference-shaped fallback for the other
// operand types: BF16 / F16 / TF32 / E4M3 products are exact in FP32, so only
// the accumulation order differs from the tensor-core kernel.
//
// The same tiles with an FP16 accumulator (fused half multiply-adds, k in
// ascending order for every output) give Recipe F's Gram slot: FP16 input
// with FP16 accumulation (the h_a symbol of the paper's precision table).
//
// Tiles of 64 x 64 outputs over the lower triangle of each outer step's
// (s b) x (s b) Gram; 256 threads, 4 x 4 outputs per thread, K staged 32 at a
// time through shared memory (stored k-major so a thread reads 4 rows with
// one 16-byte load).  Long steps use 128 x 128 tiles (below).
#include <type_traits>

#include "glm_baselines.cuh"

namespace glm {
namespace {

constexpr int kTile = 64, kK = 32, kThreads = 256;

__device__ __forceinline__ void load8_any(const void *base, int dt, int64_t off,
                                          float (&o)[8]) {
  if (dt == GLM_F32 || dt == GLM_TF32) {
    Vec8<float>::load(static_cast<const float *>(base) + off, o);
  } else if (dt == GLM_BF16) {
    Vec8<__nv_bfloat16>::load(static_cast<const __nv_bfloat16 *>(base) + off, o);
  } else if (dt == GLM_F16) {
    Vec8<__half>::load(static_cast<const __half *>(base) + off, o);
  } else {  // E4M3 bytes
    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(
        static_cast<const uint8_t *>(base) + off));
    const uint32_t ww[2] = {w.x, w.y};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const __nv_fp8_storage_t byte = (ww[i >> 2] >> (8 * (i & 3))) & 0xFF;
      const __half_raw hr = __nv_cvt_fp8_to_halfraw(byte, __NV_E4M3);
      o[i] = __half2float(__half(hr));
    }
  }
}

template <bool kAccF16>
__global__ void __launch_bounds__(kThreads)
k_gram_simt(GramArgs a) {
  const int64_t sb = (int64_t)a.s * a.b;
  const int64_t g = blockIdx.y;
  const int64_t rows_g = min(sb, a.rows - g * sb);
  // lower-triangular tile pair (TJ >= TI) from the linear block index
  const int64_t t = blockIdx.x;
  int64_t TJ = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (TJ * (TJ + 1) / 2 > t) --TJ;
  while ((TJ + 1) * (TJ + 2) / 2 <= t) ++TJ;
  const int64_t TI = t - TJ * (TJ + 1) / 2;
  const int64_t r0 = TJ * kTile, c0 = TI * kTile;
  const int64_t r_last = min(r0 + kTile, rows_g) - 1;
  if (r_last < r0 || r_last / a.b <= c0 / a.b) return;  // nothing strictly lower

  __shared__ __align__(16) float As[kK][kTile];
  __shared__ __align__(16) float Bs[kK][kTile];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  using Acc = typename std::conditional<kAccF16, __half, float>::type;
  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0.f);
  const int eb = elem_bytes(a.dt);
  const char *Yg = static_cast<const char *>(a.Y) + g * sb * a.ld * eb;
  // loader mapping: 256 threads x 8 k-values = 64 rows x 32 k
  const int lrow = tid >> 2, lk = (tid & 3) * 8;
  for (int64_t k0 = 0; k0 < a.n; k0 += kK) {
    float va[8], vb[8];
    const int64_t ra = r0 + lrow, rb = c0 + lrow;
    if (ra < rows_g && k0 + lk < a.n) load8_any(Yg, a.dt, ra * a.ld + k0 + lk, va);
    else {
#pragma unroll
      for (int i = 0; i < 8; ++i) va[i] = 0.f;
    }
    if (rb < rows_g && k0 + lk < a.n) load8_any(Yg, a.dt, rb * a.ld + k0 + lk, vb);
    else {
#pragma unroll
      for (int i = 0; i < 8; ++i) vb[i] = 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      As[lk + i][lrow] = va[i];
      Bs[lk + i][lrow] = vb[i];
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kK; ++k) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
      const float ar[4] = {av.x, av.y, av.z, av.w};
      const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if constexpr (kAccF16)  // FP16 operands: the conversions are exact
            acc[i][j] = __hfma(__float2half_rn(ar[i]), __float2half_rn(br[j]), acc[i][j]);
          else
            acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
    }
  }
  // epilogue: strictly block-lower entries into the row-block layout
  float *Gg = a.G + g * gram_size(a.s, a.b);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t rho = r0 + ty * 4 + i;
    if (rho >= rows_g) continue;
    const int64_t j = rho / a.b, l = rho - j * a.b;
    float *grow = Gg + gram_off(j, a.b) + l * gram_ld(j, a.b);
    const float sr = a.rs ? a.rs[g * sb + rho] : 1.f;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int64_t col = c0 + tx * 4 + jj;
      if (col < j * a.b &&
          in_bounds(grow + col < a.G + a.nouter * gram_size(a.s, a.b), a.flag)) {
        float v = (float)acc[i][jj];
        if (a.rs) v = v * sr * a.rs[g * sb + col];
        grow[col] = v;
      }
    }
  }
}

// The same products and per-output summation order (one chain per output,
// k ascending) in tiles of 128 x 128 for steps of at least 1,024 rows: each
// thread owns 8 x 8 outputs (rows ty*4 + {0..3} and + 64, columns tx*4 +
// {0..3} and + 64), so shared memory delivers one byte per FMA rather than
// two; K chunks of 16 are double-buffered, the next chunk's rows travelling
// through registers while the current one is consumed.  Results are
// bit-identical to the 64 x 64 kernel's.  Measured on GB300 (FP32, CUDA
// events): the wide shape's step (s b = 2,048, n = 2,048) 32.7 -> 43.9
// TFLOP/s, FP16 accumulation 35.1 -> 50.5; at s b = 512 the 64 x 64 tiles
// stay ahead (29.2 against 27.1).
constexpr int kTile2 = 128, kK2 = 16;

template <bool kAccF16>
__global__ void __launch_bounds__(kThreads, 2)
k_gram_simt128(GramArgs a) {
  const int64_t sb = (int64_t)a.s * a.b;
  const int64_t g = blockIdx.y;
  const int64_t rows_g = min(sb, a.rows - g * sb);
  const int64_t t = blockIdx.x;
  int64_t TJ = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (TJ * (TJ + 1) / 2 > t) --TJ;
  while ((TJ + 1) * (TJ + 2) / 2 <= t) ++TJ;
  const int64_t TI = t - TJ * (TJ + 1) / 2;
  const int64_t r0 = TJ * kTile2, c0 = TI * kTile2;
  const int64_t r_last = min(r0 + kTile2, rows_g) - 1;
  if (r_last < r0 || r_last / a.b <= c0 / a.b) return;  // nothing strictly lower

  __shared__ __align__(16) float As[2][kK2][kTile2];
  __shared__ __align__(16) float Bs[2][kK2][kTile2];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  using Acc = typename std::conditional<kAccF16, __half, float>::type;
  Acc acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = Acc(0.f);
  const int eb = elem_bytes(a.dt);
  const char *Yg = static_cast<const char *>(a.Y) + g * sb * a.ld * eb;
  // loader mapping: 256 threads x 8 k-values = 128 rows x 16 k
  const int lrow = tid >> 1, lk = (tid & 1) * 8;
  const int64_t ra = r0 + lrow, rb = c0 + lrow;
  float va[8], vb[8];
  auto fetch = [&](int64_t k0) {
    if (ra < rows_g && k0 + lk < a.n) load8_any(Yg, a.dt, ra * a.ld + k0 + lk, va);
    else {
#pragma unroll
      for (int i = 0; i < 8; ++i) va[i] = 0.f;
    }
    if (rb < rows_g && k0 + lk < a.n) load8_any(Yg, a.dt, rb * a.ld + k0 + lk, vb);
    else {
#pragma unroll
      for (int i = 0; i < 8; ++i) vb[i] = 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      As[buf][lk + i][lrow] = va[i];
      Bs[buf][lk + i][lrow] = vb[i];
    }
  };
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = 0; k0 < a.n; k0 += kK2) {
    const bool more = k0 + kK2 < a.n;
    if (more) fetch(k0 + kK2);  // in flight while this chunk is consumed
#pragma unroll
    for (int k = 0; k < kK2; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4 + 64]);
      const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if constexpr (kAccF16)  // FP16 operands: the conversions are exact
            acc[i][j] = __hfma(__float2half_rn(ar[i]), __float2half_rn(br[j]), acc[i][j]);
          else
            acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
    }
    if (more) {
      stash(buf ^ 1);  // the other buffer: last read before the previous barrier
      __syncthreads();
      buf ^= 1;
    }
  }
  // epilogue: strictly block-lower entries into the row-block layout
  float *Gg = a.G + g * gram_size(a.s, a.b);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t rho = r0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (rho >= rows_g) continue;
    const int64_t j = rho / a.b, l = rho - j * a.b;
    float *grow = Gg + gram_off(j, a.b) + l * gram_ld(j, a.b);
    const float sr = a.rs ? a.rs[g * sb + rho] : 1.f;
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int64_t col = c0 + tx * 4 + (jj & 3) + (jj >> 2) * 64;
      if (col < j * a.b &&
          in_bounds(grow + col < a.G + a.nouter * gram_size(a.s, a.b), a.flag)) {
        float v = (float)acc[i][jj];
        if (a.rs) v = v * sr * a.rs[g * sb + col];
        grow[col] = v;
      }
    }
  }
}

template <bool kAccF16>
int launch_t(const GramArgs &a, cudaStream_t st) {
  if (a.s < 2 || a.nouter <= 0) return GLM_OK;
  const int64_t sb = (int64_t)a.s * a.b;
  const bool big = sb >= 1024;  // 128 x 128 tiles
  const int64_t T = (sb + (big ? kTile2 : kTile) - 1) / (big ? kTile2 : kTile);
  const int64_t pairs = T * (T + 1) / 2;
  if (pairs > 0x7fffffff || a.nouter > 65535)
    return set_error(GLM_EINVAL, "gram: problem too large for one launch");
  dim3 grid((unsigned)pairs, (unsigned)a.nouter);
  if (big) k_gram_simt128<kAccF16><<<grid, kThreads, 0, st>>>(a);
  else k_gram_simt<kAccF16><<<grid, kThreads, 0, st>>>(a);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // namespace

int launch_gram_simt(const GramArgs &a, cudaStream_t st) { return launch_t<false>(a, st); }

int launch_gram_simt_f16acc(const GramArgs &a, cudaStream_t st) {
  if (a.dt != GLM_F16 || a.rs)
    return set_error(GLM_EINVAL, "FP16-accumulate Gram needs FP16 operands");
  return launch_t<true>(a, st);
}

}  // namespace glm
