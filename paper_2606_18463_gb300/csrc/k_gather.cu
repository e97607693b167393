// k_gather.cu -- sampling + row gather (paper Algorithm 1, sampling and
// gather steps).  One warp per gathered row: lane 0 draws the row index from
// the counter-based Philox stream, the warp streams the row with 16-byte
// loads, dequantizes it (per-column power-of-two scales), rounds it to the
// Gram / GEMV operand types and writes zero-padded rows of a dense Y.
#include "glm_internal.cuh"

namespace glm {
namespace {

constexpr int kWarps = 8;

template <typename TS>
__global__ void __launch_bounds__(kWarps * 32)
k_gather(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp_global = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const TS *A = static_cast<const TS *>(a.A);
  for (int64_t row = warp_global; row < a.rows; row += nwarps) {
    int32_t idx = 0;
    if (lane == 0) idx = draw_row(a.seed, a.problem, a.q0 + (uint64_t)row, (uint64_t)a.m);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (!in_bounds(idx >= 0 && idx < a.m, lane == 0 ? a.flag : nullptr)) continue;
    const TS *src = A + (int64_t)idx * a.lda;
    char *d1 = static_cast<char *>(a.out1) + row * a.ld1 * elem_bytes(a.dt1);
    char *d2 = a.out2 ? static_cast<char *>(a.out2) + row * a.ld2 * elem_bytes(a.dt2)
                      : nullptr;
    const int64_t ldmax = a.ld1 > a.ld2 ? a.ld1 : a.ld2;
    for (int64_t c = (int64_t)lane * 8; c < ldmax; c += 256) {
      float v[8];
      if (c < a.n) {
        Vec8<TS>::load(src + c, v);
        if (a.colscale) {
          const float4 s0 = __ldg(reinterpret_cast<const float4 *>(a.colscale + c));
          const float4 s1 = __ldg(reinterpret_cast<const float4 *>(a.colscale + c) + 1);
          v[0] *= s0.x; v[1] *= s0.y; v[2] *= s0.z; v[3] *= s0.w;
          v[4] *= s1.x; v[5] *= s1.y; v[6] *= s1.z; v[7] *= s1.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
      }
      if (c < a.ld1) store8(d1 + c * elem_bytes(a.dt1), a.dt1, v);
      if (d2 && c < a.ld2) store8(d2 + c * elem_bytes(a.dt2), a.dt2, v);
    }
    if (lane == 0) a.ylab[(row / a.lab_sb) * a.lab_sbp + row % a.lab_sb] = __ldg(a.y + idx);
  }
}

// FP8-E4M3 operand: copy bytes of the per-row-scaled FP8 copy of A (made at
// create time) and the row scale; optionally also the GEMV operand from the
// main storage.
template <typename TS>
__global__ void __launch_bounds__(kWarps * 32)
k_gather_e4m3(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp_global = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kWarps;
  const TS *A = static_cast<const TS *>(a.A);
  for (int64_t row = warp_global; row < a.rows; row += nwarps) {
    int32_t idx = 0;
    if (lane == 0) idx = draw_row(a.seed, a.problem, a.q0 + (uint64_t)row, (uint64_t)a.m);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (!in_bounds(idx >= 0 && idx < a.m, lane == 0 ? a.flag : nullptr)) continue;
    const uint8_t *s8 = a.A8 + (int64_t)idx * a.lda8;
    uint8_t *d1 = static_cast<uint8_t *>(a.out1) + row * a.ld1;
    for (int64_t c = (int64_t)lane * 16; c < a.ld1; c += 512) {
      uint4 w = make_uint4(0, 0, 0, 0);
      if (c < a.lda8) w = __ldg(reinterpret_cast<const uint4 *>(s8 + c));
      *reinterpret_cast<uint4 *>(d1 + c) = w;
    }
    if (a.out2) {
      const TS *src = A + (int64_t)idx * a.lda;
      char *d2 = static_cast<char *>(a.out2) + row * a.ld2 * elem_bytes(a.dt2);
      for (int64_t c = (int64_t)lane * 8; c < a.ld2; c += 256) {
        float v[8];
        if (c < a.n) {
          Vec8<TS>::load(src + c, v);
          if (a.colscale) {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] *= __ldg(a.colscale + c + i);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = 0.f;
        }
        store8(d2 + c * elem_bytes(a.dt2), a.dt2, v);
      }
    }
    if (lane == 0) {
      a.ylab[(row / a.lab_sb) * a.lab_sbp + row % a.lab_sb] = __ldg(a.y + idx);
      a.rscale[row] = __ldg(a.rs8 + idx);
    }
  }
}

}  // namespace

int launch_gather(const GatherArgs &a, cudaStream_t st) {
  if (a.rows <= 0) return GLM_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (a.rows + kWarps - 1) / kWarps;
  const int grid = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  if (a.dt1 == GLM_E4M3) {
    switch (a.a_dt) {
    case GLM_F32: k_gather_e4m3<float><<<grid, kWarps * 32, 0, st>>>(a); break;
    case GLM_BF16: k_gather_e4m3<__nv_bfloat16><<<grid, kWarps * 32, 0, st>>>(a); break;
    case GLM_F16: k_gather_e4m3<__half><<<grid, kWarps * 32, 0, st>>>(a); break;
    default: return set_error(GLM_EINVAL, "gather: bad storage type");
    }
  } else {
    switch (a.a_dt) {
    case GLM_F32: k_gather<float><<<grid, kWarps * 32, 0, st>>>(a); break;
    case GLM_BF16: k_gather<__nv_bfloat16><<<grid, kWarps * 32, 0, st>>>(a); break;
    case GLM_F16: k_gather<__half><<<grid, kWarps * 32, 0, st>>>(a); break;
    default: return set_error(GLM_EINVAL, "gather: bad storage type");
    }
  }
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // namespace glm
