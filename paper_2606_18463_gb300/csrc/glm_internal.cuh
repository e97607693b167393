// glm_internal.cuh -- shared device helpers and host-side structures of
// libglm (CA-SGD for GLMs on sm_103a).  Nothing here is visible through the
// C ABI; see include/glm.h for the public contract.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "glm.h"

namespace glm {

// ---------------------------------------------------------------------------
// Error reporting (thread-local last error, see glm_last_error)
// ---------------------------------------------------------------------------
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *what);

#define GLM_CUDA_TRY(expr)                                                     \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess) return ::glm::cuda_error(e_, #expr);                \
  } while (0)

// Device allocation through the failure-injection hook (glm_debug_fail_alloc);
// returns the CUDA status (cudaErrorMemoryAllocation when injected).
cudaError_t dev_malloc(void **p, size_t bytes);

#define GLM_TRY(expr)                                                          \
  do {                                                                         \
    int rc_ = (expr);                                                          \
    if (rc_ != GLM_OK) return rc_;                                             \
  } while (0)

// Device flag bits (one uint32 per handle, raised with atomicOr).
enum : unsigned {
  FLAG_NONFINITE = 1u,
  FLAG_BAD_LABEL = 2u,
  FLAG_TIMEOUT = 4u,
  FLAG_BOUNDS = 8u,  // checked builds: an index fell outside its buffer
};

// Checked builds (-DGLM_CHECKED): a kernel tests each computed index against
// its buffer before the access; an index outside it raises FLAG_BOUNDS (when
// the launch has a flag word) and the access is skipped.  Other builds
// compile the test away.
#ifdef GLM_CHECKED
__device__ __forceinline__ bool in_bounds(bool ok, unsigned *flag) {
  if (!ok && flag) atomicOr(flag, FLAG_BOUNDS);
  return ok;
}
#else
__device__ __forceinline__ bool in_bounds(bool, unsigned *) { return true; }
#endif

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) on the device.
// Counter (k, 0, 0, 0), key (seed, problem); draw q uses word q & 3 of block
// q >> 2 and becomes row floor(U * m / 2^64).
// ---------------------------------------------------------------------------
struct U64x4 {
  uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t k_lo, uint64_t k_hi,
                                               uint64_t c0) {
  const uint64_t kMul0 = 0xD2E7470EE14C6C93ull, kMul1 = 0xCA5A826395121157ull;
  const uint64_t kWeyl0 = 0x9E3779B97F4A7C15ull, kWeyl1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = c0, x1 = 0, x2 = 0, x3 = 0;
  uint64_t k0 = k_lo, k1 = k_hi;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(kMul0, x0), lo0 = kMul0 * x0;
    const uint64_t hi1 = __umul64hi(kMul1, x2), lo1 = kMul1 * x2;
    const uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  U64x4 o;
  o.v[0] = x0; o.v[1] = x1; o.v[2] = x2; o.v[3] = x3;
  return o;
}

__device__ __forceinline__ int32_t draw_row(uint64_t seed, uint64_t problem,
                                            uint64_t q, uint64_t m) {
  const U64x4 blk = philox4x64_10(seed, problem, q >> 2);
  const uint64_t w = blk.v[q & 3];
  return (int32_t)__umul64hi(w, m);
}

// ---------------------------------------------------------------------------
// Element conversions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tf32_round(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Load 8 consecutive storage elements as floats.
template <typename T> struct Vec8;

template <> struct Vec8<float> {
  __device__ __forceinline__ static void load(const float *p, float (&o)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
};

template <> struct Vec8<__nv_bfloat16> {
  __device__ __forceinline__ static void load(const __nv_bfloat16 *p,
                                              float (&o)[8]) {
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(w[i] << 16);
      o[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};

template <> struct Vec8<__half> {
  __device__ __forceinline__ static void load(const __half *p, float (&o)[8]) {
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
      float2 f = __half22float2(h);
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

// Store 8 floats as element type `dt` (GLM_F32 / GLM_TF32 / GLM_BF16 /
// GLM_F16), rounding to nearest (ties to even; TF32 ties away).
__device__ __forceinline__ void store8(void *dst, int dt, const float (&v)[8]) {
  if (dt == GLM_F32 || dt == GLM_TF32) {
    float w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = (dt == GLM_TF32) ? tf32_round(v[i]) : v[i];
    float4 *d = reinterpret_cast<float4 *>(dst);
    d[0] = make_float4(w[0], w[1], w[2], w[3]);
    d[1] = make_float4(w[4], w[5], w[6], w[7]);
  } else if (dt == GLM_BF16) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  } else {  // GLM_F16
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
      w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__host__ __device__ inline int elem_bytes(int dt) {
  switch (dt) {
  case GLM_F32: case GLM_TF32: return 4;
  case GLM_BF16: case GLM_F16: return 2;
  case GLM_E4M3: return 1;
  case GLM_F64: return 8;
  }
  return 0;
}

__host__ __device__ inline int64_t round_up(int64_t v, int64_t a) {
  return (v + a - 1) / a * a;
}

// ---------------------------------------------------------------------------
// Packed strictly block-lower Gram layout (per outer iteration): block row j
// (1 <= j < s) holds b rows of j*b values G[j b + l][0 .. j b), row stride
// gram_ld(j, b) = round_up(j b, 4) floats (16-byte aligned rows), starting
// at float offset gram_off(j, b); gram_size(s, b) floats per iteration.
// ---------------------------------------------------------------------------
__host__ __device__ inline int64_t gram_ld(int64_t j, int64_t b) { return round_up(j * b, 4); }

__host__ __device__ inline int64_t gram_off(int64_t j, int64_t b) {
  int64_t o = 0;
  for (int64_t t = 1; t < j; ++t) o += b * gram_ld(t, b);
  return o;
}

__host__ __device__ inline int64_t gram_size(int64_t s, int64_t b) { return gram_off(s, b); }

// ---------------------------------------------------------------------------
// Inline PTX: mbarriers, cluster-scope asynchronous stores, async copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init_cluster() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
               ::"r"(bar), "r"(bytes) : "memory");
}

// Non-suspending probe of a phase (a thread parked inside try_wait can take
// microseconds to resume, which dominates latency-bound exchanges).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded spin: gives up after `budget` SM clock cycles and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  long long budget) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Address of the same shared-memory location in cluster CTA `rank`.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// Store to a (possibly remote) cluster shared address and signal `bytes`
// on the destination CTA's mbarrier.
__device__ __forceinline__ void st_async(uint32_t raddr, float v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];"
               ::"r"(raddr), "r"(__float_as_uint(v)), "r"(rbar) : "memory");
}

__device__ __forceinline__ void st_async(uint32_t raddr, double v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
               ::"r"(raddr), "l"(__double_as_longlong(v)), "r"(rbar) : "memory");
}

__device__ __forceinline__ void st_async_v4(uint32_t raddr, float a, float b, float c, float d,
                                            uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
      ::"r"(raddr), "f"(a), "f"(b), "f"(c), "f"(d), "r"(rbar) : "memory");
}

__device__ __forceinline__ void st_async_v2(uint32_t raddr, double a, double b, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
      ::"r"(raddr), "d"(a), "d"(b), "r"(rbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// TMA: 2D tiled load of box {x, y} (x innermost) into shared memory,
// completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int32_t x,
                                            int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(bar) : "memory");
}

// TMA: 4D tiled load of box {x, y, z, w} coordinates (x innermost) into
// shared memory, completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *tmap, int32_t x, int32_t y,
                                            int32_t z, int32_t w, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar) : "memory");
}

// TMA: prefetch a 4D box into L2 (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_4d(const void *tmap, int32_t x, int32_t y, int32_t z,
                                                int32_t w) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];"
               ::"l"(tmap), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

// Bulk (non-tensor) copy global -> shared; size and both addresses must be
// multiples of 16 bytes.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Host: encode a 2D row-major tensor map (inner = columns) with a box of
// box_inner x box_outer elements, no swizzle, zero fill out of bounds.
int make_tmap_2d(CUtensorMap *out, const void *base, int dt, uint64_t inner, uint64_t outer,
                 uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer);
// Same with 128-byte swizzling (tcgen05 K-major operand tiles); box_inner
// elements must span exactly 128 bytes.
int make_tmap_2d_sw128(CUtensorMap *out, const void *base, int dt, uint64_t inner,
                       uint64_t outer, uint64_t row_bytes, uint32_t box_inner,
                       uint32_t box_outer);

// Host: encode a 4D FP32 tensor map (dims[0] innermost; byte strides of
// dims 1..3, multiples of 16) with a box of box[0..3] elements, no swizzle,
// zero fill out of bounds.
int make_tmap_4d_f32(CUtensorMap *out, const void *base, const uint64_t dims[4],
                     const uint64_t strides[3], const uint32_t box[4]);

// Bulk prefetch of [src, src + bytes) from global memory into L2 (src
// 16-byte aligned, bytes a multiple of 16); no data reach shared memory.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Losses (paper Sec. 2.1): u = dL/dr and L itself
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T dloss(int loss, T z, T y);

template <> __device__ __forceinline__ float dloss<float>(int loss, float z, float y) {
  if (loss == GLM_LOGISTIC) {
    // -y * sigma(-y z) computed without overflow
    const float t = y * z;
    const float e = expf(-fabsf(t));
    const float inv = __frcp_rn(1.f + e);
    const float sig_neg_t = (t >= 0.f) ? e * inv : inv;
    return -y * sig_neg_t;
  }
  if (loss == GLM_POISSON) return expf(z) - y;
  return z - y;
}

template <> __device__ __forceinline__ double dloss<double>(int loss, double z, double y) {
  if (loss == GLM_LOGISTIC) {
    const double t = y * z;
    const double e = exp(-fabs(t));
    const double sig_neg_t = (t >= 0.0) ? e / (1.0 + e) : 1.0 / (1.0 + e);
    return -y * sig_neg_t;
  }
  if (loss == GLM_POISSON) return exp(z) - y;
  return z - y;
}

__device__ __forceinline__ float loss_term(int loss, float z, float y) {
  if (loss == GLM_LOGISTIC) {
    const float t = y * z;
    return fmaxf(-t, 0.f) + log1pf(expf(-fabsf(t)));
  }
  if (loss == GLM_POISSON) return expf(z) - y * z;
  const float d = z - y;
  return 0.5f * d * d;
}

// ---------------------------------------------------------------------------
// Host-side structures
// ---------------------------------------------------------------------------
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t need);
  void release();
  ~DevBuf() { release(); }
};

struct RunKey {
  int s = 0, gram_dt = 0, gemv_dt = 0, rec64 = 0, kahan = 0, cluster = 0,
      gram_impl = 0, sgd = 0, timing = 0;
  int64_t b = 0, iters = 0, first_iter = 0, chunk = 0, probe = 0;
  int chain = 0;
  uint64_t seed = 0;
  uint32_t problem = 0;
  float eta = 0.f, lambda = 0.f;
  float *x = nullptr;
  bool operator==(const RunKey &o) const;
};

struct Handle {
  int64_t m = 0, n = 0, lda = 0;
  int loss = GLM_LOGISTIC, dtype = GLM_F32;
  void *A = nullptr;            // m x lda storage elements
  float *y = nullptr;           // m labels
  float *colscale = nullptr;    // n power-of-two scales, or null
  uint8_t *A8 = nullptr;        // optional FP8-E4M3 copy, m x lda8
  float *rowscale8 = nullptr;   // its per-row scales
  int64_t lda8 = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  unsigned *dflag = nullptr;    // device flag word
  double *loss_partials = nullptr;
  double *loss_out = nullptr;   // device double
  // run scratch, double-buffered by chunk so the x-independent work of chunk
  // k+1 (side stream) overlaps the chain of chunk k (handle stream)
  DevBuf ygram[2], ygemv[2], ylab[2], yscale[2], gbuf[2];
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_bulk[2] = {}, ev_chain[2] = {};
  // captured run graph
  cudaGraphExec_t graph = nullptr;
  RunKey graph_key;
  // per-kernel timing events of the last timed run: [chunk][kernel][start,end]
  std::vector<cudaEvent_t> tev;
  int64_t tev_chunks = 0;
  int tev_valid = 0;
};

// ---------------------------------------------------------------------------
// Kernel launchers (implemented in the k_*.cu files)
// ---------------------------------------------------------------------------
struct GatherArgs {
  const void *A; int64_t lda; int a_dt;        // storage
  const float *colscale;                       // or null
  const uint8_t *A8; const float *rs8; int64_t lda8;  // FP8 copy (E4M3 out)
  const float *y;
  int64_t m, n, rows;                          // rows to gather
  uint64_t q0, seed, problem;                  // first global draw
  void *out1; int dt1; int64_t ld1;            // primary output (gram operand)
  void *out2; int dt2; int64_t ld2;            // optional second output
  float *ylab; float *rscale;                  // labels / row scales (E4M3)
  int64_t lab_sb, lab_sbp;                     // label of row r at (r/sb)*sbp + r%sb
  unsigned *flag;                              // device flag word (checked builds), or null
};
int launch_gather(const GatherArgs &a, cudaStream_t st);

struct GramArgs {
  const void *Y; int dt; int64_t ld;
  const float *rs;        // row scales (E4M3) or null
  int64_t nouter, rows;   // rows valid in total (tail masking)
  int s; int64_t b, n;
  float *G;
  unsigned *flag;         // device flag word for FLAG_TIMEOUT, or null
  long long probe;        // > 0: failure-path probe wait (SM cycles), else 0
  int tile_n;             // tcgen05 tile width: 0 automatic, 128 or 256
};
int launch_gram_simt(const GramArgs &a, cudaStream_t st);
int launch_gram_tc(const GramArgs &a, cudaStream_t st);
// tcgen05 Gram of F16 operands with an F16 accumulator (Recipe F's Gram slot)
int launch_gram_tc_f16acc(const GramArgs &a, cudaStream_t st);
bool gram_tc_supported(int dt, int64_t ld);

// residual-path division: reciprocal rounded to nearest (one extra rounding)
__device__ __forceinline__ float fast_rcp(float v) { return __frcp_rn(v); }

struct ChainArgs {
  CUtensorMap ymap;       // 2D map over the staged GEMV operand rows (TMA)
  const void *Y; int dt; int64_t ldy;
  const float *ylab;
  const float *G;
  float *x;
  unsigned *flag;
  int64_t n, b;
  int s, s_last, nouter, loss;
  float alpha;
  int rec64, kahan, cluster;
  int64_t sbp;            // labels of outer step h start at ylab[h * sbp]
  int prefetch;           // 1: stage Y / labels / G through shared memory
  long long probe;        // > 0: failure-path probe wait (SM cycles), else 0
  double cpow[257];    // c^j, j = 0..s
  double cinv[257];    // c^-j
};
int launch_chain(const ChainArgs &a, cudaStream_t st);
// 1 when the resident chain (k_chain) stages this shape's Y and G on chip
bool chain_resident_staged(const ChainArgs &a);
// streaming chain (k_chain_stream): layout limits and launch
bool chain_stream_ok(const ChainArgs &a);
int launch_chain_stream(const ChainArgs &a, cudaStream_t st);
int chain_max_cluster(const ChainArgs &a);
bool chain_cluster_ok(int C, int64_t b);

// One problem of one round of a batched run (device table filled by the host).
// The round covers `nouter` outer steps of s b gathered rows each (the last
// one holds s_last b rows; the rest of its rows are zero).
struct BatchItem {
  const void *A; int64_t lda; const float *colscale; const float *y;  // storage
  int64_t m; int n; int a_dt;
  uint64_t seed, problem, q0;   // Philox key and first global draw of the round
  int nouter, s, s_last, b;
  void *Y; int y_dt; int64_t ldy;  // nouter * s * b gathered rows (Gram and GEMV operand)
  float *lab;                      // nouter * s * b labels
  float *G;                        // nouter * gram_size(s, b) floats (packed lower blocks)
  float *x;                        // FP32[n] iterate, in/out
  int loss, kahan;
  float alpha;                     // eta / b
  double c;                        // 1 - eta lambda
  unsigned *flag;                  // the problem's device flag word
};
int launch_gather_batch(const BatchItem *items, int nitems, int64_t max_rows, cudaStream_t st,
                        int a_dt);
// Persistent chain over a work queue: CTAs take items order[0], order[1], ...
// (*queue must be 0 on entry).  Every item of one launch has the same y_dt.
int launch_chain_batch(const BatchItem *items, const int *order, int nitems, int *queue,
                       int y_dt, int rec64, int max_n, int max_sb, int max_s, cudaStream_t st);

int launch_loss(Handle *h, const float *x, float lambda, cudaStream_t st);
// CA-SGD under a narrow precision recipe (glm_ca_opts.accumulate / state_dtype)
int run_recipe(Handle *h, int s, int64_t b, float eta, float lambda, int64_t iters,
               uint64_t seed, float *x, const glm_ca_opts *o);
int launch_sample(uint64_t seed, uint64_t problem, int64_t first, int64_t count,
                  int64_t m, int32_t *out, cudaStream_t st);
int launch_create_convert(Handle *h, const void *src, int src_dt, int64_t row0,
                          int64_t rows, cudaStream_t st);
int launch_colsumsq(const void *src, int src_dt, int64_t rows, int64_t n,
                    double *acc, cudaStream_t st);
int launch_fp8_copy(Handle *h, const void *src, int src_dt, int64_t row0,
                    int64_t rows, cudaStream_t st);
int launch_check_labels(const float *y, int64_t m, int loss, unsigned *flag,
                        cudaStream_t st);

}  // namespace glm
