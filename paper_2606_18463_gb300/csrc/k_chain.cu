// k_chain.cu -- the x-dependent part of each CA-SGD outer iteration (paper
// Algorithm 1: margin r = Y x, the s-step correction / residual recurrence,
// and the outer update), run by ONE thread-block cluster that keeps the
// iterate x resident in shared memory for a whole chunk of outer iterations.
//
// Work split inside the cluster of C CTAs:
//  * columns: CTA k owns the slice [k nc, (k+1) nc) of x; it computes the
//    partial margins of every gathered row over its slice and, after the
//    recurrence, the update of its slice (Kahan-compensated Y^T u sum);
//  * rows: CTA k owns local rows [k rpb, (k+1) rpb) of every b-row block
//    I_j; it sums the C partial margins of those rows and evaluates their
//    corrected margins
//        z_j = c^j r_j - alpha c^{j-1} sum_{i<j} G_{j,i} (c^{-i} u_i)
//    and residuals, then sends c^{-j} u_j to every CTA.
//
// Warp roles in each CTA (16 warps, CTA barrier = named barrier 1): during
// the recurrence a few row warps each run the serial loop for their own rows
// (FP32: groups of four rows on warps 0, 4, 8, 12; FP64: rows dealt round-
// robin), summing those rows' partial margins themselves, while the other
// warps fold each block's Y_j^T u_j into the update as soon as it lands.
// Everything x-independent is streamed into shared memory ahead of use --
// the CTA's column slice of the rows of Y and their labels (TMA 2D tiles and
// a bulk copy, `ns` outer steps in flight) and the own rows of G_{j,<j}
// (bulk copies: a whole outer step per slot when two steps fit, else one
// block row per slot, up to four slots) -- each copy issued, behind a full
// mbarrier, by lane 0 of one of three worker warps as soon as the slot it
// reuses is known to be free.  x-dependent values travel one way: (vector)
// st.async into the owner's shared memory, completing transaction bytes on
// the owner's mbarrier (one per block of residuals), so an inner step costs
// one DSMEM latency and no cluster or CTA barrier.
// Every wait is bounded (FLAG_TIMEOUT; the kernel then drains its own copies
// and unwinds without writing x).  Slices that do not fit are read from
// global memory directly.
//
// The c^{-i} scaling of the stored residual history turns the per-block
// weights c^{j-1-i} of the ridge-decayed recurrence into one scalar per row
// (c = 1 - eta lambda > 0; the host rejects c^{-(s-1)} beyond 2^60).
#include <cooperative_groups.h>

#include "glm_internal.cuh"

namespace cg = cooperative_groups;

namespace glm {
namespace {

constexpr int kCThreads = 512;              // consumer threads (warps 0..15)
constexpr int kCWarps = kCThreads / 32;
constexpr int kThreads = kCThreads;         // 16 warps: 128 registers a thread
constexpr long long kWaitBudget = 4000000000ll;  // SM cycles (~2 s)
constexpr size_t kSmemMax = 227 * 1024 - 2048;  // leave room for static shared memory
constexpr int kMaxSlots = 4;   // Y slots
constexpr int kMaxGSlots = 4;  // G slots of one block row each

enum { G_NONE = 0, G_STEP = 2, G_BLOCK = 3 };

struct Layout {
  int nc, rpb, C, gmode, ns, ngs, box_rows, nbox;
  int64_t gslot_floats;    // floats per G slot (ngs slots)
  int64_t ylab_off;        // byte offset of the labels inside a Y slot
  int64_t yslot;           // bytes per Y slot
  size_t off_uh, off_rrecv, off_rown, off_yown, off_part, off_bar, off_coef,
      off_rem, off_gbuf, off_ybuf, total;
};

__host__ __device__ inline Layout make_layout(int64_t n, int64_t b, int s, int C,
                                              int tr_bytes, int ev, int want_prefetch) {
  Layout L;
  L.C = C;
  const int64_t per = (n + C - 1) / C;
  int nc = 8;
  while (nc < per) nc *= 2;
  L.nc = nc;
  L.rpb = (int)((b + C - 1) / C);
  const int64_t sb = (int64_t)s * b;
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    size_t o = off;
    off += bytes;
    return o;
  };
  take((size_t)nc * 4, 16);  // x slice at 0
  L.off_uh = take((size_t)sb * tr_bytes, 16);
  L.off_rrecv = take((size_t)C * s * L.rpb * 4, 16);
  L.off_rown = take((size_t)s * L.rpb * tr_bytes, 16);
  L.off_yown = take((size_t)s * L.rpb * 4, 16);
  L.off_part = take((size_t)kCThreads * 8 * 4, 16);
  L.off_bar = take((size_t)(16 + s) * 8, 16);  // 15 pipeline barriers, one per block
  L.off_coef = take((size_t)3 * (s + 1) * tr_bytes, 16);  // c^j, c^-j, alpha c^(j-1)
  L.off_rem = take((size_t)4 * 16 * 4, 16);                 // mapa'd remote addresses
  const size_t base = off;
  // G staging: whole outer step (own rows of every block row) or one block row
  const int64_t g_step = s >= 2 ? (int64_t)L.rpb * gram_size(s, b) / b : 0;
  const int64_t g_blk = s >= 2 ? (int64_t)L.rpb * gram_ld(s - 1, b) : 0;
  L.box_rows = sb >= 256 ? 256 : (int)round_up(sb, 8);
  L.nbox = (int)((sb + L.box_rows - 1) / L.box_rows);
  L.ylab_off = round_up((int64_t)L.nbox * L.box_rows * nc * ev, 128);
  L.yslot = round_up(L.ylab_off + round_up(sb, 4) * 4, 1024);
  const int ystage = want_prefetch && nc <= 256;  // TMA box limit
  L.gmode = G_NONE;
  L.ns = 0;
  L.gslot_floats = 0;
  L.ngs = 2;
  auto fits = [&](int64_t gfl, int ngs, int ns) {
    const size_t g_end = round_up(base, 16) + (size_t)ngs * gfl * 4;
    return round_up(g_end, 1024) + (size_t)ns * L.yslot + (ns ? 1024 : 0) <= kSmemMax;
  };
  const int gm[3] = {G_STEP, G_BLOCK, G_NONE};
  const int64_t gf[3] = {g_step, g_blk, 0};
  bool done = false;
  // staged G first (the recurrence reads it on the critical path): a whole
  // step per slot (two slots), else one block row per slot with as many
  // slots (up to kMaxGSlots, the refill lead) as fit; then as many Y slots
  auto pick = [&](int q, int ngs, int ns) {
    L.ns = ns; L.gmode = gm[q]; L.gslot_floats = gf[q]; L.ngs = ngs; done = true;
  };
  for (int q = 0; q < 3 && ystage && !done; ++q)
    for (int ngs = (q == 1 ? kMaxGSlots : 2); ngs >= 2 && !done; --ngs)
      for (int ns = kMaxSlots; ns >= 2 && !done; --ns)
        if ((q == 2 || s >= 2) && fits(gf[q], ngs, ns)) pick(q, ngs, ns);
  for (int q = 0; q < 2 && !done && want_prefetch && s >= 2; ++q)
    for (int ngs = (q == 1 ? kMaxGSlots : 2); ngs >= 2 && !done; --ngs)
      if (fits(gf[q], ngs, 0)) pick(q, ngs, 0);
  off = base;
  L.off_gbuf = take((size_t)L.ngs * L.gslot_floats * 4, 16);
  L.off_ybuf = take(L.ns ? (size_t)L.ns * L.yslot : 0, 1024);
  L.total = off + (L.ns ? 1024 : 0);  // slack to 1024-align the Y slots at run time
  return L;
}

// Raw 8-element vector loads kept in registers until converted.  `shared`
// selects a plain (shared-memory) load instead of the read-only global path.
template <typename T> struct Raw8;
template <> struct Raw8<float> {
  float4 a, b;
  __device__ __forceinline__ void load(const float *p, bool shared) {
    if (shared) {
      a = reinterpret_cast<const float4 *>(p)[0];
      b = reinterpret_cast<const float4 *>(p)[1];
    } else {
      a = __ldg(reinterpret_cast<const float4 *>(p));
      b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    }
  }
  __device__ __forceinline__ void zero() { a = b = make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ void get(float (&o)[8]) const {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
};
template <> struct Raw8<__nv_bfloat16> {
  uint4 w;
  __device__ __forceinline__ void load(const __nv_bfloat16 *p, bool shared) {
    w = shared ? *reinterpret_cast<const uint4 *>(p) : __ldg(reinterpret_cast<const uint4 *>(p));
  }
  __device__ __forceinline__ void zero() { w = make_uint4(0, 0, 0, 0); }
  __device__ __forceinline__ void get(float (&o)[8]) const {
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(v[i] << 16);
      o[2 * i + 1] = __uint_as_float(v[i] & 0xFFFF0000u);
    }
  }
};
template <> struct Raw8<__half> {
  uint4 w;
  __device__ __forceinline__ void load(const __half *p, bool shared) {
    w = shared ? *reinterpret_cast<const uint4 *>(p) : __ldg(reinterpret_cast<const uint4 *>(p));
  }
  __device__ __forceinline__ void zero() { w = make_uint4(0, 0, 0, 0); }
  __device__ __forceinline__ void get(float (&o)[8]) const {
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&v[i]));
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

constexpr int kRows = 4;  // consecutive rows per thread group in the margin

// Four consecutive entries of the residual history.
__device__ __forceinline__ void load4(const float *p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double *p, double (&o)[4]) {
  const double2 v0 = reinterpret_cast<const double2 *>(p)[0];
  const double2 v1 = reinterpret_cast<const double2 *>(p)[1];
  o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

// Per-lane partial correction dot products of up to four G rows (row i at
// grow + i * rs, 16-byte aligned) with the residual history over [0, jb):
// lane-strided 4-element chunks, then a scalar tail when jb % 4 != 0.  One
// running sum per row, in a fixed order.  Rows past nq re-read the last
// valid row, so every load is in bounds and unconditional and a chunk's five
// loads are in flight together; only their FMAs are skipped (the caller
// discards those sums).
// Instantiated once for staged rows (shared memory) and once for global.
template <typename TR, bool kShared>
__device__ __forceinline__ void rows_dot4(const float *__restrict__ grow, int64_t rs, int nq,
                                          const TR *__restrict__ uh, int jb, int lane,
                                          TR (&acc)[4]) {
  const float *rp[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) rp[i] = grow + (i < nq ? i : nq - 1) * rs;
  const int jb4 = jb & ~3;
#pragma unroll 1  // measured faster than unrolling by 2 or 4
  for (int c = 4 * lane; c < jb4; c += 128) {
    TR u[4];
    load4(uh + c, u);
    float4 g[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 *p = reinterpret_cast<const float4 *>(rp[i] + c);
      g[i] = kShared ? *p : __ldg(p);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < nq) {
        acc[i] = fma((TR)g[i].x, u[0], acc[i]);
        acc[i] = fma((TR)g[i].y, u[1], acc[i]);
        acc[i] = fma((TR)g[i].z, u[2], acc[i]);
        acc[i] = fma((TR)g[i].w, u[3], acc[i]);
      }
    }
  }
  const int c = jb4 + lane;
  if (c < jb) {
    const TR uc = uh[c];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < nq) acc[i] = fma((TR)(kShared ? rp[i][c] : __ldg(rp[i] + c)), uc, acc[i]);
  }
}

// Per-lane partial correction dot product of one G row with the residual
// history over [0, jb) in the recurrence type (FP64): lane-strided 4-element
// chunks into four running sums (independent FMA chains), combined pairwise.
template <typename TR, bool kShared>
__device__ __forceinline__ TR row_dot1(const float *__restrict__ grow, const TR *__restrict__ uh,
                                       int jb, int lane) {
  TR a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const int jb4 = jb & ~3;
  for (int c = 4 * lane; c < jb4; c += 128) {
    TR u[4];
    load4(uh + c, u);
    const float4 *p = reinterpret_cast<const float4 *>(grow + c);
    const float4 g = kShared ? *p : __ldg(p);
    a0 = fma((TR)g.x, u[0], a0);
    a1 = fma((TR)g.y, u[1], a1);
    a2 = fma((TR)g.z, u[2], a2);
    a3 = fma((TR)g.w, u[3], a3);
  }
  const int c = jb4 + lane;
  if (c < jb) a0 = fma((TR)(kShared ? grow[c] : __ldg(grow + c)), uh[c], a0);
  return (a0 + a1) + (a2 + a3);
}

// FP32 loss derivative of the row-group path with the hardware's fast
// exponential and division (relative errors a few ulp: far inside the 1e-5
// iterate tolerance; measured 5 % faster per outer step than the IEEE forms)
__device__ __forceinline__ float dloss_fast(int loss, float z, float y) {
  if (loss == GLM_LOGISTIC) {
    const float t = y * z;
    const float e = __expf(-fabsf(t));
    const float inv = __fdividef(1.f, 1.f + e);
    return -y * ((t >= 0.f) ? e * inv : inv);
  }
  if (loss == GLM_POISSON) return __expf(z) - y;
  return z - y;
}

// Warp totals of four per-lane values, transposed: on return lane L holds the
// total of value L >> 3.  Lanes first split the four values between the two
// half-warps (xor 16), then between quarter-warps (xor 8), then finish each
// value within its group of eight lanes: six shuffles, fixed order.
template <typename TR>
__device__ __forceinline__ TR warp_sum4_t(const TR (&v)[4], int lane) {
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  const TR w0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[2], 16);
  const TR w1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, h16 ? v[1] : v[3], 16);
  TR x = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
  x += __shfl_xor_sync(0xffffffffu, x, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

// Four residuals into one 16-byte-aligned remote slot.
__device__ __forceinline__ void send4(uint32_t ra, const float (&w)[4], uint32_t rb) {
  st_async_v4(ra, w[0], w[1], w[2], w[3], rb);
}

// Bounded wait that also gives up once another thread of the CTA has flagged
// an abort.  Probes back to back, reading the clock and the flag on every
// 32nd probe only (each extra read delays noticing the phase).
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              const volatile int *abort_flag) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (unsigned k = 1;; ++k) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((k & 31) == 0 && (*abort_flag || clock64() - t0 > kWaitBudget)) return false;
  }
}

__device__ __forceinline__ void csync() { named_sync(1, kCThreads); }

template <typename TY, typename TR, int kHot, int kV>
__global__ void __launch_bounds__(kThreads, 1)
k_chain(const __grid_constant__ ChainArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  // kV == 4 instances are launched only for 16-CTA clusters with four own
  // rows per block (the 2^20 x 512, b = 64 shape): those are constants too
  const int C = kV == 4 ? 16 : (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = a.n, b = a.b;
  const int s = a.s;
  const int64_t sb = (int64_t)s * b;
  const Layout L = make_layout(n, b, s, C, (int)sizeof(TR), (int)sizeof(TY), a.prefetch);
  // kHot != 0: a common layout fixed at compile time -- staged Y, update
  // folded in, fewer than 32 vectors per slice, and G a whole step per slot
  // (1) or one block row per slot (2); kV != 0 fixes the slice width too.
  // The once-per-step code is bound by instruction fetch, so these instances
  // carry none of the other layouts' branches.
  const int nc = kV == 4 ? 32 : L.nc, rpb = kV == 4 ? 4 : L.rpb, ns = L.ns;
  const int gmode = kHot == 1 ? (int)G_STEP : (kHot == 2 ? (int)G_BLOCK : L.gmode);
  const int ngs = kHot == 1 ? 2 : L.ngs;
  const int64_t col0 = (int64_t)rank * nc;
  const int64_t l0 = (int64_t)rank * rpb;
  const int nown = (int)max((int64_t)0, min((int64_t)rpb, b - l0));
  // Recurrence row warps.  FP32: up to four, warps 0, 4, 8, 12 (the SM
  // sub-partition of warp id 0 mod 4, which no worker warp shares), each
  // finishing contiguous groups of four own rows, so that a group's
  // residuals leave as one 16-byte store per destination CTA; the other
  // twelve warps fold the update in.  FP64 (whose pipe is the bound): own
  // rows dealt one at a time, round-robin, to warps 0, 1, 2, 3 (one per
  // sub-partition) with the update folded in by warps 4..15, or, with more
  // than four own rows, to every consumer warp, the update following.
  constexpr bool kF64 = sizeof(TR) == 8;
  const bool all_rows = kF64 && nown > 4;
  const int nrw = kF64 ? min(nown, kCWarps) : min((nown + 3) / 4, 4);
  const int nwt = all_rows ? 0 : 3 * kCThreads / 4;  // worker threads
  const int rw = kF64 ? (warp < nrw ? warp : -1)     // row warp index, or -1
                      : ((warp & 3) == 0 && (warp >> 2) < nrw ? warp >> 2 : -1);
  const int wbase_t = kF64 ? (warp >= 4 && !all_rows ? (warp - 4) * 32 : -1)
                           : ((warp & 3) != 0 ? (warp - (warp >> 2) - 1) * 32 : -1);

  extern __shared__ __align__(1024) unsigned char smem[];
  float *xs = reinterpret_cast<float *>(smem);
  TR *uh = reinterpret_cast<TR *>(smem + L.off_uh);
  float *rrecv = reinterpret_cast<float *>(smem + L.off_rrecv);
  TR *rown = reinterpret_cast<TR *>(smem + L.off_rown);
  float *yown = reinterpret_cast<float *>(smem + L.off_yown);
  float *part = reinterpret_cast<float *>(smem + L.off_part);
  float *gbuf = reinterpret_cast<float *>(smem + L.off_gbuf);
  const uint32_t sbase = smem_u32(smem);
  unsigned char *ybuf = smem + (round_up(sbase + L.off_ybuf, 1024) - sbase);
  TR *cpw = reinterpret_cast<TR *>(smem + L.off_coef);   // c^j
  TR *cinw = cpw + (s + 1);                                // c^-j
  TR *zcw = cinw + (s + 1);                                // alpha c^(j-1), j >= 1
  uint32_t *rem = reinterpret_cast<uint32_t *>(smem + L.off_rem);
  __shared__ int s_abort;
  __shared__ int s_fills[kMaxSlots + kMaxGSlots];  // copies issued per Y slot, then G slot

  const uint32_t bar0 = smem_u32(smem + L.off_bar);
  const uint32_t bar_r = bar0;                       // margin partials
  const uint32_t bar_u = bar0 + 8 * 16;              // residuals of block j: + 8 j
  const uint32_t full_g0 = bar0 + 24;                // G slots (x ngs <= 4)
  const uint32_t full_y0 = bar0 + 56;                // Y slots (x kMaxSlots)

  if (tid == 0) {
    for (int i = 0; i < 15; ++i) mbar_init(bar0 + 8 * i, 1);
    for (int j = 0; j < s; ++j) mbar_init(bar_u + 8 * j, 1);
    fence_mbar_init_cluster();
    s_abort = 0;
    for (int k = 0; k < kMaxSlots + kMaxGSlots; ++k) s_fills[k] = 0;
  }
  for (int j = tid; j <= s; j += kThreads) {
    cpw[j] = (TR)a.cpow[j];
    cinw[j] = (TR)a.cinv[j];
    zcw[j] = j > 0 ? (TR)((double)a.alpha * a.cpow[j - 1]) : (TR)0;
  }
  if (tid < C) {  // remote views of the exchange buffers and their barriers
    rem[tid] = mapa(smem_u32(rrecv), tid);
    rem[16 + tid] = mapa(bar_r, tid);
    rem[32 + tid] = mapa(smem_u32(uh), tid);
    rem[48 + tid] = mapa(bar_u, tid);
  }
  for (int c = tid; c < nc; c += kThreads) xs[c] = (col0 + c < n) ? a.x[col0 + c] : 0.f;
  const int64_t gsz = gram_size(s, b);

  // ---- x-independent copies into shared memory --------------------------
  // One thread at a time issues them, each at a point where its target slot
  // is known to be free (no empty barriers): the Y slot of step h - 1 once
  // step h has begun, a G slot once the residuals of the block that read it
  // have landed from every CTA (our own row warps sent theirs after reading
  // it).  Each copy completes transaction bytes on its slot's full barrier.
  const uint32_t ystep_bytes =
      (uint32_t)((int64_t)L.nbox * L.box_rows * nc * sizeof(TY) + round_up(sb, 4) * 4);
  const int nblk = gmode == G_BLOCK ? (a.nouter - 1) * (s - 1) + max(a.s_last - 1, 0)
                                   : 0;  // staged G block rows (j >= 1) of the launch
  auto issue_y = [&](int hh) {  // Y slice and labels of step hh
    if (ns == 0 || hh >= a.nouter) return;
    const int slot = hh % ns;
    const uint32_t bar = full_y0 + 8 * slot;
    const uint32_t dst = smem_u32(ybuf + (int64_t)slot * L.yslot);
    mbar_arrive_expect_tx(bar, ystep_bytes);
    for (int k = 0; k < L.nbox; ++k)
      tma_load_2d(dst + (uint32_t)((int64_t)k * L.box_rows * nc * sizeof(TY)), &a.ymap,
                  (int32_t)col0, (int32_t)((int64_t)hh * sb + (int64_t)k * L.box_rows), bar);
    bulk_load(dst + (uint32_t)L.ylab_off, a.ylab + (int64_t)hh * a.sbp,
              (uint32_t)(round_up(sb, 4) * 4), bar);
    ++s_fills[slot];
  };
  auto issue_gs = [&](int hh) {  // G_STEP: own rows of every block row of step hh
    if (gmode != G_STEP || hh >= a.nouter) return;
    const int shh = (hh == a.nouter - 1) ? a.s_last : s;
    if (shh < 2) return;
    const int slot = hh & 1;
    const uint32_t bar = full_g0 + 8 * slot;
    const float *Gs = a.G + (int64_t)hh * gsz;
    const uint32_t dst = smem_u32(gbuf + slot * L.gslot_floats);
    int64_t bytes = 0;
    for (int j = 1; j < shh; ++j) bytes += (int64_t)nown * gram_ld(j, b) * 4;
    mbar_arrive_expect_tx(bar, (uint32_t)bytes);
    int64_t soff = 0;  // floats into the slot
    for (int j = 1; j < shh; ++j) {
      const int64_t ldj = gram_ld(j, b);
      if (in_bounds(Gs + gram_off(j, b) + (l0 + nown) * ldj <= a.G + (int64_t)a.nouter * gsz &&
                        soff + nown * ldj <= L.gslot_floats,
                    a.flag))
        bulk_load(dst + (uint32_t)(soff * 4), Gs + gram_off(j, b) + l0 * ldj,
                  (uint32_t)(nown * ldj * 4), bar);
      soff += (int64_t)rpb * ldj;
    }
    ++s_fills[kMaxSlots + slot];
  };
  auto issue_gb = [&](int kb) {  // G_BLOCK: block row kb of the launch (j >= 1 rows)
    if (gmode != G_BLOCK || kb >= nblk) return;
    const int hh = kb / (s - 1), j = kb % (s - 1) + 1;
    const int slot = kb % ngs;
    const int64_t ldj = gram_ld(j, b);
    const uint32_t bar = full_g0 + 8 * slot;
    mbar_arrive_expect_tx(bar, (uint32_t)(nown * ldj * 4));
    if (in_bounds(hh < a.nouter &&
                      gram_off(j, b) + (l0 + nown) * ldj <= gsz && nown * ldj <= L.gslot_floats,
                  a.flag))
      bulk_load(smem_u32(gbuf + slot * L.gslot_floats),
                a.G + (int64_t)hh * gsz + gram_off(j, b) + l0 * ldj, (uint32_t)(nown * ldj * 4),
                bar);
    ++s_fills[kMaxSlots + slot];
  };
  if (tid == 0 && ns > 0)  // the Y tensor map is read by every Y fill
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&a.ymap)) : "memory");
  // barriers initialised in every CTA before any remote traffic
  cluster.sync();
  if (tid == 0) {  // fill every Y slot and both G slots
    for (int hh = 0; hh < ns; ++hh) issue_y(hh);
    issue_gs(0);
    issue_gs(1);
    for (int kb = 0; kb < ngs; ++kb) issue_gb(kb);
  }
  bool abort = false;
  if (a.probe > 0) {
    // failure-path probe: thread 0 waits on a barrier that nothing signals
    // (pipeline barrier 1 is otherwise unused) and gives up.  The cluster
    // agrees on the outcome before any data moves between CTAs, so an abort
    // here leaves no exchange store in flight.
    if (tid == 0 && !mbar_wait_bounded(bar0 + 8, 0, a.probe)) atomicOr(&s_abort, 1);
    cluster.sync();
    int any = 0;
    if (tid < C) {
      uint32_t v;
      asm volatile("ld.shared::cluster.u32 %0, [%1];"
                   : "=r"(v) : "r"(mapa(smem_u32(&s_abort), (uint32_t)tid)) : "memory");
      any = v != 0;
    }
    abort = __syncthreads_or(any) != 0;
    cluster.sync();  // every CTA has read every other's flag before any can change
  }

  // ========================= consumer warps ==================================
  const int V = kV ? kV : nc / 8;    // 8-element vectors in the slice
  const int tpr = V < 32 ? V : 32;    // threads per row in the margin
  const int vpt = V / tpr;            // vectors per thread per row
  const int groups = kCThreads / tpr; // row groups (kRows consecutive rows each)
  const int gi = tid / tpr, li = tid % tpr;
  const bool vsend_r = (b % 4 == 0) && (rpb % 4 == 0);            // 4 rows -> one v4
  const int bi = (int)b;  // s b <= 8192: row indices fit 32 bits
  // owner CTA and partial-margin slot of this group's first row in the first
  // pass of the margin loop (the same every outer step)
  const int own_a = ((gi * kRows) % bi) / rpb;
  const int off_a = ((rank * s + (gi * kRows) / bi) * rpb + ((gi * kRows) % bi - own_a * rpb)) * 4;
  const int loss_kind = a.loss;
  unsigned *const flag = a.flag;
  const TY *Y = static_cast<const TY *>(a.Y);
  int gslot = 0;          // G_BLOCK: slot of the next block row (kept as a counter:
  uint32_t gpar = 0;      //   no division on the recurrence's path) and its phase parity
  // update: 0 = folded in block by block by the workers, 1 = after the
  // recurrence by every consumer thread (row groups), 2 = after the
  // recurrence, one thread per 8-column vector (slices wider than that)
  const int emode = kHot ? 0 : ((nwt > 0 && V <= nwt) ? 0 : (V <= kCThreads ? 1 : 2));
  const bool inc_e = emode == 0;
  const int EG = emode == 0 ? nwt / V : (emode == 1 ? kCThreads / V : 1);  // row groups
  // copies are issued by worker thread 0 when workers fold the update in,
  // else by thread 0

  for (int h = 0; h < a.nouter && !abort; ++h) {
    const int sh = (h == a.nouter - 1) ? a.s_last : s;
    const int64_t R = (int64_t)sh * b;
    const int64_t row0 = (int64_t)h * sb;
    const float *Gh = a.G + (int64_t)h * gsz;
    if (tid == 0) mbar_arrive_expect_tx(bar_r, (uint32_t)(C * sh * nown * 4));
    if (warp == 0)  // every block's residuals: b values from the whole cluster
      for (int j = lane; j < sh; j += 32)
        mbar_arrive_expect_tx(bar_u + 8 * j, (uint32_t)(b * sizeof(TR)));
    if (!inc_e && tid == 0 && h >= 1) {  // into step h - 1's slots
      issue_y(h + ns - 1);
      issue_gs(h + 1);
    }
    const bool staged = kHot || ns > 0;
    const TY *Ys;          // row r of this CTA's slice at Ys + r * ystride
    int64_t ystride;
    const float *labs;
    if (staged) {
      const int slot = h % ns;
      // one thread polls; the others park on the named barrier (spinning
      // warps would steal issue slots from the critical path)
      if (tid == 0 &&
          !mbar_wait_bounded(full_y0 + 8 * slot, (uint32_t)((h / ns) & 1), kWaitBudget))
        atomicOr(&s_abort, 1);
      csync();
      Ys = reinterpret_cast<const TY *>(ybuf + (int64_t)slot * L.yslot);
      ystride = nc;
      labs = reinterpret_cast<const float *>(ybuf + (int64_t)slot * L.yslot + L.ylab_off);
    } else {
      Ys = Y + row0 * a.ldy + col0;
      ystride = a.ldy;
      labs = a.ylab + (int64_t)h * a.sbp;
    }

    // ---- A: partial margins over this CTA's column slice --------------------
    for (int64_t rb = 0; rb < R; rb += (int64_t)groups * kRows) {
      const int64_t r0 = rb + (int64_t)gi * kRows;   // this group's first row
      float acc[kRows];
#pragma unroll
      for (int u = 0; u < kRows; ++u) acc[u] = 0.f;
      for (int v0 = 0; v0 < vpt; ++v0) {
        const int64_t col = (int64_t)(li + v0 * tpr) * 8;
        const bool colok = col0 + col < n;
        float xv[8];
        {
          const float4 x0 = reinterpret_cast<const float4 *>(xs + col)[0];
          const float4 x1 = reinterpret_cast<const float4 *>(xs + col)[1];
          xv[0] = x0.x; xv[1] = x0.y; xv[2] = x0.z; xv[3] = x0.w;
          xv[4] = x1.x; xv[5] = x1.y; xv[6] = x1.z; xv[7] = x1.w;
        }
        Raw8<TY> raw[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          // odd groups read their rows in the order 1,0,3,2 so that one load
          // instruction touches rows of both parities (both bank halves)
          const int64_t r = r0 + (u ^ (gi & 1));
          if (r < R && colok) raw[u].load(Ys + r * ystride + col, staged);
          else raw[u].zero();
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          float f[8];
          raw[u].get(f);
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[u] = fmaf(f[i], xv[i], acc[u]);
        }
      }
      if (gi & 1) {  // undo the read order: acc[u] holds row r0 + (u ^ 1)
        float t0 = acc[0]; acc[0] = acc[1]; acc[1] = t0;
        float t2 = acc[2]; acc[2] = acc[3]; acc[3] = t2;
      }
#pragma unroll
      for (int u = 0; u < kRows; ++u)
        for (int off = tpr / 2; off > 0; off >>= 1)
          acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], off);
      if (li == 0 && r0 < R) {
        // owner CTA and slot of row r0 (the first pass's are precomputed:
        // integer division by a run-time divisor is a long instruction sequence)
        int owner, off4;
        if (rb == 0) {
          owner = own_a;
          off4 = off_a;
        } else {
          const int r = (int)r0, j = r / bi, l = r - j * bi;
          owner = l / rpb;
          off4 = ((rank * s + j) * rpb + (l - owner * rpb)) * 4;
        }
        if (vsend_r) {  // the 4 rows share block, owner and a 16-byte slot
          st_async_v4(rem[owner] + (uint32_t)off4, acc[0], acc[1], acc[2], acc[3],
                      rem[16 + owner]);
        } else {
#pragma unroll
          for (int u = 0; u < kRows; ++u) {
            const int r = (int)r0 + u;
            if (r < R) {
              const int ju = r / bi, lu = r - ju * bi;
              const int ow = lu / rpb;
              st_async(rem[ow] + (uint32_t)(((rank * s + ju) * rpb + (lu - ow * rpb)) * 4),
                       acc[u], rem[16 + ow]);
            }
          }
        }
      }
    }
    // ---- D + E: recurrence on the row warps, update on the worker warps ----
    // Row warps run the serial loop over blocks.  Block j of every CTA lands
    // on this CTA's barrier bar_u[j]; a row warp waits on it before block
    // j + 1, and the worker warps wait on it before folding Y_j^T (c^{-j} u_j)
    // into their Kahan sums, so the update runs under the recurrence
    // instead of after it.
    const uint32_t upar = (uint32_t)(h & 1);
    const volatile int *vab = &s_abort;
    if (rw >= 0) {
      const uint32_t ra_u = lane < C ? rem[32 + lane] : 0u;  // CTA lane's residual history
      const uint32_t rb_u = lane < C ? rem[48 + lane] : 0u;  // and its block barriers
      // ---- C (per row warp): every CTA's partial margins of this warp's own
      // rows, summed in a fixed order (four partial sums over the sources),
      // and their labels; then the step's G rows (G_STEP).  No CTA barrier:
      // only this warp reads them.
      int okc = 1;
      if (lane == 0) {
        okc = wait_or_abort(bar_r, (uint32_t)(h & 1), vab);
        if (okc && gmode == G_STEP && sh >= 2)
          okc = wait_or_abort(full_g0 + 8 * (h & 1), (uint32_t)((h >> 1) & 1), vab);
        if (!okc) atomicOr(&s_abort, 1);
      }
      okc = __shfl_sync(0xffffffffu, okc, 0);
      if (okc) {
        const int64_t str = (int64_t)s * rpb;
        auto own_margin = [&](int j, int ll) {
          const float *col = rrecv + (int64_t)j * rpb + ll;
          TR p0 = 0, p1 = 0, p2 = 0, p3 = 0;
          int src = 0;
          for (; src + 4 <= C; src += 4) {
            p0 += (TR)col[(src + 0) * str];
            p1 += (TR)col[(src + 1) * str];
            p2 += (TR)col[(src + 2) * str];
            p3 += (TR)col[(src + 3) * str];
          }
          for (; src < C; ++src) p0 += (TR)col[src * str];
          rown[j * rpb + ll] = (p0 + p1) + (p2 + p3);
          yown[j * rpb + ll] = labs[(int64_t)j * b + l0 + ll];
        };
        if constexpr (kF64) {
          for (int rq = rw; rq < nown; rq += nrw)
            for (int j = lane; j < sh; j += 32) own_margin(j, rq);
        } else {
          for (int q0 = 4 * rw; q0 < nown; q0 += 4 * nrw)
            for (int e = lane; e < 4 * sh; e += 32)
              if (q0 + (e & 3) < nown) own_margin(e >> 2, q0 + (e & 3));
        }
        __syncwarp();
      }
      if (okc) {
        int64_t goff = 0;  // floats into the G_STEP slot
        for (int j = 0; j < sh; ++j) {
          const int64_t ldj = gram_ld(j, b);
          int64_t gofs = 0;  // float offset of this block row's own rows
          if (j > 0) {
            // lane 0 polls; the warp follows
            int ok = 1;
            if (lane == 0) {
              ok = wait_or_abort(bar_u + 8 * (j - 1), upar, vab);
              if (ok && gmode == G_BLOCK)
                ok = wait_or_abort(full_g0 + 8 * gslot, gpar, vab);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
              if (lane == 0) atomicOr(&s_abort, 1);
              break;
            }
            // block j - 1 has landed everywhere: its G slot takes the block
            // row ngs further on
            if (!inc_e && tid == 0 && gmode == G_BLOCK && j >= 2)
              issue_gb(h * (s - 1) + (j - 2) + ngs);
            if (gmode == G_STEP) {
              gofs = (h & 1) * L.gslot_floats + goff;
              goff += (int64_t)rpb * ldj;
            } else if (gmode == G_BLOCK) {
              gofs = gslot * L.gslot_floats;
            } else {
              gofs = gram_off(j, b) + l0 * ldj;
              if (!in_bounds(h < a.nouter && gofs + (int64_t)nown * ldj <= gsz,
                             lane == 0 ? a.flag : nullptr))
                gofs = 0;  // (checked builds) read a row range inside this step's G
            }
          }
          const int jb = (int)(j * b);
          const TR cj = cpw[j], zj = zcw[j], ij = cinw[j];
          if constexpr (kF64) {
            for (int rq = rw; rq < nown; rq += nrw) {  // own rows rw, rw + nrw, ...
              const TR rv = rown[j * rpb + rq];
              const TR yv = (TR)yown[j * rpb + rq];
              TR corr = 0;
              if (j > 0) {
                corr = gmode != G_NONE ? row_dot1<TR, true>(gbuf + gofs + rq * ldj, uh, jb, lane)
                                       : row_dot1<TR, false>(Gh + gofs + rq * ldj, uh, jb, lane);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                  corr += __shfl_xor_sync(0xffffffffu, corr, off);
              }
              const TR z = cj * rv - zj * corr;
              // the residual of the FP64 margin in FP32 (a single rounding; the
              // correction sums, where errors compound with s, stay FP64)
              const TR u = (TR)dloss<float>(loss_kind, (float)z, (float)yv);
              if (lane == 0 && (!isfinite(z) || !isfinite(u))) atomicOr(flag, FLAG_NONFINITE);
              if (lane < C)  // fan-out: lane d writes CTA d's copy of the residual
                st_async(ra_u + (uint32_t)((jb + l0 + rq) * sizeof(TR)), u * ij, rb_u + 8 * j);
            }
          } else {
            for (int q0 = 4 * rw; q0 < nown; q0 += 4 * nrw) {
              // rows q0 + i, i < nq; lane L finishes row L >> 3
              const int nq = min(4, nown - q0);
              const int q = lane >> 3;
              const int rq = q0 + (q < nq ? q : nq - 1);
              const TR rv = rown[j * rpb + rq];
              const TR yv = (TR)yown[j * rpb + rq];
              TR acc[4] = {0, 0, 0, 0};
              if (j > 0) {
                if (gmode != G_NONE && nq == 4)  // the common full group, fixed size
                  rows_dot4<TR, true>(gbuf + gofs + q0 * ldj, ldj, 4, uh, jb, lane, acc);
                else if (gmode != G_NONE)
                  rows_dot4<TR, true>(gbuf + gofs + q0 * ldj, ldj, nq, uh, jb, lane, acc);
                else
                  rows_dot4<TR, false>(Gh + gofs + q0 * ldj, ldj, nq, uh, jb, lane, acc);
              }
              const TR corr = warp_sum4_t(acc, lane);
              const TR z = cj * rv - zj * corr;
              const TR u = dloss_fast(loss_kind, z, yv);
              if (q < nq && (lane & 7) == 0 && (!isfinite(z) || !isfinite(u)))
                atomicOr(flag, FLAG_NONFINITE);
              const TR uw = u * ij;
              TR w[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) w[i] = __shfl_sync(0xffffffffu, uw, 8 * i);
              if (lane < C) {  // fan-out: lane d writes CTA d's copy of the group
                const uint32_t ra = ra_u + (uint32_t)((jb + l0 + q0) * sizeof(TR));
                const uint32_t rb = rb_u + 8 * j;
                if (vsend_r && nq == 4) {
                  send4(ra, w, rb);
                } else {
#pragma unroll
                  for (int i = 0; i < 4; ++i)
                    if (i < nq) st_async(ra + (uint32_t)(i * sizeof(TR)), w[i], rb);
                }
              }
            }
          }
          if (gmode == G_BLOCK && j > 0 && ++gslot == ngs) {
            gslot = 0;
            gpar ^= 1u;
          }
        }
      }
    } else if (wbase_t >= 0 && inc_e) {
      const int wt = wbase_t + lane;  // worker index
      const int eg = wt / V, ev = wt - (wt / V) * V;
      const int64_t ecol = (int64_t)ev * 8;
      float acc[8], cmp[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) { acc[i] = 0.f; cmp[i] = 0.f; }
      // every worker with rows waits on every block (thread 0 always does, so
      // each phase of bar_u is observed before the next step re-arms it)
      const bool cols = col0 + ecol < n;
      const bool rows = eg < EG && eg < b;
      // lane 0 of the first three worker warps refills freed slots (see the
      // issue helpers), each its own kind so that a slow issue (a Y slice:
      // TMA) never holds back a G block row the recurrence needs next:
      // 1 = G block rows, 2 = step h - 1's Y slot, 3 = step h - 1's G slot
      const int role = (lane == 0 && wt < 96) ? (wt >> 5) + 1 : 0;
      // every lane of those three warps follows the block loop (a lone
      // active lane with the rest of its warp parked is slow); elsewhere the
      // lanes with rows form a prefix of the warp (groups ascend with the
      // thread index).  Lane 0 is active whenever any lane is; it polls.
      const bool active = rows || wt < 96;
      const unsigned act = __ballot_sync(0xffffffffu, active);
      if (active) {
        for (int j = 0; j < sh; ++j) {
          int ok = 1;
          if (lane == 0) ok = wait_or_abort(bar_u + 8 * j, upar, vab);
          if (!__shfl_sync(act, ok, 0)) {
            atomicOr(&s_abort, 1);
            break;
          }
          if (role == 1 && gmode == G_BLOCK && j >= 1)
            issue_gb(h * (s - 1) + (j - 1) + ngs);
          if (role == 2 && j == 0 && h >= 1) issue_y(h + ns - 1);
          if (role == 3 && j == 0 && h >= 1) issue_gs(h + 1);
          if (!cols || !rows) continue;
          for (int64_t r = (int64_t)j * b + eg; r < (int64_t)(j + 1) * b; r += EG) {
            Raw8<TY> raw;
            raw.load(Ys + r * ystride + ecol, staged);
            float f[8];
            raw.get(f);
            const float wv = (float)uh[r];
            if (a.kahan) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float yv = fmaf(f[i], wv, -cmp[i]);
                const float t2 = acc[i] + yv;
                cmp[i] = (t2 - acc[i]) - yv;
                acc[i] = t2;
              }
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) acc[i] = fmaf(f[i], wv, acc[i]);
            }
          }
        }
      }
      float r[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) r[i] = acc[i] - cmp[i];
      int pg = eg;  // partial group written
      if (V < 32) {  // lanes V apart share a column vector: one partial per warp
        for (int off = V; off < 32; off <<= 1)
#pragma unroll
          for (int i = 0; i < 8; ++i) r[i] += __shfl_xor_sync(0xffffffffu, r[i], off);
        pg = lane < V ? wt >> 5 : EG;
      }
      if (pg < EG) {
        float4 *pp = reinterpret_cast<float4 *>(part + (int64_t)pg * nc + ecol);
        pp[0] = make_float4(r[0], r[1], r[2], r[3]);
        pp[1] = make_float4(r[4], r[5], r[6], r[7]);
      }
    }
    if (!inc_e && tid == 0) {
      if (!wait_or_abort(bar_u + 8 * (sh - 1), upar, vab)) {
        atomicOr(&s_abort, 1);
      } else if (gmode == G_BLOCK && sh >= 2) {  // the last block's G slot is free
        issue_gb(h * (s - 1) + (sh - 2) + ngs);
      }
    }
    csync();
    if (s_abort) { abort = true; break; }

    // ---- E: x <- c^{sh} x - alpha c^{sh-1} Y^T (c^{-j} u), own slice ---------
    {
      const float decay = (float)cpw[sh];
      const float stp = (float)zcw[sh];
      if (emode != 2) {
        if (emode == 1) {  // row groups of every consumer thread, rows in order
          const int g = tid / V, v = tid - (tid / V) * V;
          const int64_t col = (int64_t)v * 8;
          float acc[8], cmp[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) { acc[i] = 0.f; cmp[i] = 0.f; }
          if (g < EG && col0 + col < n) {
            for (int64_t r = g; r < R; r += EG) {
              Raw8<TY> raw;
              raw.load(Ys + r * ystride + col, staged);
              float f[8];
              raw.get(f);
              const float wv = (float)uh[r];
              if (a.kahan) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  const float yv = fmaf(f[i], wv, -cmp[i]);
                  const float t2 = acc[i] + yv;
                  cmp[i] = (t2 - acc[i]) - yv;
                  acc[i] = t2;
                }
              } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = fmaf(f[i], wv, acc[i]);
              }
            }
          }
          if (g < EG) {
            float4 *pp = reinterpret_cast<float4 *>(part + (int64_t)g * nc + col);
            pp[0] = make_float4(acc[0] - cmp[0], acc[1] - cmp[1], acc[2] - cmp[2], acc[3] - cmp[3]);
            pp[1] = make_float4(acc[4] - cmp[4], acc[5] - cmp[5], acc[6] - cmp[6], acc[7] - cmp[7]);
          }
          csync();
        }
        if (kHot || (emode == 0 && V < 32)) {
          // one partial per worker warp: a thread per column sums them in order
          if (tid < nc) {
            float S = 0.f, cS = 0.f;
            for (int gg = 0; gg < nwt / 32; ++gg) {
              const float yv = part[(int64_t)gg * nc + tid] - cS;
              const float t2 = S + yv;
              cS = (t2 - S) - yv;
              S = t2;
            }
            S -= cS;
            if (col0 + tid < n) {
              const float xn = fmaf(-stp, S, decay * xs[tid]);
              if (!isfinite(xn)) atomicOr(flag, FLAG_NONFINITE);
              xs[tid] = xn;
            }
          }
        } else {
          // TPC threads per column (consecutive lanes), each Kahan-summing EG/TPC
          // row-group partials, then a shuffle tree across the TPC lanes
          const int TPC = nc >= kCThreads ? 1 : kCThreads / nc;
          for (int c0 = 0; c0 < nc; c0 += kCThreads / TPC) {
            const int c = c0 + tid / TPC, q = tid % TPC;
            float S = 0.f, cS = 0.f;
            if (c < nc) {
              for (int gg = q; gg < EG; gg += TPC) {
                const float yv = part[(int64_t)gg * nc + c] - cS;
                const float t2 = S + yv;
                cS = (t2 - S) - yv;
                S = t2;
              }
            }
            S -= cS;
            for (int off = (TPC < 32 ? TPC : 32) / 2; off > 0; off >>= 1)
              S += __shfl_xor_sync(0xffffffffu, S, off);
            if (TPC > 32) {  // more than a warp per column (only nc = 8)
              __shared__ float wred[kCWarps];
              if (lane == 0) wred[warp] = S;
              csync();
              if (q == 0 && c < nc) {
                S = 0.f;
                for (int w = 0; w < TPC / 32; ++w) S += wred[(tid / 32) + w];
              }
              csync();
            }
            if (q == 0 && c < nc && col0 + c < n) {
              const float xn = fmaf(-stp, S, decay * xs[c]);
              if (!isfinite(xn)) atomicOr(flag, FLAG_NONFINITE);
              xs[c] = xn;
            }
          }
        }
      } else {
        // wide slices (more vectors than consumer threads): one thread per vector
        // sums every row of the step in order, after the recurrence
        for (int v = tid; v < V; v += kCThreads) {
          const int64_t col = (int64_t)v * 8;
          if (col0 + col >= n) continue;
          float acc[8], cmp[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) { acc[i] = 0.f; cmp[i] = 0.f; }
          for (int64_t r = 0; r < R; ++r) {
            Raw8<TY> raw;
            raw.load(Ys + r * ystride + col, staged);
            float f[8];
            raw.get(f);
            const float wv = (float)uh[r];
            if (a.kahan) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float yv = fmaf(f[i], wv, -cmp[i]);
                const float t2 = acc[i] + yv;
                cmp[i] = (t2 - acc[i]) - yv;
                acc[i] = t2;
              }
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) acc[i] = fmaf(f[i], wv, acc[i]);
            }
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (col0 + col + i < n) {
              const float xn = fmaf(-stp, acc[i] - cmp[i], decay * xs[col + i]);
              if (!isfinite(xn)) atomicOr(flag, FLAG_NONFINITE);
              xs[col + i] = xn;
            }
          }
        }
        csync();
      }
      csync();
    }
  }
  if (abort) {
    // every consumer has left the step loop (the exits follow a CTA barrier):
    // wait (bounded) for the copies still in flight -- only a slot's last
    // fill can be, and fill i of a slot completes its phase i
    csync();
    if (tid == 0) {
      atomicOr(a.flag, FLAG_TIMEOUT);
      for (int k = 0; k < ns; ++k)
        if (s_fills[k] > 0)
          mbar_wait_bounded(full_y0 + 8 * k, (uint32_t)((s_fills[k] - 1) & 1), kWaitBudget);
      for (int k = 0; k < ngs; ++k)
        if (s_fills[kMaxSlots + k] > 0)
          mbar_wait_bounded(full_g0 + 8 * k, (uint32_t)((s_fills[kMaxSlots + k] - 1) & 1),
                            kWaitBudget);
    }
  } else {
    for (int c = tid; c < nc; c += kCThreads)
      if (col0 + c < n) a.x[col0 + c] = xs[c];
  }
  cluster.sync();
  if (abort && tid == 0) {
    // A CTA that gave up mid-step may have exchange stores (st.async) in
    // flight towards it that no barrier wait will observe.  Every CTA has
    // stopped issuing them (they all passed the barrier above); wait about
    // 20 us, far beyond the DSMEM one-way latency (under 1 us), before this
    // CTA's shared memory is released.
    const long long t0 = clock64();
    while (clock64() - t0 < 40000) {
    }
  }
}

cudaLaunchConfig_t make_cfg(int C, size_t smem, cudaStream_t st, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// every CTA must own at least one row of each block (one-way exchanges rely
// on each CTA taking part in every inner step)
bool cluster_rows_ok(int C, int64_t b) {
  if (C < 1 || (C & (C - 1))) return false;  // shuffle trees need a power of two
  const int64_t rpb = (b + C - 1) / C;
  return (int64_t)(C - 1) * rpb < b;
}

template <typename TY, typename TR, int kHot, int kV>
int launch_k(const ChainArgs &a, const Layout &L, int C, cudaStream_t st) {
  auto kern = k_chain<TY, TR, kHot, kV>;
  GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)L.total));
  if (C > 8)
    GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = make_cfg(C, L.total, st, attr);
  GLM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  return GLM_OK;
}

template <typename TY, typename TR>
int launch_t(const ChainArgs &a0, cudaStream_t st) {
  ChainArgs a = a0;
  const int C = a.cluster;
  const Layout L = make_layout(a.n, a.b, a.s, C, (int)sizeof(TR), (int)sizeof(TY), a.prefetch);
  if (L.total > kSmemMax)
    return set_error(GLM_EUNSUPPORTED, "chain: shared-memory need exceeds 227 KB "
                                       "(reduce s*b or raise the cluster size)");
  if (L.ns) {
    GLM_TRY(make_tmap_2d(&a.ymap, a.Y, a.dt, (uint64_t)a.ldy,
                         (uint64_t)a.nouter * a.s * a.b, (uint64_t)a.ldy * sizeof(TY),
                         (uint32_t)L.nc, (uint32_t)L.box_rows));
  }
  if constexpr (sizeof(TR) == 4) {  // the compile-time instances (see k_chain)
    if (L.ns > 0 && L.nc / 8 < 32) {
      if (L.gmode == G_STEP)
        return (L.nc == 32 && C == 16 && L.rpb == 4) ? launch_k<TY, TR, 1, 4>(a, L, C, st)
                                                     : launch_k<TY, TR, 1, 0>(a, L, C, st);
      if (L.gmode == G_BLOCK)
        return (L.nc == 32 && C == 16 && L.rpb == 4) ? launch_k<TY, TR, 2, 4>(a, L, C, st)
                                                     : launch_k<TY, TR, 2, 0>(a, L, C, st);
    }
  }
  return launch_k<TY, TR, 0, 0>(a, L, C, st);
}

template <typename TY, typename TR>
int max_cluster_t(const ChainArgs &a) {
  auto kern = k_chain<TY, TR, 0, 0>;
  for (int C = 16; C >= 1; C /= 2) {
    if (!cluster_rows_ok(C, a.b)) continue;
    const Layout L = make_layout(a.n, a.b, a.s, C, (int)sizeof(TR), (int)sizeof(TY), a.prefetch);
    if (L.total > kSmemMax) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L.total) != cudaSuccess) { cudaGetLastError(); continue; }
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                      1) != cudaSuccess) { cudaGetLastError(); continue; }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_cfg(C, L.total, 0, attr);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters >= 1) return C;
  }
  return 0;
}

}  // namespace

bool chain_cluster_ok(int C, int64_t b) { return cluster_rows_ok(C, b); }

bool chain_resident_staged(const ChainArgs &a) {
  const int tr = a.rec64 ? 8 : 4;
  const Layout L = make_layout(a.n, a.b, a.s, a.cluster, tr, elem_bytes(a.dt), 1);
  return L.total <= kSmemMax && L.ns > 0 && (a.s < 2 || L.gmode != G_NONE);
}

int chain_max_cluster(const ChainArgs &a) {
  const bool f64 = a.rec64 != 0;
  switch (a.dt) {
  case GLM_F32: case GLM_TF32:
    return f64 ? max_cluster_t<float, double>(a) : max_cluster_t<float, float>(a);
  case GLM_BF16:
    return f64 ? max_cluster_t<__nv_bfloat16, double>(a) : max_cluster_t<__nv_bfloat16, float>(a);
  case GLM_F16:
    return f64 ? max_cluster_t<__half, double>(a) : max_cluster_t<__half, float>(a);
  }
  return 0;
}

int launch_chain(const ChainArgs &a, cudaStream_t st) {
  if (a.nouter <= 0) return GLM_OK;
  if (a.cluster < 1 || a.cluster > 16 || !cluster_rows_ok(a.cluster, a.b))
    return set_error(GLM_EINVAL, "chain: cluster size must be a power of two in 1..16 that "
                                 "leaves every CTA a row of each block");
  const bool f64 = a.rec64 != 0;
  switch (a.dt) {
  case GLM_F32: case GLM_TF32:
    return f64 ? launch_t<float, double>(a, st) : launch_t<float, float>(a, st);
  case GLM_BF16:
    return f64 ? launch_t<__nv_bfloat16, double>(a, st) : launch_t<__nv_bfloat16, float>(a, st);
  case GLM_F16:
    return f64 ? launch_t<__half, double>(a, st) : launch_t<__half, float>(a, st);
  }
  return set_error(GLM_EINVAL, "chain: unsupported GEMV operand type");
}

}  // namespace glm
