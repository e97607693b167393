// k_chain_stream.cu -- the x-dependent part of each CA-SGD outer iteration
// (paper Algorithm 1: margins, the s-step correction / residual recurrence,
// the outer update) for shapes whose step does not fit on chip: wide rows
// (n in the thousands) and long blocks (s b in the thousands, where the
// strictly block-lower G of one step is hundreds of MB).  One thread-block
// cluster of C CTAs, like k_chain, but everything x-independent is STREAMED
// through three shared-memory rings by a producer warp, so that each SM keeps
// ~100-150 KB of copies in flight (what HBM latency x bandwidth asks for)
// instead of issuing dependent loads:
//   ring M  margin tiles: this CTA's own rows of each block, full width
//           (TMA boxes of 256 columns);
//   ring U  update tiles: every row of each block, this CTA's column slice
//           (TMA boxes of nc columns);
//   ring G  pieces of this CTA's own rows of each block row of G_L, PC
//           columns at a time, in column order: one 4D TMA box per piece
//           where b and PC are multiples of its inner width, else one bulk
//           copy per row; when a step's G is far larger than L2, the boxes
//           are also prefetched into L2 a few pieces ahead.
// Work split in the cluster:
//   * rows: CTA k owns rows [k rpb, (k+1) rpb) of every b-row block; it
//     computes their full margins r = Y x (x is replicated in every CTA), and
//     runs their recurrence
//         z_j = c^j r_j - alpha c^{j-1} sum_{i<j} G_{j,i} (c^{-i} u_i),
//     streaming its G rows; the part of the dot over blocks < j - 1 needs no
//     new residual and runs while block j - 1's residuals are in flight;
//     each residual group goes to every CTA (st.async, one mbarrier per
//     block);
//   * columns: CTA k owns columns [k nc, (k+1) nc) of the update
//         x <- c^s x - alpha c^{s-1} Y^T (c^{-j} u_j),
//     folding each block in as soon as its residuals have landed, then sends
//     its new slice of x to every CTA (the all-gather the next step's
//     margins wait for; it also orders the reuse of the residual history).
// Warp roles (16 warps): warp 15 producer (lane 0 issues copies as ring
// slots free up: G first, then update tiles, then margin tiles); warps 0..14
// margins; then warps 0..3 recurrence (groups of four own rows), warps 4..14
// update.  Every wait is bounded (FLAG_TIMEOUT, then the kernel drains its
// copies and unwinds without writing x).
//
// Recurrence arithmetic (recurrence_f64): 0 FP32; 1 FP64 (history and sums
// FP64; the residual is the FP32 loss derivative of the FP64 margin); 2
// compensated FP32: the residual history in FP32, per-lane Kahan sums of the
// FP32 products, lanes combined in FP64 -- the correction's rounding error
// stays near 2 u_32 sum |G| |c^{-i} u| whatever its length, as with FP64
// sums, at FP32 arithmetic rates (FP64 runs at 1/64 of them on GB300).
#include <cooperative_groups.h>
#include <string.h>

#include <type_traits>

#include "glm_internal.cuh"

namespace cg = cooperative_groups;

namespace glm {
namespace {

constexpr int kThreads = 512;
constexpr int kProducer = 15;    // warp index
constexpr int kCons = 15;        // consumer warps 0..14 (margins)
constexpr int kRowW = 4;         // recurrence warps 0..3
constexpr int kWork = 11;        // update warps 4..14
constexpr long long kWaitBudget = 4000000000ll;
constexpr size_t kSmemMax = 227 * 1024 - 1024;
constexpr int kMaxRing = 4;
constexpr int kMaxGmap = 63;     // G tensor maps (block rows 1..s-1, s <= 64)
constexpr int kPrefetch = 8;     // G pieces prefetched into L2 ahead of their copies

struct SLayout {
  int C, rpb, nc, npad, mbw, mshift, mbox, TM, TU, PC, NM, NU, NG, V, ngrp;
  size_t slot;
  size_t off_x, off_uh, off_rown, off_yown, off_part, off_bar, off_coef, off_rem, off_ring, total;
};

// ev: bytes per Y element; tr: bytes per history entry
__host__ __device__ inline SLayout stream_layout(int64_t n, int64_t b, int s, int C, int ev,
                                                 int tr, int64_t ldy) {
  SLayout L;
  L.C = C;
  L.rpb = (int)((b + C - 1) / C);
  const int64_t per = (n + C - 1) / C;
  L.nc = (int)round_up(per, 8);
  L.npad = L.nc * C;
  // margin tiles: full-width rows in TMA boxes of 256 columns (64 for rows
  // narrower than 256: the staged rows are padded to multiples of 64)
  L.mbw = ldy >= 256 ? 256 : 64;
  L.mshift = ldy >= 256 ? 8 : 6;
  L.mbox = (int)((n + L.mbw - 1) / L.mbw);
  L.V = L.nc / 8;
  L.ngrp = (kWork * 32) / (L.V > 0 ? L.V : 1);
  const int64_t sb = (int64_t)s * b;
  size_t off = 0;
  auto take = [&](size_t bytes, size_t align) {
    off = (off + align - 1) / align * align;
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.off_x = take((size_t)L.npad * 4, 16);
  L.off_uh = take((size_t)sb * tr, 16);
  L.off_rown = take((size_t)s * L.rpb * tr, 16);
  L.off_yown = take((size_t)s * L.rpb * 4, 16);
  L.off_part = take((size_t)L.ngrp * L.nc * 4, 16);
  L.off_bar = take((size_t)(2 + s + 6 * kMaxRing) * 8, 16);  // x, u[s], rings, probe
  L.off_coef = take((size_t)3 * (s + 1) * tr, 16);
  L.off_rem = take((size_t)4 * 16 * 4, 16);
  const size_t fixed = (off + 1023) / 1024 * 1024;
  // rings, in order of preference: double-buffered margin and update tiles
  // and three G pieces of 32 KB; then 32 KB G pieces with single-buffered
  // margin and update tiles, ahead of smaller pieces, since the recurrence
  // pays a fixed cost per piece (long blocks: 2,016 pieces of 256 columns per
  // step at b = 256 ran 28 % slower than half as many of 512); then smaller
  // slots.  At most kMaxRing slots per ring (the barrier block's size).
  L.slot = 0;
  L.NM = L.NU = L.NG = 0;
  const int cand[13][4] = {{2, 2, 3, 32}, {2, 2, 2, 32}, {2, 2, 3, 24}, {2, 2, 2, 24},
                           {1, 1, 2, 32}, {2, 2, 4, 16}, {2, 2, 3, 16}, {2, 2, 2, 16},
                           {1, 2, 2, 32}, {1, 2, 2, 16}, {2, 2, 2, 8}, {1, 1, 2, 16},
                           {1, 1, 2, 8}};
  for (int q = 0; q < 13 && !L.slot; ++q) {
    const size_t sl = (size_t)cand[q][3] * 1024;
    const int nr = cand[q][0] + cand[q][1] + cand[q][2];
    if (fixed + (size_t)nr * sl + 1024 <= kSmemMax) {
      L.slot = sl;
      L.NM = cand[q][0];
      L.NU = cand[q][1];
      L.NG = cand[q][2];
    }
  }
  L.off_ring = fixed;
  L.total = fixed + (size_t)(L.NM + L.NU + L.NG) * L.slot + 1024;  // +1 KB: run-time alignment
  // box heights: at most 256 rows (TMA) and at most one outer step's rows
  const int cap = (int)(sb < 256 ? sb : 256);
  L.TM = L.slot ? (int)(L.slot / ((size_t)L.mbox * L.mbw * ev)) : 0;
  if (L.TM > cap) L.TM = cap;
  L.TU = L.slot ? (int)(L.slot / ((size_t)L.nc * ev)) : 0;
  if (L.TU > cap) L.TU = cap;
  L.PC = L.slot ? (int)((L.slot / ((size_t)L.rpb * 4)) / 4 * 4) : 0;
  return L;
}

template <typename T> struct Raw8s;
template <> struct Raw8s<float> {
  __device__ __forceinline__ static void get(const float *p, float (&o)[8]) {
    const float4 a = reinterpret_cast<const float4 *>(p)[0];
    const float4 b = reinterpret_cast<const float4 *>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
};
template <> struct Raw8s<__nv_bfloat16> {
  __device__ __forceinline__ static void get(const __nv_bfloat16 *p, float (&o)[8]) {
    const uint4 w = *reinterpret_cast<const uint4 *>(p);
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[2 * i] = __uint_as_float(v[i] << 16);
      o[2 * i + 1] = __uint_as_float(v[i] & 0xFFFF0000u);
    }
  }
};
template <> struct Raw8s<__half> {
  __device__ __forceinline__ static void get(const __half *p, float (&o)[8]) {
    const uint4 w = *reinterpret_cast<const uint4 *>(p);
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&v[i]));
      o[2 * i] = f.x;
      o[2 * i + 1] = f.y;
    }
  }
};

// Bounded wait; after 64 back-to-back probes a waiter off the critical path
// (nap > 0) sleeps `nap` ns between probes, so that a dozen waiting warps do
// not crowd the shared-memory pipe the rings' copies and the recurrence use.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              const volatile int *abort_flag,
                                              unsigned nap = 0) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (unsigned k = 1;; ++k) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((k & 31) == 0 && (*abort_flag || clock64() - t0 > kWaitBudget)) return false;
    if (nap && k > 64) __nanosleep(nap);
  }
}

// Warp-uniform wait: every lane probes the barrier (one broadcast read), so
// the loop does not diverge; the outcome is made uniform before returning.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, int lane,
                                          const volatile int *ab, unsigned nap = 0) {
  (void)lane;
  const bool ok = wait_or_abort(bar, parity, ab, nap);
  return __all_sync(0xffffffffu, ok);
}

// Barrier of the consumer warps (named barrier 1) that also ORs a predicate
// over them, so that every consumer takes the same abort decision.
__device__ __forceinline__ bool consumers_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %1, 0;\n\t"
      "barrier.red.or.pred b, 1, %2, a;\n\tselp.u32 %0, 1, 0, b;\n\t}"
      : "=r"(r) : "r"((uint32_t)p), "n"(kCons * 32) : "memory");
  return r != 0;
}

// Warp totals of four per-lane values, transposed: lane L ends with the total
// of value L >> 3 (six shuffles, fixed order).
template <typename T>
__device__ __forceinline__ T sum4_t(const T (&v)[4], int lane) {
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  const T w0 = (h16 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[2], 16);
  const T w1 = (h16 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, h16 ? v[1] : v[3], 16);
  T x = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
  x += __shfl_xor_sync(0xffffffffu, x, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

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

// Partial correction dots of up to four own rows (piece rows q0 + i, row
// stride PC floats in shared memory) with the history uh[c0 ..) over `w`
// columns; lane-strided 4-column chunks and a scalar tail.  MODE 0: FP32,
// 1: FP64, 2: FP32 products with Kahan-compensated per-lane sums (MODE 0 and
// 2 keep two sums per row, over alternate columns; FP64 one).
template <int MODE>
struct DotAcc {
  using TA = typename std::conditional<MODE == 1, double, float>::type;
  TA s[4], c[4], s2[4], c2[4];  // MODE 2: two compensated sums per row
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i) { s[i] = 0; c[i] = 0; s2[i] = 0; c2[i] = 0; }
  }
  // the second compensated sum (MODE 2: columns y, w of each chunk, so that
  // each Kahan chain is half as long; measured 4 % faster per outer step on
  // the large least-squares shape)
  __device__ __forceinline__ void add2(int i, TA p) {
    const float y = p - c2[i];
    const float t = s2[i] + y;
    c2[i] = (t - s2[i]) - y;
    s2[i] = t;
  }
  __device__ __forceinline__ void add(int i, TA p) {
    if (MODE == 2) {
      const float y = p - c[i];
      const float t = s[i] + y;
      c[i] = (t - s[i]) - y;
      s[i] = t;
    } else {
      s[i] += p;
    }
  }
};

template <int MODE, typename TH>
__device__ __forceinline__ void piece_dot4(const float *__restrict__ g, int PC, int nq,
                                           const TH *__restrict__ uh, int w, int lane,
                                           DotAcc<MODE> &acc) {
  using TA = typename DotAcc<MODE>::TA;
  const float *rp[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) rp[i] = g + (i < nq ? i : nq - 1) * PC;
  const int w4 = w & ~3;
#pragma unroll 2
  for (int c = 4 * lane; c < w4; c += 128) {
    TA u[4];
    if constexpr (sizeof(TH) == 8) {
      const double2 v0 = reinterpret_cast<const double2 *>(uh + c)[0];
      const double2 v1 = reinterpret_cast<const double2 *>(uh + c)[1];
      u[0] = v0.x; u[1] = v0.y; u[2] = v1.x; u[3] = v1.y;
    } else {
      const float4 v = *reinterpret_cast<const float4 *>(uh + c);
      u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
    }
    float4 gv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) gv[i] = *reinterpret_cast<const float4 *>(rp[i] + c);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i < nq) {
        if (MODE == 2) {
          acc.add(i, gv[i].x * u[0]);
          acc.add2(i, gv[i].y * u[1]);
          acc.add(i, gv[i].z * u[2]);
          acc.add2(i, gv[i].w * u[3]);
        } else {
          // FP32: columns x, z and y, w into two sums per row (half-length
          // FMA chains; measured 2 % faster per outer step on the wide shape)
          acc.s[i] = fma((TA)gv[i].x, u[0], acc.s[i]);
          if (MODE == 0) acc.c[i] = fma((TA)gv[i].y, u[1], acc.c[i]);
          else acc.s[i] = fma((TA)gv[i].y, u[1], acc.s[i]);
          acc.s[i] = fma((TA)gv[i].z, u[2], acc.s[i]);
          if (MODE == 0) acc.c[i] = fma((TA)gv[i].w, u[3], acc.c[i]);
          else acc.s[i] = fma((TA)gv[i].w, u[3], acc.s[i]);
        }
      }
    }
  }
  const int c = w4 + lane;
  if (c < w) {
    const TA uc = (TA)uh[c];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < nq) {
        if (MODE == 2) acc.add(i, rp[i][c] * (float)uc);
        else acc.s[i] = fma((TA)rp[i][c], uc, acc.s[i]);
      }
  }
}

struct StreamArgs {
  CUtensorMap mmap;       // margin map: box (256 columns, TM rows) over staged Y
  CUtensorMap umap;       // update map: box (nc columns, TU rows)
  const float *ylab;
  const float *G;
  float *x;
  unsigned *flag;
  int64_t n, b, ldy, sbp;
  int s, s_last, nouter, loss, kahan;
  float alpha;
  long long probe;
  double cpow[257], cinv[257];
  // gtma != 0: G pieces arrive as one TMA box each through gmap[j - 1], a 4D
  // view of block row j -- {ginner columns, ld_j / ginner column groups, b
  // rows, outer steps} -- whose box {ginner, PC / ginner, rpb, 1} lands as
  // the piece's rpb rows of PC floats, the layout the row copies produce
  int gtma, ginner;
  int gpf;  // 1: also prefetch G pieces into L2 (gtma; a step's G far larger than L2)
  CUtensorMap gmap[kMaxGmap];
};

template <typename TY, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_chain_stream(const __grid_constant__ StreamArgs a) {
  using TH = typename std::conditional<MODE == 1, double, float>::type;  // history type
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = a.n, b = a.b;
  const int s = a.s;
  const int64_t sb = (int64_t)s * b;
  const SLayout L = stream_layout(n, b, s, C, (int)sizeof(TY), (int)sizeof(TH), a.ldy);
  const int L_NG = L.NG;
  const int L_NM = L.NM;
  const int L_NU = L.NU;
  const int L_PC = L.PC;
  const int L_TM = L.TM;
  const int L_TU = L.TU;
  const int L_V = L.V;
  const int L_mbox = L.mbox;
  const int L_mbw = L.mbw;
  const int L_mshift = L.mshift;
  const int L_nc = L.nc;
  const int L_ngrp = L.ngrp;
  const int L_npad = L.npad;
  const size_t L_off_bar = L.off_bar;
  const size_t L_off_coef = L.off_coef;
  const size_t L_off_part = L.off_part;
  const size_t L_off_rem = L.off_rem;
  const size_t L_off_ring = L.off_ring;
  const size_t L_off_rown = L.off_rown;
  const size_t L_off_uh = L.off_uh;
  const size_t L_off_x = L.off_x;
  const size_t L_off_yown = L.off_yown;
  const int L_rpb = L.rpb;
  const size_t L_slot = L.slot;
  const int rpb = L_rpb, nc = L_nc;
  const int64_t l0 = (int64_t)rank * rpb;
  const int nown = (int)max((int64_t)0, min((int64_t)rpb, b - l0));
  const int64_t col0 = (int64_t)rank * nc;

  extern __shared__ __align__(1024) unsigned char smem[];
  float *xf = reinterpret_cast<float *>(smem + L_off_x);
  TH *uh = reinterpret_cast<TH *>(smem + L_off_uh);
  TH *rown = reinterpret_cast<TH *>(smem + L_off_rown);
  float *yown = reinterpret_cast<float *>(smem + L_off_yown);
  float *part = reinterpret_cast<float *>(smem + L_off_part);
  TH *cpw = reinterpret_cast<TH *>(smem + L_off_coef);
  TH *cinw = cpw + (s + 1);
  TH *zcw = cinw + (s + 1);
  uint32_t *rem = reinterpret_cast<uint32_t *>(smem + L_off_rem);
  const uint32_t sbase = smem_u32(smem);
  unsigned char *ring = smem + (round_up(sbase + L_off_ring, 1024) - sbase);
  unsigned char *ringM = ring;
  unsigned char *ringU = ringM + (size_t)L_NM * L_slot;
  unsigned char *ringG = ringU + (size_t)L_NU * L_slot;
  const uint32_t bar0 = smem_u32(smem + L_off_bar);
  const uint32_t bar_x = bar0;
  const uint32_t bar_u = bar0 + 8;                       // + 8 j, j < s
  const uint32_t fullM = bar0 + 8 * (1 + s);             // + 8 k
  const uint32_t emptyM = fullM + 8 * kMaxRing;
  const uint32_t fullU = emptyM + 8 * kMaxRing;
  const uint32_t emptyU = fullU + 8 * kMaxRing;
  const uint32_t fullG = emptyU + 8 * kMaxRing;
  const uint32_t emptyG = fullG + 8 * kMaxRing;
  const uint32_t probe_bar = emptyG + 8 * kMaxRing;     // never signalled
  __shared__ int s_abort;
  __shared__ int s_fills[3];  // fills issued per ring (M, U, G)

  // row warps: groups of four own rows
  const int ngroups = (nown + 3) / 4;
  const int nrw = min(ngroups, kRowW);

  if (tid == 0) {
    mbar_init(bar_x, 1);
    for (int j = 0; j < s; ++j) mbar_init(bar_u + 8 * j, 1);
    for (int k = 0; k < kMaxRing; ++k) {
      mbar_init(fullM + 8 * k, 1);
      mbar_init(emptyM + 8 * k, kCons);
      mbar_init(fullU + 8 * k, 1);
      mbar_init(emptyU + 8 * k, kWork);
      mbar_init(fullG + 8 * k, 1);
      mbar_init(emptyG + 8 * k, nrw > 0 ? nrw : 1);
    }
    mbar_init(probe_bar, 1);
    fence_mbar_init_cluster();
    s_abort = 0;
    s_fills[0] = s_fills[1] = s_fills[2] = 0;
    // residual blocks of step 0 (every CTA sends b values per block)
    const int sh0 = a.nouter == 1 ? a.s_last : s;
    for (int j = 0; j < sh0; ++j) mbar_arrive_expect_tx(bar_u + 8 * j, (uint32_t)(b * sizeof(TH)));
  }
  for (int j = tid; j <= s; j += kThreads) {
    cpw[j] = (TH)a.cpow[j];
    cinw[j] = (TH)a.cinv[j];
    zcw[j] = j > 0 ? (TH)((double)a.alpha * a.cpow[j - 1]) : (TH)0;
  }
  if (tid < C) {
    rem[tid] = mapa(smem_u32(uh), tid);
    rem[16 + tid] = mapa(bar_u, tid);
    rem[32 + tid] = mapa(smem_u32(xf), tid);
    rem[48 + tid] = mapa(bar_x, tid);
  }
  for (int64_t c = tid; c < L_npad; c += kThreads) xf[c] = c < n ? a.x[c] : 0.f;
  cluster.sync();

  bool abort = false;
  if (a.probe > 0) {  // failure-path probe, agreed by the cluster before any exchange
    if (tid == 0 && !mbar_wait_bounded(probe_bar, 0, a.probe))
      atomicOr(&s_abort, 1);
    cluster.sync();
    int any = 0;
    if (tid < C) {
      uint32_t v;
      asm volatile("ld.shared::cluster.u32 %0, [%1];"
                   : "=r"(v) : "r"(mapa(smem_u32(&s_abort), (uint32_t)tid)) : "memory");
      any = v != 0;
    }
    abort = __syncthreads_or(any) != 0;
    cluster.sync();
  }
  const volatile int *vab = &s_abort;
  const int mt_per_blk = (nown + L_TM - 1) / max(L_TM, 1);     // margin tiles per block
  const int ut_per_blk = (int)((b + L_TU - 1) / max(L_TU, 1));  // update tiles per block
  const int gsz = (int)gram_size(s, b);

  if (warp == kProducer) {
    // ===================== producer ===================================
    if (!abort) {
      // The whole warp runs the loop in lockstep (every lane keeps the same
      // cursors); lane 0 owns the barrier operations and the lanes issue a
      // piece's row copies and a margin tile's boxes side by side.
      // cursors: outer step, block, tile / piece of each ring's sequence
      int mh = 0, mj = 0, mt = 0, mk = 0;           // M: step, block, tile, fill count
      int uhh = 0, uj = 0, ut = 0, uk = 0;
      int gh = 0, gj = 1, gp = 0, gk = 0;
      auto shof = [&](int hh) { return hh == a.nouter - 1 ? a.s_last : s; };
      // G cursor kept incrementally (no per-piece offset sums or divisions):
      // first float of this CTA's own rows of block row gj of step gh, the
      // row stride, the block row's width, the slot and its phase
      const float *grow = nullptr;
      int64_t gld = 0, gjb = 0;
      int gslot = 0;
      uint32_t gphase = 0;
      auto gstart = [&]() {  // (re)position at (gh, gj); skip steps without block rows >= 1
        while (gh < a.nouter && gj >= shof(gh)) { ++gh; gj = 1; gp = 0; }
        if (gh < a.nouter) {
          gjb = (int64_t)gj * b;
          gld = gram_ld(gj, b);
          grow = a.G + (int64_t)gh * gsz + gram_off(gj, b) + l0 * gld;
        }
      };
      gstart();
      if (nown == 0) { mh = a.nouter; gh = a.nouter; }
      // a step's G far larger than L2 (it streams from HBM): a second G
      // cursor runs kPrefetch pieces ahead of the copies into shared memory
      // and prefetches those boxes into L2, so that each piece's copy meets
      // L2 rather than HBM latency
      int ph = 0, pj = 1, pp = 0, pf = 0;  // cursor and pieces prefetched
      auto pnext = [&]() {                 // advance (ph, pj, pp) by one piece
        if ((int64_t)(pp + 1) * L_PC < (int64_t)pj * b) {
          ++pp;
        } else {
          pp = 0;
          ++pj;
        }
        while (ph < a.nouter && pj >= shof(ph)) { ++ph; pj = 1; }
      };
      while (ph < a.nouter && pj >= shof(ph)) { ++ph; pj = 1; }
      if (nown == 0) ph = a.nouter;
      auto prefetch_to = [&](int target) {  // until pf == target (lane 0)
        for (; pf < target && ph < a.nouter; ++pf) {
          if (in_bounds(pj >= 1 && pj - 1 < kMaxGmap, a.flag))
            tma_prefetch_4d(&a.gmap[pj - 1], 0, (int32_t)((int64_t)pp * L_PC / a.ginner),
                            (int32_t)l0, (int32_t)ph);
          pnext();
        }
      };
      if (a.gpf && lane == 0) prefetch_to(kPrefetch);
      const uint32_t mbytes = (uint32_t)((size_t)L_mbox * L_mbw * L_TM * sizeof(TY));
      const uint32_t mboxb = (uint32_t)((size_t)L_mbw * L_TM * sizeof(TY));
      const uint32_t ubytes = (uint32_t)((size_t)nc * L_TU * sizeof(TY));
      int uslot = 0, mslot = 0;
      uint32_t uphase = 0, mphase = 0;
      int32_t uy = 0, my = (int32_t)l0;   // first row of the next update / margin tile
      long long last = clock64();
      while (mh < a.nouter || uhh < a.nouter || gh < a.nouter) {
        bool did = false;
        // G pieces first: the recurrence's critical path
        int fr = 0;
        if (lane == 0)
          fr = (gh < a.nouter && (gk < L_NG || mbar_test_wait(emptyG + 8 * gslot, gphase ^ 1u)))
               | ((uhh < a.nouter && (uk < L_NU || mbar_test_wait(emptyU + 8 * uslot, uphase ^ 1u)))
                  << 1)
               | ((mh < a.nouter && (mk < L_NM || mbar_test_wait(emptyM + 8 * mslot, mphase ^ 1u)))
                  << 2);
        fr = __shfl_sync(0xffffffffu, fr, 0);
        if (fr & 1) {
          const int64_t c0 = (int64_t)gp * L_PC;
          const int64_t w = min((int64_t)L_PC, gjb - c0);
          const uint32_t wb = (uint32_t)(round_up(w, 4) * 4);
          const uint32_t dst = smem_u32(ringG + (size_t)gslot * L_slot);
          const uint32_t full = fullG + 8 * gslot;
          if (a.gtma) {  // the whole piece in one box (rows past b read as zeros)
            if (lane == 0) {
              mbar_arrive_expect_tx(full, (uint32_t)(L_PC * L.rpb * 4));
              if (in_bounds(gj >= 1 && gj - 1 < kMaxGmap, a.flag))
                tma_load_4d(dst, &a.gmap[gj - 1], 0, (int32_t)(c0 / a.ginner), (int32_t)l0,
                            (int32_t)gh, full);
              if (a.gpf) prefetch_to(gk + 1 + kPrefetch);
            }
          } else {
            if (lane == 0) mbar_arrive_expect_tx(full, wb * (uint32_t)nown);
            __syncwarp();
            if (lane < nown &&  // one row of the piece per lane
                in_bounds(grow + c0 + (int64_t)lane * gld + wb / 4 <= a.G + (int64_t)a.nouter * gsz &&
                              c0 + (int64_t)wb / 4 <= gld,
                          a.flag))
              bulk_load(dst + (uint32_t)(lane * L_PC * 4), grow + c0 + (int64_t)lane * gld, wb, full);
          }
          ++gk;
          if (++gslot == L_NG) { gslot = 0; gphase ^= 1u; }
          did = true;
          if (c0 + w >= gjb) {
            // next block row: its offset follows this one's b rows of gld floats
            grow += (int64_t)b * gld - l0 * gld;
            ++gj;
            gp = 0;
            if (gj < shof(gh)) {
              gjb = (int64_t)gj * b;
              gld = gram_ld(gj, b);
              grow += l0 * gld;
            } else {
              ++gh;
              gj = 1;
              gstart();
            }
          } else {
            ++gp;
          }
        }
        if (fr & 2) {
          const uint32_t full = fullU + 8 * uslot;
          if (lane == 0) {
            mbar_arrive_expect_tx(full, ubytes);
            tma_load_2d(smem_u32(ringU + (size_t)uslot * L_slot), &a.umap, (int32_t)col0, uy, full);
          }
          ++uk;
          if (++uslot == L_NU) { uslot = 0; uphase ^= 1u; }
          did = true;
          uy += L_TU;
          if (++ut == ut_per_blk) {
            ut = 0;
            if (++uj == shof(uhh)) { uj = 0; ++uhh; }
            uy = (int32_t)((int64_t)uhh * sb + (int64_t)uj * b);
          }
        }
        if (fr & 4) {
          const uint32_t full = fullM + 8 * mslot;
          if (lane == 0) mbar_arrive_expect_tx(full, mbytes);
          __syncwarp();
          const uint32_t dst = smem_u32(ringM + (size_t)mslot * L_slot);
          if (lane < L_mbox)  // one box of the tile per lane
            tma_load_2d(dst + (uint32_t)lane * mboxb, &a.mmap, lane * L_mbw, my, full);
          ++mk;
          if (++mslot == L_NM) { mslot = 0; mphase ^= 1u; }
          did = true;
          my += L_TM;
          if (++mt == mt_per_blk) {
            mt = 0;
            if (++mj == shof(mh)) { mj = 0; ++mh; }
            my = (int32_t)((int64_t)mh * sb + (int64_t)mj * b + l0);
          }
        }
        if (did) {
          last = clock64();
        } else {
          int give_up = 0;
          if (lane == 0) give_up = *vab || clock64() - last > kWaitBudget;
          if (__shfl_sync(0xffffffffu, give_up, 0)) {
            if (lane == 0) atomicOr(&s_abort, 1);
            break;
          }
          __nanosleep(200);  // nothing to refill: leave the issue slots to the consumers
        }
      }
      if (lane == 0) {
        s_fills[0] = mk;
        s_fills[1] = uk;
        s_fills[2] = gk;
      }
    }
  } else if (!abort) {
    // ===================== consumers ==================================
    int mk = 0, uk = 0, gk = 0;  // fills consumed per ring (same sequences)
    int cms = 0, cus = 0, cgs = 0;           // their slots
    uint32_t cmp_ = 0, cup = 0, cgp = 0;     // and phase parities
    const int ct = tid;          // 0 .. 479
    // update assignment: worker thread -> (8-column vector v, row group g)
    const int wt = tid - kRowW * 32;                   // 0 .. 351 for workers
    const int ev = wt >= 0 ? wt % max(L_V, 1) : 0;
    const int eg = wt >= 0 ? wt / max(L_V, 1) : 0;
    for (int h = 0; h < a.nouter; ++h) {
      const int sh = (h == a.nouter - 1) ? a.s_last : s;
      const float *labh = a.ylab + (int64_t)h * a.sbp;
      // ---- margins of own rows (full width) ------------------------------
      bool ok = h == 0 || warp_wait(bar_x, (uint32_t)((h - 1) & 1), lane, vab, 32);
      for (int j = 0; j < sh && ok && nown > 0; ++j) {
        for (int t = 0; t < mt_per_blk; ++t) {
          const int slot = cms;
          if (!warp_wait(fullM + 8 * slot, cmp_, lane, vab, 32)) {
            ok = false;
            break;
          }
          const TY *tile = reinterpret_cast<const TY *>(ringM + (size_t)slot * L_slot);
          const int r_end = min(L_TM, nown - t * L_TM);
          for (int r = warp; r < r_end; r += kCons) {
            float acc = 0.f;
            for (int c = lane * 8; c < (int)n; c += 256) {
              float v[8];
              Raw8s<TY>::get(tile + ((size_t)(c >> L_mshift) * L_TM + r) * L_mbw +
                                 (c & (L_mbw - 1)), v);
              const float4 x0 = *reinterpret_cast<const float4 *>(xf + c);
              const float4 x1 = *reinterpret_cast<const float4 *>(xf + c + 4);
              acc = fmaf(v[0], x0.x, acc); acc = fmaf(v[1], x0.y, acc);
              acc = fmaf(v[2], x0.z, acc); acc = fmaf(v[3], x0.w, acc);
              acc = fmaf(v[4], x1.x, acc); acc = fmaf(v[5], x1.y, acc);
              acc = fmaf(v[6], x1.z, acc); acc = fmaf(v[7], x1.w, acc);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
              const int q = t * L_TM + r;
              rown[j * rpb + q] = (TH)acc;
              yown[j * rpb + q] = labh[(int64_t)j * b + l0 + q];
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(emptyM + 8 * slot);
          ++mk;
          if (++cms == L_NM) { cms = 0; cmp_ ^= 1u; }
        }
      }
      if (tid == 0 && ok) mbar_arrive_expect_tx(bar_x, (uint32_t)(L_npad * 4));  // this step's x
      if (consumers_or(!ok || *vab)) {  // own margins complete (or give up together)
        atomicOr(&s_abort, 1);
        break;
      }
      // ---- recurrence (warps 0..3) | update (warps 4..14) ---------------
      const uint32_t upar = (uint32_t)(h & 1);
      if (warp < kRowW) {
        const int rw = warp;
        for (int j = 0; j < sh && ok; ++j) {
          const int64_t jb = (int64_t)j * b;
          const int npieces = j > 0 ? (int)((jb + L_PC - 1) / L_PC) : 0;
          // accumulators for this warp's groups (up to two groups of four rows)
          DotAcc<MODE> acc[2];
          acc[0].zero();
          acc[1].zero();
          bool waited = j == 0;  // block j - 1's residuals landed (j = 0: none needed)
          for (int p = 0; p < npieces; ++p) {
            const int64_t c0 = (int64_t)p * L_PC;
            const int w = (int)min((int64_t)L_PC, jb - c0);
            if (!waited && c0 + w > jb - b) {  // the piece reaches block j - 1
              if (!warp_wait(bar_u + 8 * (j - 1), upar, lane, vab)) { ok = false; break; }
              waited = true;
            }
            const int slot = cgs;
            if (rw < nrw) {
              if (!warp_wait(fullG + 8 * slot, cgp, lane, vab)) {
                ok = false;
                break;
              }
              const float *gp = reinterpret_cast<const float *>(ringG + (size_t)slot * L_slot);
#pragma unroll
              for (int gi = 0; gi < 2; ++gi) {  // constant indices keep acc in registers
                const int q0 = 4 * rw + 4 * kRowW * gi;
                if (q0 < nown)
                  piece_dot4<MODE, TH>(gp + (size_t)q0 * L_PC, L_PC, min(4, nown - q0), uh + c0,
                                       w, lane, acc[gi]);
              }
              __syncwarp();
              if (lane == 0) mbar_arrive(emptyG + 8 * slot);
            }
            ++gk;
            if (++cgs == L_NG) { cgs = 0; cgp ^= 1u; }
          }
          if (!ok) break;
          if (j >= 1 && !waited) {
            if (!warp_wait(bar_u + 8 * (j - 1), upar, lane, vab)) { ok = false; break; }
          }
          if (rw < nrw) {
            const TH cj = cpw[j], zj = zcw[j], ij = cinw[j];
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
              const int q0 = 4 * rw + 4 * kRowW * gi;
              if (q0 >= nown) continue;
              const int nq = min(4, nown - q0);
              const int q = lane >> 3;
              const int rq = q0 + (q < nq ? q : nq - 1);
              TH corr;
              if (MODE == 2) {
                double v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  v[i] = ((double)acc[gi].s[i] - (double)acc[gi].c[i]) +
                         ((double)acc[gi].s2[i] - (double)acc[gi].c2[i]);
                corr = (TH)sum4_t<double>(v, lane);
              } else {
                TH v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                  v[i] = MODE == 0 ? (TH)(acc[gi].s[i] + acc[gi].c[i]) : (TH)acc[gi].s[i];
                corr = sum4_t<TH>(v, lane);
              }
              const TH rv = rown[j * rpb + rq];
              const float yv = yown[j * rpb + rq];
              TH z;
              float u;
              if (MODE == 2) {
                const double zd = (double)cj * (double)rv - (double)zj * (double)corr;
                z = (TH)zd;
                u = dloss<float>(a.loss, (float)zd, yv);
              } else if (MODE == 1) {
                z = cj * rv - zj * corr;
                u = dloss<float>(a.loss, (float)z, yv);
              } else {
                z = cj * rv - zj * corr;
                u = dloss_fast(a.loss, (float)z, yv);
              }
              if (q < nq && (lane & 7) == 0 && (!isfinite((float)z) || !isfinite(u)))
                atomicOr(a.flag, FLAG_NONFINITE);
              const TH uw = (TH)u * ij;
              TH wv[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) wv[i] = __shfl_sync(0xffffffffu, uw, 8 * i);
              if (lane < C) {
                const uint32_t ra = rem[lane] + (uint32_t)((jb + l0 + q0) * sizeof(TH));
                const uint32_t rb = rem[16 + lane] + 8 * j;
                if (sizeof(TH) == 4 && nq == 4 && ((jb + l0 + q0) % 4) == 0) {
                  st_async_v4(ra, (float)wv[0], (float)wv[1], (float)wv[2], (float)wv[3], rb);
                } else {
#pragma unroll
                  for (int i = 0; i < 4; ++i)
                    if (i < nq) st_async(ra + (uint32_t)(i * sizeof(TH)), wv[i], rb);
                }
              }
            }
          }
        }
      } else {
        // update workers: Y_j^T (c^{-j} u_j) of this CTA's column slice
        float accv[8], cmp[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { accv[i] = 0.f; cmp[i] = 0.f; }
        for (int j = 0; j < sh && ok; ++j) {
          if (!warp_wait(bar_u + 8 * j, upar, lane, vab, 256)) { ok = false; break; }
          for (int t = 0; t < ut_per_blk; ++t) {
            const int slot = cus;
            if (!warp_wait(fullU + 8 * slot, cup, lane, vab, 256)) {
              ok = false;
              break;
            }
            const TY *tile = reinterpret_cast<const TY *>(ringU + (size_t)slot * L_slot);
            const int r_end = (int)min((int64_t)L_TU, b - (int64_t)t * L_TU);
            if (eg < L_ngrp && col0 + ev * 8 < n) {
              for (int r = eg; r < r_end; r += L_ngrp) {
                float f[8];
                Raw8s<TY>::get(tile + (size_t)r * nc + ev * 8, f);
                const float wv = (float)uh[(int64_t)j * b + (int64_t)t * L_TU + r];
                if (a.kahan) {
#pragma unroll
                  for (int i = 0; i < 8; ++i) {
                    const float yv = fmaf(f[i], wv, -cmp[i]);
                    const float t2 = accv[i] + yv;
                    cmp[i] = (t2 - accv[i]) - yv;
                    accv[i] = t2;
                  }
                } else {
#pragma unroll
                  for (int i = 0; i < 8; ++i) accv[i] = fmaf(f[i], wv, accv[i]);
                }
              }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(emptyU + 8 * slot);
            ++uk;
            if (++cus == L_NU) { cus = 0; cup ^= 1u; }
          }
        }
        if (eg < L_ngrp) {
          float4 *pp = reinterpret_cast<float4 *>(part + (size_t)eg * nc + ev * 8);
          pp[0] = make_float4(accv[0] - cmp[0], accv[1] - cmp[1], accv[2] - cmp[2], accv[3] - cmp[3]);
          pp[1] = make_float4(accv[4] - cmp[4], accv[5] - cmp[5], accv[6] - cmp[6], accv[7] - cmp[7]);
        }
      }
      if (consumers_or(!ok || *vab)) {
        atomicOr(&s_abort, 1);
        break;
      }
      // ---- x <- c^sh x - alpha c^{sh-1} (sum of partials), own slice, then
      //      the all-gather (residual barriers of the next step armed first)
      if (tid == 0 && h + 1 < a.nouter) {
        const int sh2 = (h + 1 == a.nouter - 1) ? a.s_last : s;
        for (int j = 0; j < sh2; ++j)
          mbar_arrive_expect_tx(bar_u + 8 * j, (uint32_t)(b * sizeof(TH)));
      }
      named_sync(1, kCons * 32);
      const float decay = (float)cpw[sh], stp = (float)zcw[sh];
      for (int c = ct; c < nc; c += kCons * 32) {
        float S = 0.f, cS = 0.f;
        for (int g = 0; g < L_ngrp; ++g) {
          const float yv = part[(size_t)g * nc + c] - cS;
          const float t2 = S + yv;
          cS = (t2 - S) - yv;
          S = t2;
        }
        S -= cS;
        float xn = 0.f;
        if (col0 + c < n) {
          xn = fmaf(-stp, S, decay * xf[col0 + c]);
          if (!isfinite(xn)) atomicOr(a.flag, FLAG_NONFINITE);
        }
        part[c] = xn;  // group 0's row of partials is free now: stage the new slice
      }
      named_sync(1, kCons * 32);
      // send the new slice to every CTA (itself included), 16 bytes at a time
      for (int e = ct; e < C * (nc / 4); e += kCons * 32) {
        const int d = e / (nc / 4), v4 = e - d * (nc / 4);
        const float4 xv = reinterpret_cast<const float4 *>(part)[v4];
        st_async_v4(rem[32 + d] + (uint32_t)((col0 + 4 * v4) * 4), xv.x, xv.y, xv.z, xv.w,
                    rem[48 + d]);
      }
    }
    if (!*vab) {
      // the last step's all-gather: wait for it, then write x back
      if (!warp_wait(bar_x, (uint32_t)((a.nouter - 1) & 1), lane, vab)) atomicOr(&s_abort, 1);
    }
  }
  __syncthreads();
  const bool aborted = s_abort != 0;
  if (aborted) {
    if (tid == 0) {
      atomicOr(a.flag, FLAG_TIMEOUT);
      // drain this CTA's copies: each ring's last fills (bounded waits)
      auto drain = [&](uint32_t full0, int nsl, int fills) {
        for (int k = max(0, fills - nsl); k < fills; ++k)
          mbar_wait_bounded(full0 + 8 * (k % nsl), (uint32_t)((k / nsl) & 1), kWaitBudget);
      };
      drain(fullM, L_NM, s_fills[0]);
      drain(fullU, L_NU, s_fills[1]);
      drain(fullG, L_NG, s_fills[2]);
    }
  } else {
    for (int64_t c = col0 + tid; c < min(col0 + nc, n); c += kThreads) a.x[c] = xf[c];
  }
  cluster.sync();
  if (aborted && tid == 0) {
    // exchange stores may still be in flight towards this CTA (see k_chain)
    const long long t0 = clock64();
    while (clock64() - t0 < 40000) {
    }
  }
}

template <typename TY, int MODE>
int launch_sm(const StreamArgs &a, const SLayout &L, int C, cudaStream_t st) {
  auto kern = k_chain_stream<TY, MODE>;
  GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)L.total));
  if (C > 8)
    GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = L.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  GLM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  return GLM_OK;
}

template <typename TY>
int launch_sy(const StreamArgs &a, const SLayout &L, int C, int mode, cudaStream_t st) {
  if (mode == 1) return launch_sm<TY, 1>(a, L, C, st);
  if (mode == 2) return launch_sm<TY, 2>(a, L, C, st);
  return launch_sm<TY, 0>(a, L, C, st);
}

SLayout layout_of(const ChainArgs &a) {
  const int tr = a.rec64 == 1 ? 8 : 4;
  return stream_layout(a.n, a.b, a.s, a.cluster, elem_bytes(a.dt), tr, a.ldy);
}

}  // namespace

bool chain_stream_ok(const ChainArgs &a) {
  if (a.cluster < 1 || a.cluster > 16) return false;
  const SLayout L = layout_of(a);
  return L.slot > 0 && L.rpb <= 32 && L.nc <= 256 && L.TM >= 1 && L.TU >= 1 &&
         (a.s < 2 || L.PC >= 4) && L.total <= kSmemMax && a.s <= 256 &&
         L.NM <= kMaxRing && L.NU <= kMaxRing && L.NG <= kMaxRing;
}

int launch_chain_stream(const ChainArgs &a, cudaStream_t st) {
  if (a.nouter <= 0) return GLM_OK;
  if (!chain_stream_ok(a))
    return set_error(GLM_EUNSUPPORTED, "streaming chain: shape outside its layout limits");
  const SLayout L = layout_of(a);
  StreamArgs sa;
  memset(&sa, 0, sizeof(sa));
  const int eb = elem_bytes(a.dt);
  const uint64_t rows = (uint64_t)a.nouter * a.s * a.b;
  GLM_TRY(make_tmap_2d(&sa.mmap, a.Y, a.dt, (uint64_t)a.ldy, rows, (uint64_t)a.ldy * eb,
                       (uint32_t)L.mbw, (uint32_t)L.TM));
  GLM_TRY(make_tmap_2d(&sa.umap, a.Y, a.dt, (uint64_t)a.ldy, rows, (uint64_t)a.ldy * eb,
                       (uint32_t)L.nc, (uint32_t)L.TU));
  sa.ylab = a.ylab;
  sa.G = a.G;
  sa.x = a.x;
  sa.flag = a.flag;
  sa.n = a.n;
  sa.b = a.b;
  sa.ldy = a.ldy;
  sa.sbp = a.sbp;
  sa.s = a.s;
  sa.s_last = a.s_last;
  sa.nouter = a.nouter;
  sa.loss = a.loss;
  sa.kahan = a.kahan;
  sa.alpha = a.alpha;
  sa.probe = a.probe;
  for (int j = 0; j <= a.s; ++j) {
    sa.cpow[j] = a.cpow[j];
    sa.cinv[j] = a.cinv[j];
  }
  // G pieces by TMA: every block row's width (j b) and the piece width PC
  // are multiples of the box's inner width (at most 256 columns)
  int gi = 256;
  while (gi >= 8 && (a.b % gi != 0 || L.PC % gi != 0)) gi /= 2;
  if (a.s >= 2 && a.s - 1 <= kMaxGmap && gi >= 8 && L.PC / gi <= 256 && L.rpb <= 256) {
    const int64_t gsz = gram_size(a.s, a.b);
    for (int j = 1; j < a.s; ++j) {
      const int64_t ldj = gram_ld(j, a.b);
      const uint64_t dims[4] = {(uint64_t)gi, (uint64_t)(ldj / gi), (uint64_t)a.b,
                                (uint64_t)a.nouter};
      const uint64_t strides[3] = {(uint64_t)gi * 4, (uint64_t)ldj * 4, (uint64_t)gsz * 4};
      const uint32_t box[4] = {(uint32_t)gi, (uint32_t)(L.PC / gi), (uint32_t)L.rpb, 1u};
      GLM_TRY(make_tmap_4d_f32(&sa.gmap[j - 1], a.G + gram_off(j, a.b), dims, strides, box));
    }
    sa.gtma = 1;
    sa.ginner = gi;
    // measured: prefetching pays where a step's G streams from HBM (the
    // large least-squares shape, 528 MB) and costs a little where it stays
    // in L2 (the wide shape at s = 32, 32 MB)
    sa.gpf = gsz * 4 > (64ll << 20);
  }
  switch (a.dt) {
  case GLM_F32: case GLM_TF32: return launch_sy<float>(sa, L, a.cluster, a.rec64, st);
  case GLM_BF16: return launch_sy<__nv_bfloat16>(sa, L, a.cluster, a.rec64, st);
  case GLM_F16: return launch_sy<__half>(sa, L, a.cluster, a.rec64, st);
  }
  return set_error(GLM_EINVAL, "streaming chain: unsupported GEMV operand type");
}

}  // namespace glm
