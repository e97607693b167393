// k_gram_tc.cu -- strictly block-lower Gram G_{j,i} = Y_j Y_i^T (i < j) on
// the 5th-generation tensor cores (paper Algorithm 1, Gram step; Sec. 5.2's
// G_L is the only part the recurrence reads).
//
// One persistent CTA per SM walks a static list of 128 x N output tiles
// (N = 256, or 128 when the wide tiles would leave SMs idle) of the lower
// triangle of every outer iteration's (s b) x (s b) Gram; tiles holding no
// strictly-lower block entry are skipped.  A 128 x 256 tile reads 1.5 times
// fewer operand bytes per flop than a 128 x 128 one, which is what keeps the
// SMs' operand stream from L2 below the tensor cores' rate.  Warp roles:
//   warp 0      TMA producer: the tile's 128 A rows and N B rows of Y
//               (K-major, 128-byte swizzle) per 128-byte K chunk into a
//               STAGES-deep ring;
//   warp 1      allocates 2N TMEM columns (two N-column FP32 accumulators)
//               and one elected lane issues tcgen05.mma (M=128, N), four
//               MMAs per K chunk, committing each stage back to the producer
//               and each finished accumulator to the epilogue;
//   warps 2..5  epilogue: tcgen05.ld 32x32b rows out of TMEM, per-row scales
//               (E4M3), masked FP32 stores into the padded row-block layout.
// Operand kinds: BF16 / F16 (kind::f16), TF32 (kind::tf32, FP32 container
// already rounded to TF32), E4M3 (kind::f8f6f4, one power-of-two scale per row
// applied at readout).  Accumulation is FP32, except for the FP16-accumulate
// instance (Recipe F's Gram slot: F16 operands, F16 accumulator in TMEM --
// one value in the low half of each 32-bit column -- widened at readout).  Every mbarrier wait
// is bounded; on timeout the kernel records FLAG_TIMEOUT, drains its own
// work (bounded) and frees its TMEM.
#include "glm_internal.cuh"

namespace glm {
namespace {

constexpr int kStages = 4;
constexpr int kTile = 128;                 // M (rows of a tile)
constexpr int kChunkBytes = 128;           // K bytes per stage row (one SW128 atom)
constexpr int kOperandBytes = kTile * kChunkBytes;  // 16 KB per 128 rows per stage
constexpr int kThreads = 192;
constexpr long long kBudget = 4000000000ll;

template <int kN> struct TileCfg {
  static constexpr int kBBytes = kN * kChunkBytes;             // B rows per stage
  static constexpr int kStageBytes = kOperandBytes + kBBytes;  // A + B
  static constexpr uint32_t kTmemCols = 2 * kN;                // two accumulators
  static constexpr size_t kSmem = 1024 + (size_t)kStages * kStageBytes + 8 * (2 * kStages + 6) + 32;
};

struct TcArgs {
  CUtensorMap ymap;       // 2D (ld, rows) map, box (128 bytes of K, 128 rows), SW128
  const float *rs;        // per-row scales (E4M3) or null
  float *G;
  unsigned *flag;
  long long probe;        // > 0: failure-path probe wait before the first MMA
  int64_t nouter, rows, b, n, ld;
  int s, dt, nk;          // nk: K chunks
  int ksplit, kper;       // K split into ksplit ranges of kper chunks (1: none)
};

// ---- PTX wrappers (tcgen05 / TMEM) -------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(dst_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
               ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

template <int DT> __device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc,
                                                         uint64_t bdesc, uint32_t idesc,
                                                         uint32_t accum) {
  if (DT == GLM_TF32) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  } else if (DT == GLM_E4M3) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  } else {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  }
}

// 32-byte global store of eight floats (the address must be 32-byte aligned).
__device__ __forceinline__ void st_global_v8(float *p, float a, float b, float c, float d,
                                             float e, float f, float g, float h) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
               ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d), "f"(e), "f"(f), "f"(g), "f"(h)
               : "memory");
}

// Asynchronous form: starts the load of 32 columns into r; r is valid only
// after tmem_ld_wait(r) (which takes r as an operand, so that no use of r
// can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld32_start(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31])
               :: "memory");
}

// Bounded wait that also gives up once another role of the CTA has aborted
// (the abort flag is read on every 64th probe).
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity,
                                              const volatile int *abort_flag) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (unsigned k = 1;; ++k) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((k & 63) == 0 && (*abort_flag || clock64() - t0 > kBudget)) return false;
  }
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart (SBO), version 1 (sm_100+).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)1 << 16;                          // LBO (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                // SBO
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // layout: SWIZZLE_128B
  return d;
}

// Instruction descriptor: D FP32 (or F16), A/B K-major, M = 128, N = kN.
template <int DT, int kN, bool kAcc16 = false>
__host__ __device__ constexpr uint32_t instr_desc() {
  // operand format field: kind::f16 -> F16 0 / BF16 1; kind::tf32 -> 2;
  // kind::f8f6f4 -> E4M3 0; accumulator format: F16 0, F32 1
  return ((kAcc16 ? 0u : 1u) << 4)                                     // D format
         | ((uint32_t)(DT == GLM_BF16 ? 1 : DT == GLM_TF32 ? 2 : 0) << 7)  // A format
         | ((uint32_t)(DT == GLM_BF16 ? 1 : DT == GLM_TF32 ? 2 : 0) << 10) // B format
         | ((uint32_t)(kN >> 3) << 17)                                  // N >> 3
         | ((uint32_t)(kTile >> 4) << 24);                              // M >> 4
}

// Lower-triangular tiles of one outer iteration: row tiles tj of 128 rows,
// column panels ti of kN rows of Y with ti * kN <= tj * 128 + 127.  With
// q = kN / 128 row tiles per panel, row tile tj has tj / q + 1 panels, so the
// q row tiles of group k = tj / q hold q (k + 1) tiles and the groups before
// group k hold q k (k + 1) / 2.
template <int kN> __host__ __device__ inline int64_t tiles_per_outer(int64_t sb) {
  constexpr int64_t q = kN / kTile;
  const int64_t T = (sb + kTile - 1) / kTile;   // row tiles
  int64_t P = 0;
  for (int64_t k = 0; k * q < T; ++k) P += min(q, T - k * q) * (k + 1);
  return P;
}

// Output tile t of the flattened (outer step, lower-triangular tile) list;
// returns false when the tile holds no strictly-lower block entry.
struct Tile {
  int64_t g, tj, ti, rows_g;
};
template <int kN>
__device__ __forceinline__ bool tile_at(const TcArgs &a, int64_t P, int64_t t, Tile &o) {
  constexpr int64_t q = kN / kTile;
  const int64_t sb = (int64_t)a.s * a.b;
  o.g = t / P;
  const int64_t p = t - o.g * P;
  // group k: the largest k with q k (k + 1) / 2 <= p
  int64_t k = (int64_t)((sqrt(8.0 * (double)p / (double)q + 1.0) - 1.0) * 0.5);
  while (k > 0 && q * k * (k + 1) / 2 > p) --k;
  while (q * (k + 1) * (k + 2) / 2 <= p) ++k;
  const int64_t rem = p - q * k * (k + 1) / 2;   // < q (k + 1)
  o.tj = k * q + rem / (k + 1);
  o.ti = rem % (k + 1);
  o.rows_g = min(sb, a.rows - o.g * sb);
  const int64_t r0 = o.tj * kTile, c0 = o.ti * kN;
  const int64_t r_last = min(r0 + kTile, o.rows_g) - 1;
  return r_last >= r0 && r_last / a.b > c0 / a.b;
}

template <int DT, int kN, bool kAcc16 = false>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const __grid_constant__ TcArgs a) {
  using Cfg = TileCfg<kN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t sbase0 = smem_u32(smem_raw);
  unsigned char *smem = smem_raw + (round_up(sbase0, 1024) - sbase0);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t stage_a = sbase;                                  // + st * kStageBytes
  const uint32_t bars = sbase + kStages * Cfg::kStageBytes;        // 8-byte barriers
  const uint32_t full0 = bars, empty0 = bars + 8 * kStages;
  const uint32_t tfull0 = bars + 16 * kStages, tempty0 = tfull0 + 16;
  const uint32_t drain = tempty0 + 16;        // MMA unwind barrier
  const uint32_t probe_bar = drain + 8;       // never signalled (failure-path probe)
  const uint32_t tmem_slot = drain + 16;      // 16-byte aligned TMEM address slot
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull0 + 8 * i, 1);
      mbar_init(tempty0 + 8 * i, 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    mbar_init(probe_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *reinterpret_cast<volatile uint32_t *>(smem + (tmem_slot - sbase));

  const int64_t sb = (int64_t)a.s * a.b;
  const int64_t P = tiles_per_outer<kN>(sb);
  const int64_t ntiles = a.nouter * P * a.ksplit;  // work units: (tile, K range)
  volatile int *vabort = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t t = blockIdx.x; t < ntiles && !*vabort; t += gridDim.x) {
        Tile tl;
        if (!tile_at<kN>(a, P, t / a.ksplit, tl)) continue;
        const int kb = (int)(t % a.ksplit) * a.kper, ke = min(a.nk, kb + a.kper);
        const int32_t ya = (int32_t)(tl.g * sb + tl.tj * kTile);
        const int32_t yb = (int32_t)(tl.g * sb + tl.ti * kN);
        for (int kc = kb; kc < ke; ++kc, ++it) {
          const int st = (int)(it % kStages);
          if (it >= kStages &&
              !wait_or_abort(empty0 + 8 * st, (uint32_t)((it / kStages - 1) & 1), vabort)) {
            atomicOr(&s_abort, 1);
            break;
          }
          const uint32_t full = full0 + 8 * st;
          mbar_arrive_expect_tx(full, Cfg::kStageBytes);
          const int32_t xk = kc * (kChunkBytes / elem_bytes(DT));
          const uint32_t dA = stage_a + st * Cfg::kStageBytes;
          tma_load_2d(dA, &a.ymap, xk, ya, full);
#pragma unroll
          for (int h = 0; h < kN / kTile; ++h)  // B: kN rows in boxes of 128
            tma_load_2d(dA + kOperandBytes + h * kOperandBytes, &a.ymap, xk, yb + h * kTile,
                        full);
        }
      }
      // unwind: wait (bounded) for the loads still in flight
      if (*vabort)
        for (int64_t i = (it > kStages ? it - kStages : 0); i < it; ++i)
          mbar_wait_bounded(full0 + 8 * (i % kStages), (uint32_t)((i / kStages) & 1), kBudget);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<DT, kN, kAcc16>();
      int64_t it = 0, tc = 0;
      // failure-path probe: a wait on a barrier nothing signals gives up
      if (a.probe > 0 && !mbar_wait_bounded(probe_bar, 0, a.probe)) atomicOr(&s_abort, 1);
      for (int64_t t = blockIdx.x; t < ntiles && !*vabort; t += gridDim.x) {
        Tile tl;
        if (!tile_at<kN>(a, P, t / a.ksplit, tl)) continue;
        const int kb = (int)(t % a.ksplit) * a.kper, ke = min(a.nk, kb + a.kper);
        const int buf = (int)(tc & 1);
        if (tc >= 2 &&
            !wait_or_abort(tempty0 + 8 * buf, (uint32_t)((tc / 2 - 1) & 1), vabort)) {
          atomicOr(&s_abort, 1);
          break;
        }
        tc_fence_after();
        const uint32_t tmem_d = tmem_base + (uint32_t)(buf * kN);
        bool ok = true;
        for (int kc = kb; kc < ke; ++kc, ++it) {
          const int st = (int)(it % kStages);
          if (!wait_or_abort(full0 + 8 * st, (uint32_t)((it / kStages) & 1), vabort)) {
            atomicOr(&s_abort, 1);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = stage_a + st * Cfg::kStageBytes;
          const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + kOperandBytes);
#pragma unroll
          for (int k = 0; k < kChunkBytes / 32; ++k)  // 32 bytes of K per MMA
            tc_mma<DT>(tmem_d, da + 2 * k, db + 2 * k, idesc, (kc != kb) || k != 0);
          tc_commit(empty0 + 8 * st);  // stage free once these MMAs have read it
        }
        if (!ok) break;
        tc_commit(tfull0 + 8 * buf);   // accumulator ready for the epilogue
        ++tc;
      }
      // unwind: make sure no MMA issued here is still running before TMEM is freed
      if (*vabort) {
        tc_commit(drain);
        mbar_wait_bounded(drain, 0, kBudget);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int quad = warp & 3;  // TMEM lanes 32*quad .. 32*quad+31
    int64_t tc = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      Tile tl;
      if (!tile_at<kN>(a, P, t / a.ksplit, tl)) continue;
      const int buf = (int)(tc & 1);
      if (!wait_or_abort(tfull0 + 8 * buf, (uint32_t)((tc / 2) & 1), vabort)) {
        atomicOr(&s_abort, 1);
        break;
      }
      tc_fence_after();
      const int64_t rho = tl.tj * kTile + quad * 32 + lane;  // this thread's row
      const int64_t j = rho / a.b, l = rho - j * a.b;
      const bool row_ok = rho < tl.rows_g;
      const int64_t limit = j * a.b;                           // columns < j b
      float *grow = a.G + tl.g * gram_size(a.s, a.b) + gram_off(j, a.b) + l * gram_ld(j, a.b);
      const float srow = (DT == GLM_E4M3 && row_ok) ? a.rs[tl.g * sb + rho] : 1.f;
      // chunk cc's 32 columns of this lane's row: scale and store
      auto store_chunk = [&](uint32_t (&r)[32], int cc) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
        if (kAcc16) {  // F16 accumulator: the low 16 bits of each column
#pragma unroll
          for (int i = 0; i < 32; ++i)
            v[i] = __half2float(__ushort_as_half((unsigned short)(__float_as_uint(v[i]) & 0xFFFFu)));
        }
        const int64_t c0 = tl.ti * kN + cc * 32;
        if (!row_ok || c0 >= limit) return;
        if (!in_bounds(tl.g < a.nouter && grow + min(c0 + 32, limit) <=
                           a.G + a.nouter * gram_size(a.s, a.b),
                       a.flag))
          return;
        if (DT == GLM_E4M3) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            v[i] *= srow * ((c0 + i < limit) ? __ldg(a.rs + tl.g * sb + c0 + i) : 0.f);
        }
        if (a.ksplit > 1) {  // partial sums over one K range: added into zeroed G
          // (16-byte vector atomics: rows start on 16-byte boundaries, c0 % 32 == 0)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (c0 + 4 * q + 4 <= limit) {
              atomicAdd(reinterpret_cast<float4 *>(grow + c0 + 4 * q),
                        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (c0 + 4 * q + i < limit) atomicAdd(grow + c0 + 4 * q + i, v[4 * q + i]);
            }
          }
        } else if (c0 + 32 <= limit && (reinterpret_cast<uintptr_t>(grow + c0) & 31) == 0) {
          // 32-byte stores: each lane writes its own row, so a store instruction
          // touches 32 rows; wider stores halve the instructions the SM's
          // store path has to split (the epilogue bounds the K = 1,024 tiles)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            st_global_v8(grow + c0 + 8 * q, v[8 * q], v[8 * q + 1], v[8 * q + 2], v[8 * q + 3],
                         v[8 * q + 4], v[8 * q + 5], v[8 * q + 6], v[8 * q + 7]);
        } else if (c0 + 32 <= limit) {
          float4 *d = reinterpret_cast<float4 *>(grow + c0);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (c0 + i < limit) grow[c0 + i] = v[i];
        }
      };
      // the next chunk's TMEM load is in flight while this chunk is stored
      auto taddr = [&](int cc) {
        return tmem_base + (uint32_t)(buf * kN + cc * 32) + ((uint32_t)(quad * 32) << 16);
      };
      uint32_t ra[32], rb[32];
      tmem_ld32_start(taddr(0), ra);
      tmem_ld_wait(ra);
#pragma unroll 1
      for (int cc = 0; cc < kN / 32; cc += 2) {  // kN / 32 is even
        tmem_ld32_start(taddr(cc + 1), rb);
        store_chunk(ra, cc);
        __syncwarp();  // the TMEM loads and waits are warp-wide (.sync.aligned)
        tmem_ld_wait(rb);
        if (cc + 2 < kN / 32) tmem_ld32_start(taddr(cc + 2), ra);
        store_chunk(rb, cc + 1);
        __syncwarp();
        if (cc + 2 < kN / 32) tmem_ld_wait(ra);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
      ++tc;
    }
  }
  __syncthreads();
  if (s_abort && threadIdx.x == 0 && a.flag) atomicOr(a.flag, FLAG_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::kTmemCols);
  }
}

template <int kN>
int launch_n(const TcArgs &a, int sms, int64_t ntiles, cudaStream_t st, bool acc16) {
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  const size_t smem = TileCfg<kN>::kSmem;
  void (*kern)(TcArgs);
  switch (a.dt) {
  case GLM_BF16: kern = k_gram_tc<GLM_BF16, kN>; break;
  case GLM_F16: kern = acc16 ? k_gram_tc<GLM_F16, kN, true> : k_gram_tc<GLM_F16, kN>; break;
  case GLM_TF32: kern = k_gram_tc<GLM_TF32, kN>; break;
  default: kern = k_gram_tc<GLM_E4M3, kN>; break;
  }
  GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, kThreads, smem, st>>>(a);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

}  // namespace

bool gram_tc_supported(int dt, int64_t ld) {
  if (dt == GLM_E4M3) return ld % 128 == 0;
  if (dt == GLM_BF16 || dt == GLM_F16 || dt == GLM_TF32) return ld % 64 == 0;
  return false;
}

namespace {

int launch_gram_tc_impl(const GramArgs &g, cudaStream_t st, bool acc16) {
  if (g.s < 2 || g.nouter <= 0) return GLM_OK;
  if (acc16 && g.dt != GLM_F16)
    return set_error(GLM_EINVAL, "tcgen05 Gram with FP16 accumulation needs F16 operands");
  if (!gram_tc_supported(g.dt, g.ld))
    return set_error(GLM_EUNSUPPORTED, "tcgen05 Gram: unsupported operand type or ld");
  TcArgs a;
  memset(&a, 0, sizeof(a));
  const int eb = elem_bytes(g.dt);
  GLM_TRY(make_tmap_2d_sw128(&a.ymap, g.Y, g.dt, (uint64_t)g.ld,
                             (uint64_t)g.nouter * g.s * g.b, (uint64_t)g.ld * eb,
                             (uint32_t)(kChunkBytes / eb), (uint32_t)kTile));
  a.rs = g.rs;
  a.G = g.G;
  a.flag = g.flag;
  a.probe = g.probe;
  a.nouter = g.nouter;
  a.rows = g.rows;
  a.b = g.b;
  a.n = g.n;
  a.ld = g.ld;
  a.s = g.s;
  a.dt = g.dt;
  a.nk = (int)((g.n * eb + kChunkBytes - 1) / kChunkBytes);  // K chunks covering n
  const int64_t sb = (int64_t)g.s * g.b;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // wide tiles unless they would leave SMs idle (few, long-K tiles), or as
  // the caller asks (the batched autotuner times both)
  const int64_t wide = g.nouter * tiles_per_outer<256>(sb);
  a.ksplit = 1;
  a.kper = a.nk;
  // Few wide tiles over a long K (the paper's roofline shape: n = 16,384 over
  // a few thousand rows) leave most SMs idle: split K instead, ranges of at
  // least 16 chunks, each range's partial sums added into a zeroed G.  The
  // order of those additions varies from run to run; every entry keeps its
  // Higham bound.  Not for the FP16-accumulate Gram, whose single FP16 sum is
  // what Recipe F prescribes, nor when the caller fixes the tile.
  if (!acc16 && g.tile_n == 0 && wide < sms && a.nk >= 32) {
    int64_t ks = sms / (wide > 0 ? wide : 1);
    if (ks > a.nk / 16) ks = a.nk / 16;
    if (ks > 1) {
      a.kper = (int)((a.nk + ks - 1) / ks);
      a.ksplit = (a.nk + a.kper - 1) / a.kper;
      GLM_CUDA_TRY(cudaMemsetAsync(g.G, 0, (size_t)g.nouter * gram_size(g.s, g.b) * 4, st));
      return launch_n<256>(a, sms, wide * a.ksplit, st, acc16);
    }
  }
  if (g.tile_n == 256 || (g.tile_n == 0 && wide >= sms))
    return launch_n<256>(a, sms, wide, st, acc16);
  return launch_n<128>(a, sms, g.nouter * tiles_per_outer<128>(sb), st, acc16);
}

}  // namespace

int launch_gram_tc(const GramArgs &g, cudaStream_t st) { return launch_gram_tc_impl(g, st, false); }

int launch_gram_tc_f16acc(const GramArgs &g, cudaStream_t st) {
  return launch_gram_tc_impl(g, st, true);
}

}  // namespace glm
