// k_batch.cu -- kernels of batched fits: many independent problems of uneven
// m, n and lambda (paper Algorithm 1 applied to each).
//
//  * k_gather_batch: one launch per round for every problem; grid.y is the
//    problem, one warp per gathered row (Philox draw, dequantised storage
//    row, rounded to the operand type, zero-padded to ldy).  The unused rows
//    of a short last outer step are written as zeros so that every outer step
//    of the round holds exactly s b rows (the Gram launches stack them).
//  * k_chain_batch: the x-dependent part (margins r = Y x, the s-step
//    recurrence, the outer update) of every problem of the round, in one
//    persistent launch: each CTA takes the next problem from a device work
//    queue (ordered longest first by the host), keeps its iterate in shared
//    memory for the round's outer steps, writes it back and takes the next.
//    One CTA holds the whole recurrence of a problem, so an inner step is a
//    CTA barrier, not an exchange between CTAs.
#include "glm_internal.cuh"

namespace glm {
namespace {

constexpr int kGWarps = 8;     // gather: rows per block
constexpr int kBT = 512;       // chain: threads per CTA
constexpr int kBW = kBT / 32;

template <typename TS>
__global__ void __launch_bounds__(kGWarps * 32)
k_gather_batch(const BatchItem *__restrict__ items) {
  const BatchItem &it = items[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t sb = (int64_t)it.s * it.b;
  const int64_t total = (int64_t)it.nouter * sb;
  const int64_t real = total - (int64_t)(it.s - it.s_last) * it.b;  // rows with a draw
  const int eb = elem_bytes(it.y_dt);
  const TS *A = static_cast<const TS *>(it.A);
  for (int64_t row = (int64_t)blockIdx.x * kGWarps + (threadIdx.x >> 5); row < total;
       row += (int64_t)gridDim.x * kGWarps) {
    char *dst = static_cast<char *>(it.Y) + row * it.ldy * eb;
    if (row >= real) {  // padding rows of a short last outer step
      for (int64_t c = (int64_t)lane * 8; c < it.ldy; c += 256) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        store8(dst + c * eb, it.y_dt, v);
      }
      if (lane == 0) it.lab[row] = 0.f;
      continue;
    }
    int32_t idx = 0;
    if (lane == 0) idx = draw_row(it.seed, it.problem, it.q0 + (uint64_t)row, (uint64_t)it.m);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (!in_bounds(idx >= 0 && idx < it.m, lane == 0 ? it.flag : nullptr)) continue;
    const TS *src = A + (int64_t)idx * it.lda;
    for (int64_t c = (int64_t)lane * 8; c < it.ldy; c += 256) {
      float v[8];
      if (c < it.n) {
        Vec8<TS>::load(src + c, v);
        if (it.colscale) {
          const float4 s0 = __ldg(reinterpret_cast<const float4 *>(it.colscale + c));
          const float4 s1 = __ldg(reinterpret_cast<const float4 *>(it.colscale + c) + 1);
          v[0] *= s0.x; v[1] *= s0.y; v[2] *= s0.z; v[3] *= s0.w;
          v[4] *= s1.x; v[5] *= s1.y; v[6] *= s1.z; v[7] *= s1.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
      }
      store8(dst + c * eb, it.y_dt, v);
    }
    if (lane == 0) it.lab[row] = __ldg(it.y + idx);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

struct ChainSmem {  // byte offsets of the per-CTA buffers
  size_t xs, rr, uh, coef, goff, part, total;
};
__host__ __device__ inline ChainSmem chain_smem(int max_n, int max_sb, int max_s, int tr) {
  ChainSmem L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 15) / 16 * 16;
    const size_t o = off;
    off += bytes;
    return o;
  };
  L.xs = take((size_t)round_up(max_n, 8) * 4);
  L.rr = take((size_t)max_sb * tr);
  L.uh = take((size_t)max_sb * tr);
  L.coef = take((size_t)3 * (max_s + 1) * tr);
  L.goff = take((size_t)(max_s + 1) * 8);
  L.part = take((size_t)kBT * 8 * 4);
  L.total = off;
  return L;
}

template <typename TY, typename TR>
__global__ void __launch_bounds__(kBT)
k_chain_batch(const BatchItem *__restrict__ items, const int *__restrict__ order, int nitems,
              int *queue, int max_n, int max_sb, int max_s) {
  extern __shared__ __align__(16) unsigned char sm[];
  const ChainSmem L = chain_smem(max_n, max_sb, max_s, (int)sizeof(TR));
  float *xs = reinterpret_cast<float *>(sm + L.xs);
  TR *rr = reinterpret_cast<TR *>(sm + L.rr);   // margins of the outer step's rows
  TR *uh = reinterpret_cast<TR *>(sm + L.uh);   // c^{-j} u_j
  TR *cpw = reinterpret_cast<TR *>(sm + L.coef);  // c^j
  TR *cinw = cpw + (max_s + 1);                    // c^-j
  TR *zcw = cinw + (max_s + 1);                    // alpha c^(j-1), j >= 1
  int64_t *goff = reinterpret_cast<int64_t *>(sm + L.goff);
  float *part = reinterpret_cast<float *>(sm + L.part);
  __shared__ int s_item;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int qi = s_item;
    __syncthreads();  // every thread has read s_item before it is overwritten
    if (qi >= nitems) break;
    const BatchItem &it = items[order[qi]];
    const int n = it.n, b = it.b, s = it.s, nouter = it.nouter, s_last = it.s_last;
    const int sb = s * b;
    const int64_t ldy = it.ldy, gsz = gram_size(s, b);
    const TY *Y = static_cast<const TY *>(it.Y);
    const float *lab = it.lab;
    const float *G = it.G;
    float *xg = it.x;
    unsigned *flag = it.flag;
    const int loss = it.loss, kahan = it.kahan;

    for (int i = tid; i < round_up(max_n, 8); i += kBT) xs[i] = i < n ? xg[i] : 0.f;
    if (tid == 0) {
      // c^j by repeated multiplication in FP64, the same sequence the host
      // forms for the cluster chain; alpha c^(j-1) from the previous power
      double cp = 1.0, prev = 0.0;
      for (int j = 0; j <= s; ++j) {
        cpw[j] = (TR)cp;
        cinw[j] = (TR)(1.0 / cp);
        zcw[j] = j > 0 ? (TR)((double)it.alpha * prev) : (TR)0;
        goff[j] = gram_off(j, b);
        prev = cp;
        cp *= it.c;
      }
    }
    __syncthreads();

    for (int h = 0; h < nouter; ++h) {
      const int sh = (h == nouter - 1) ? s_last : s;
      const int R = sh * b;
      const TY *Yh = Y + (int64_t)h * sb * ldy;
      const float *lh = lab + (int64_t)h * sb;
      const float *Gh = G + (int64_t)h * gsz;
      // the next outer step's rows and Gram blocks (contiguous in the round
      // buffers) stream into L2 while this step runs: the round buffers are
      // larger than L2, so without it every step would wait on DRAM
      if (tid == 0 && h + 1 < nouter) {
        prefetch_l2(Yh + (int64_t)sb * ldy, (uint32_t)((int64_t)sb * ldy * sizeof(TY)));
        if (s >= 2) prefetch_l2(Gh + gsz, (uint32_t)(gsz * 4));
      }

      // ---- margins r = Y_h x (warp per row, four rows' loads in flight) ----
      for (int r0 = warp; r0 < R; r0 += 4 * kBW) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = lane * 8; c0 < n; c0 += 256) {
          float v[4][8];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = r0 + q * kBW;
            if (r < R) {
              Vec8<TY>::load(Yh + (int64_t)r * ldy + c0, v[q]);
            } else {
#pragma unroll
              for (int k = 0; k < 8; ++k) v[q][k] = 0.f;
            }
          }
          const float4 x0 = *reinterpret_cast<const float4 *>(xs + c0);
          const float4 x1 = *reinterpret_cast<const float4 *>(xs + c0 + 4);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float a = acc[q];
            a = fmaf(v[q][0], x0.x, a); a = fmaf(v[q][1], x0.y, a);
            a = fmaf(v[q][2], x0.z, a); a = fmaf(v[q][3], x0.w, a);
            a = fmaf(v[q][4], x1.x, a); a = fmaf(v[q][5], x1.y, a);
            a = fmaf(v[q][6], x1.z, a); a = fmaf(v[q][7], x1.w, a);
            acc[q] = a;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float t = warp_sum(acc[q]);
          if (lane == 0 && r0 + q * kBW < R) rr[r0 + q * kBW] = (TR)t;
        }
      }
      __syncthreads();

      // ---- s-step recurrence: z_j = c^j r_j - alpha c^{j-1} G_{j,<j} (c^{-i} u_i) ----
      for (int j = 0; j < sh; ++j) {
        const int jb = j * b;
        const int64_t ldj = gram_ld(j, b);
        for (int l = warp; l < b; l += kBW) {
          TR corr = 0;
          if (j > 0) {
            const float *grow = Gh + goff[j] + (int64_t)l * ldj;
            TR a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            int cc = lane;
            for (; cc + 96 < jb; cc += 128) {
              a0 += (TR)__ldg(grow + cc) * uh[cc];
              a1 += (TR)__ldg(grow + cc + 32) * uh[cc + 32];
              a2 += (TR)__ldg(grow + cc + 64) * uh[cc + 64];
              a3 += (TR)__ldg(grow + cc + 96) * uh[cc + 96];
            }
            for (; cc < jb; cc += 32) a0 += (TR)__ldg(grow + cc) * uh[cc];
            corr = warp_sum((a0 + a1) + (a2 + a3));
          }
          if (lane == 0) {
            const TR z = cpw[j] * rr[jb + l] - zcw[j] * corr;
            const TR u = dloss<TR>(loss, z, (TR)lh[jb + l]);
            if (!isfinite(z) || !isfinite(u)) atomicOr(flag, FLAG_NONFINITE);
            uh[jb + l] = u * cinw[j];
          }
        }
        __syncthreads();
      }

      // ---- update x <- c^{sh} x - alpha c^{sh-1} Y^T (c^{-j} u) ----
      const int n8 = (n + 7) / 8;
      const int wide = n8 >= kBT;           // one thread per 8-column group
      const int RG = wide ? 1 : kBT / n8;   // row groups
      const int W = (wide ? kBT : n8) * 8;  // columns per pass
      const float decay = (float)cpw[sh];
      const float stp = (float)zcw[sh];
      for (int cg0 = 0; cg0 < n8; cg0 += W / 8) {
        const int g = wide ? 0 : tid / n8;
        const int cg = cg0 + (wide ? tid : tid % n8);
        if (g < RG && cg < n8) {
          float ae[8], cm[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) { ae[k] = 0.f; cm[k] = 0.f; }
          for (int r0 = g; r0 < R; r0 += 4 * RG) {
            // four rows' loads in flight, then the sums in row order
            float v[4][8];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (r0 + q * RG < R) Vec8<TY>::load(Yh + (int64_t)(r0 + q * RG) * ldy + cg * 8, v[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int r = r0 + q * RG;
              if (r >= R) break;
              const float w = (float)uh[r];
              if (kahan) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                  const float yv = fmaf(v[q][k], w, -cm[k]);
                  const float t2 = ae[k] + yv;
                  cm[k] = (t2 - ae[k]) - yv;
                  ae[k] = t2;
                }
              } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) ae[k] = fmaf(v[q][k], w, ae[k]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) part[g * W + (cg - cg0) * 8 + k] = ae[k];
        }
        __syncthreads();
        for (int cc = tid; cc < W; cc += kBT) {
          const int c = cg0 * 8 + cc;
          if (c >= n) continue;
          float S = 0.f, cS = 0.f;
          for (int gg = 0; gg < RG; ++gg) {
            const float yv = part[gg * W + cc] - cS;
            const float t2 = S + yv;
            cS = (t2 - S) - yv;
            S = t2;
          }
          const float xn = fmaf(-stp, S - cS, decay * xs[c]);
          if (!isfinite(xn)) atomicOr(flag, FLAG_NONFINITE);
          xs[c] = xn;
        }
        __syncthreads();
      }
    }
    for (int i = tid; i < n; i += kBT) xg[i] = xs[i];
    __syncthreads();
  }
}

}  // namespace

int launch_gather_batch(const BatchItem *items, int nitems, int64_t max_rows, cudaStream_t st,
                        int a_dt) {
  if (nitems <= 0 || max_rows <= 0) return GLM_OK;
  const int64_t bx = (max_rows + kGWarps - 1) / kGWarps;
  dim3 grid((unsigned)(bx < 4096 ? bx : 4096), (unsigned)nitems);
  switch (a_dt) {
  case GLM_F32: k_gather_batch<float><<<grid, kGWarps * 32, 0, st>>>(items); break;
  case GLM_BF16: k_gather_batch<__nv_bfloat16><<<grid, kGWarps * 32, 0, st>>>(items); break;
  case GLM_F16: k_gather_batch<__half><<<grid, kGWarps * 32, 0, st>>>(items); break;
  default: return set_error(GLM_EINVAL, "batched gather: bad storage type");
  }
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

template <typename TY, typename TR>
int chain_batch_t(const BatchItem *items, const int *order, int nitems, int *queue, int max_n,
                  int max_sb, int max_s, cudaStream_t st) {
  const ChainSmem L = chain_smem(max_n, max_sb, max_s, (int)sizeof(TR));
  auto kern = k_chain_batch<TY, TR>;
  if (L.total > 227 * 1024)
    return set_error(GLM_EUNSUPPORTED, "batched chain: n or s*b too large for shared memory");
  GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)L.total));
  int per_sm = 0;
  GLM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBT, L.total));
  if (per_sm < 1) return set_error(GLM_EUNSUPPORTED, "batched chain does not fit an SM");
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = nitems < sms * per_sm ? nitems : sms * per_sm;
  kern<<<grid, kBT, L.total, st>>>(items, order, nitems, queue, max_n, max_sb, max_s);
  GLM_CUDA_TRY(cudaGetLastError());
  return GLM_OK;
}

int launch_chain_batch(const BatchItem *items, const int *order, int nitems, int *queue,
                       int y_dt, int rec64, int max_n, int max_sb, int max_s, cudaStream_t st) {
  if (nitems <= 0) return GLM_OK;
  switch (y_dt) {
  case GLM_F32: case GLM_TF32:
    return rec64 ? chain_batch_t<float, double>(items, order, nitems, queue, max_n, max_sb, max_s, st)
                 : chain_batch_t<float, float>(items, order, nitems, queue, max_n, max_sb, max_s, st);
  case GLM_BF16:
    return rec64 ? chain_batch_t<__nv_bfloat16, double>(items, order, nitems, queue, max_n, max_sb,
                                                        max_s, st)
                 : chain_batch_t<__nv_bfloat16, float>(items, order, nitems, queue, max_n, max_sb,
                                                       max_s, st);
  case GLM_F16:
    return rec64 ? chain_batch_t<__half, double>(items, order, nitems, queue, max_n, max_sb, max_s, st)
                 : chain_batch_t<__half, float>(items, order, nitems, queue, max_n, max_sb, max_s, st);
  }
  return set_error(GLM_EINVAL, "batched chain: unsupported operand type");
}

}  // namespace glm
