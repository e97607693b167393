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
// All exchanges are one-way: values travel with st.async into the owner's
// shared memory and complete transaction bytes on the owner's mbarrier, so
// an inner step costs one DSMEM latency instead of a cluster barrier.  Every
// wait is bounded (FLAG_TIMEOUT, then the kernel unwinds without writing x).
// The own rows of G_{j,<j} stream into shared memory with cp.async one inner
// step ahead (double buffer) when they fit.
//
// The c^{-i} scaling of the stored residual history turns the per-block
// weights c^{j-1-i} of the ridge-decayed recurrence into one scalar per row
// (c = 1 - eta lambda > 0; the host rejects c^{-(s-1)} beyond 2^60).
#include <cooperative_groups.h>

#include "glm_internal.cuh"

namespace cg = cooperative_groups;

namespace glm {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr long long kWaitBudget = 4000000000ll;  // SM cycles (~2 s)
constexpr size_t kSmemMax = 227 * 1024;

struct Layout {
  int nc, rpb, C, gpre;
  int64_t gbuf_floats;  // one of the two G buffers
  size_t off_uh, off_rrecv, off_rown, off_yown, off_red, off_part, off_unew, off_bar,
      off_gbuf, total;
};

__host__ __device__ inline Layout make_layout(int64_t n, int64_t b, int s, int C,
                                              int tr_bytes) {
  Layout L;
  L.C = C;
  const int64_t per = (n + C - 1) / C;
  int nc = 8;
  while (nc < per) nc *= 2;
  L.nc = nc;
  L.rpb = (int)((b + C - 1) / C);
  const int64_t sb = (int64_t)s * b;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 15) / 16 * 16;
    return o;
  };
  take((size_t)nc * 4);  // x slice at 0
  L.off_uh = take((size_t)sb * tr_bytes);
  L.off_rrecv = take((size_t)C * s * L.rpb * 4);
  L.off_rown = take((size_t)s * L.rpb * tr_bytes);
  L.off_yown = take((size_t)s * L.rpb * 4);
  L.off_red = take((size_t)(L.rpb > kWarps ? L.rpb : kWarps) * tr_bytes);
  L.off_part = take((size_t)kThreads * 8 * 4);
  L.off_unew = take((size_t)L.rpb * tr_bytes);
  L.off_bar = take(4 * 8);
  L.gbuf_floats = s >= 2 ? (int64_t)L.rpb * gram_ld(s - 1, b) : 0;
  L.gpre = 0;
  L.off_gbuf = off;
  if (s >= 2 && off + 2 * (size_t)L.gbuf_floats * 4 <= kSmemMax) {
    L.gpre = 1;
    take(2 * (size_t)L.gbuf_floats * 4);
  }
  L.total = off;
  return L;
}

// Raw 8-element vector loads kept in registers until converted.
template <typename T> struct Raw8;
template <> struct Raw8<float> {
  float4 a, b;
  __device__ __forceinline__ void load(const float *p) {
    a = __ldg(reinterpret_cast<const float4 *>(p));
    b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
  }
  __device__ __forceinline__ void zero() { a = b = make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ void get(float (&o)[8]) const {
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
};
template <> struct Raw8<__nv_bfloat16> {
  uint4 w;
  __device__ __forceinline__ void load(const __nv_bfloat16 *p) {
    w = __ldg(reinterpret_cast<const uint4 *>(p));
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
  __device__ __forceinline__ void load(const __half *p) {
    w = __ldg(reinterpret_cast<const uint4 *>(p));
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

constexpr int kUnroll = 4;

template <typename TY, typename TR>
__global__ void __launch_bounds__(kThreads, 1)
k_chain(const ChainArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = a.n, b = a.b;
  const int s = a.s;
  const int64_t sb = (int64_t)s * b;
  const Layout L = make_layout(n, b, s, C, (int)sizeof(TR));
  const int nc = L.nc, rpb = L.rpb;
  const int64_t col0 = (int64_t)rank * nc;
  const int64_t l0 = (int64_t)rank * rpb;
  const int nown = (int)max((int64_t)0, min((int64_t)rpb, b - l0));

  extern __shared__ __align__(16) unsigned char smem[];
  float *xs = reinterpret_cast<float *>(smem);
  TR *uh = reinterpret_cast<TR *>(smem + L.off_uh);
  float *rrecv = reinterpret_cast<float *>(smem + L.off_rrecv);
  TR *rown = reinterpret_cast<TR *>(smem + L.off_rown);
  float *yown = reinterpret_cast<float *>(smem + L.off_yown);
  TR *red = reinterpret_cast<TR *>(smem + L.off_red);
  float *part = reinterpret_cast<float *>(smem + L.off_part);
  float *gbuf = reinterpret_cast<float *>(smem + L.off_gbuf);
  __shared__ int s_abort;
  const uint32_t bar_r = smem_u32(smem + L.off_bar);
  const uint32_t bar_u[2] = {bar_r + 8, bar_r + 16};

  if (tid == 0) {
    mbar_init(bar_r, 1);
    mbar_init(bar_u[0], 1);
    mbar_init(bar_u[1], 1);
    fence_mbar_init_cluster();
    s_abort = 0;
  }
  const TY *Y = static_cast<const TY *>(a.Y);
  for (int c = tid; c < nc; c += kThreads) xs[c] = (col0 + c < n) ? a.x[col0 + c] : 0.f;
  const int64_t gsz = gram_size(s, b);
  // barriers initialised in every CTA before any remote traffic
  cluster.sync();

  const int V = nc / 8;               // 8-element vectors in the slice
  const int tpr = V < 32 ? V : 32;    // threads per row in the margin
  const int vpt = V / tpr;            // vectors per thread per row
  const int rpp = kThreads / tpr;     // rows per pass
  const int gi = tid / tpr, li = tid % tpr;
  const uint32_t rrecv_a = smem_u32(rrecv), uh_a = smem_u32(uh);
  uint32_t J = 0;  // inner steps completed in this launch
  bool abort = false;

  for (int h = 0; h < a.nouter && !abort; ++h) {
    const int sh = (h == a.nouter - 1) ? a.s_last : s;
    const int64_t R = (int64_t)sh * b;
    const int64_t row0 = (int64_t)h * sb;
    const TY *Yh = Y + row0 * a.ldy;
    const float *Gh = a.G + (int64_t)h * gsz;
    if (tid == 0) mbar_arrive_expect_tx(bar_r, (uint32_t)(C * sh * nown * 4));

    // G rows of block j (own rows) -> gbuf[j & 1], 16-byte async copies
    auto g_prefetch = [&](int j) {
      const int64_t ldj = gram_ld(j, b);
      const float *src = Gh + gram_off(j, b) + l0 * ldj;
      float *dst = gbuf + (j & 1) * L.gbuf_floats;
      const int64_t chunks = (int64_t)nown * ldj / 4;
      for (int64_t q = tid; q < chunks; q += kThreads) cp_async16(smem_u32(dst + 4 * q), src + 4 * q);
    };
    if (L.gpre && sh >= 2) g_prefetch(1);
    cp_async_commit();

    // ---- A: partial margins over this CTA's column slice --------------------
    for (int64_t rb = 0; rb < R; rb += (int64_t)rpp * kUnroll) {
      float acc[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) acc[u] = 0.f;
      for (int v0 = 0; v0 < vpt; ++v0) {
        const int64_t col = (int64_t)(li + v0 * tpr) * 8;
        const bool colok = col0 + col < n;
        Raw8<TY> raw[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int64_t r = rb + gi + (int64_t)u * rpp;
          if (r < R && colok) raw[u].load(Yh + r * a.ldy + col0 + col);
          else raw[u].zero();
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          float f[8];
          raw[u].get(f);
#pragma unroll
          for (int i = 0; i < 8; ++i) acc[u] = fmaf(f[i], xs[col + i], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        for (int off = tpr / 2; off > 0; off >>= 1)
          acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], off);
        const int64_t r = rb + gi + (int64_t)u * rpp;
        if (li == 0 && r < R) {
          const int64_t j = r / b, l = r - j * b;
          const int owner = (int)(l / rpb);
          const int64_t ll = l - (int64_t)owner * rpb;
          const uint32_t dst = rrecv_a + (uint32_t)((((int64_t)rank * s + j) * rpb + ll) * 4);
          st_async(mapa(dst, owner), acc[u], mapa(bar_r, owner));
        }
      }
    }
    if (!mbar_wait_bounded(bar_r, h & 1, kWaitBudget)) atomicOr(&s_abort, 1);
    __syncthreads();
    if (s_abort) { abort = true; break; }

    // ---- C: own rows' margins (fixed summation order) and labels -----------
    for (int t = tid; t < sh * nown; t += kThreads) {
      const int j = t / nown, ll = t - j * nown;
      TR sum = 0;
      for (int src = 0; src < C; ++src) sum += (TR)rrecv[((int64_t)src * s + j) * rpb + ll];
      rown[j * rpb + ll] = sum;
      yown[j * rpb + ll] = a.ylab[row0 + (int64_t)j * b + l0 + ll];
    }
    __syncthreads();

    // ---- D: inner s-step recurrence -----------------------------------------
    const int wpr = nown > 0 ? max(1, kWarps / nown) : 1;
    for (int j = 0; j < sh; ++j) {
      if (j > 0) {
        const int64_t jb = (int64_t)j * b;
        const int64_t ldj = gram_ld(j, b);
        const float *gsrc;
        if (L.gpre) {
          if (j + 1 < sh) g_prefetch(j + 1);
          cp_async_commit();
          cp_async_wait<1>();
          __syncthreads();
          gsrc = gbuf + (j & 1) * L.gbuf_floats;
        } else {
          gsrc = Gh + gram_off(j, b) + l0 * ldj;
        }
        for (int item = warp; item < nown * wpr; item += kWarps) {
          const int rr = item / wpr, pp = item - rr * wpr;
          const float *grow = gsrc + rr * ldj;
          TR acc0 = 0, acc1 = 0;
          int64_t c = (int64_t)pp * 32 + lane;
          const int64_t step = 32 * (int64_t)wpr;
          for (; c + step < jb; c += 2 * step) {
            acc0 += (TR)grow[c] * uh[c];
            acc1 += (TR)grow[c + step] * uh[c + step];
          }
          if (c < jb) acc0 += (TR)grow[c] * uh[c];
          TR acc = acc0 + acc1;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
          if (lane == 0) red[item] = acc;
        }
        __syncthreads();
      }
      if (tid < nown) {
        TR corr = 0;
        if (j > 0)
          for (int p = 0; p < wpr; ++p) corr += red[tid * wpr + p];
        const TR rj = rown[j * rpb + tid];
        const TR z = (TR)a.cpow[j] * rj -
                     (j > 0 ? (TR)a.alpha * (TR)a.cpow[j - 1] * corr : (TR)0);
        const TR u = dloss<TR>(a.loss, z, (TR)yown[j * rpb + tid]);
        if (!isfinite(z) || !isfinite(u)) atomicOr(a.flag, FLAG_NONFINITE);
        const TR uw = u * (TR)a.cinv[j];
        const uint32_t dst = uh_a + (uint32_t)(((int64_t)j * b + l0 + tid) * sizeof(TR));
        for (int d = 0; d < C; ++d) st_async(mapa(dst, d), uw, mapa(bar_u[J & 1], d));
      }
      if (tid == 0) mbar_arrive_expect_tx(bar_u[J & 1], (uint32_t)(b * sizeof(TR)));
      if (!mbar_wait_bounded(bar_u[J & 1], (J >> 1) & 1, kWaitBudget)) atomicOr(&s_abort, 1);
      ++J;
      __syncthreads();
      if (s_abort) { abort = true; break; }
    }
    if (abort) break;

    // ---- E: x <- c^{sh} x - alpha c^{sh-1} Y^T (c^{-j} u), own slice ---------
    {
      const int RG = kThreads / V;
      const int g = tid / V, v = tid - (tid / V) * V;
      const int64_t col = (int64_t)v * 8;
      float acc[8], cmp[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) { acc[i] = 0.f; cmp[i] = 0.f; }
      if (g < RG && col0 + col < n) {
        for (int64_t rb = g; rb < R; rb += (int64_t)RG * kUnroll) {
          Raw8<TY> raw[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const int64_t r = rb + (int64_t)u * RG;
            if (r < R) raw[u].load(Yh + r * a.ldy + col0 + col);
            else raw[u].zero();
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const int64_t r = rb + (int64_t)u * RG;
            if (r >= R) break;
            float f[8];
            raw[u].get(f);
            const float w = (float)uh[r];
            if (a.kahan) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float yv = fmaf(f[i], w, -cmp[i]);
                const float t2 = acc[i] + yv;
                cmp[i] = (t2 - acc[i]) - yv;
                acc[i] = t2;
              }
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) acc[i] = fmaf(f[i], w, acc[i]);
            }
          }
        }
      }
      if (g < RG) {
#pragma unroll
        for (int i = 0; i < 8; ++i) part[(int64_t)g * nc + col + i] = acc[i];
      }
      __syncthreads();
      const float decay = (float)a.cpow[sh];
      const float stp = (float)((double)a.alpha * a.cpow[sh - 1]);
      for (int c = tid; c < nc; c += kThreads) {
        float S = 0.f, cS = 0.f;
        for (int gg = 0; gg < RG; ++gg) {
          const float yv = part[(int64_t)gg * nc + c] - cS;
          const float t2 = S + yv;
          cS = (t2 - S) - yv;
          S = t2;
        }
        if (col0 + c < n) {
          const float xn = fmaf(-stp, S, decay * xs[c]);
          if (!isfinite(xn)) atomicOr(a.flag, FLAG_NONFINITE);
          xs[c] = xn;
        }
      }
      __syncthreads();
    }
  }
  cp_async_wait<0>();
  if (abort) {
    if (tid == 0) atomicOr(a.flag, FLAG_TIMEOUT);
  } else {
    for (int c = tid; c < nc; c += kThreads)
      if (col0 + c < n) a.x[col0 + c] = xs[c];
  }
  cluster.sync();
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

template <typename TY, typename TR>
int launch_t(const ChainArgs &a, cudaStream_t st) {
  const int C = a.cluster;
  const Layout L = make_layout(a.n, a.b, a.s, C, (int)sizeof(TR));
  if (L.total > kSmemMax)
    return set_error(GLM_EUNSUPPORTED, "chain: shared-memory need exceeds 227 KB "
                                       "(reduce s*b or raise the cluster size)");
  auto kern = k_chain<TY, TR>;
  GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)L.total));
  if (C > 8)
    GLM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = make_cfg(C, L.total, st, attr);
  GLM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  return GLM_OK;
}

// every CTA must own at least one row of each block (one-way exchanges rely
// on each CTA taking part in every inner step)
bool cluster_rows_ok(int C, int64_t b) {
  const int64_t rpb = (b + C - 1) / C;
  return (int64_t)(C - 1) * rpb < b;
}

template <typename TY, typename TR>
int max_cluster_t(const ChainArgs &a) {
  auto kern = k_chain<TY, TR>;
  for (int C = 16; C >= 1; C /= 2) {
    if (!cluster_rows_ok(C, a.b)) continue;
    const Layout L = make_layout(a.n, a.b, a.s, C, (int)sizeof(TR));
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
    return set_error(GLM_EINVAL, "chain: cluster size must be 1..16 and leave every CTA a row");
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
