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
//    I_j; it sums the C partial margins of those rows (pushed into its
//    shared memory over DSMEM) and evaluates their corrected margins
//        z_j = c^j r_j - alpha c^{j-1} sum_{i<j} G_{j,i} (c^{-i} u_i)
//    and residuals, then broadcasts c^{-j} u_j to every CTA.
// One cluster barrier follows the margin exchange and one each inner step,
// so an outer iteration of s inner steps costs s + 1 cluster barriers.
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

struct Layout {
  int nc, rpb, C;
  size_t off_uh, off_rrecv, off_rown, off_yown, off_red, off_part, off_unew, total;
};

__host__ __device__ inline Layout make_layout(int64_t n, int64_t b, int s, int C,
                                              int tr_bytes) {
  Layout L;
  L.C = C;
  int64_t per = (n + C - 1) / C;
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
  take((size_t)nc * 4);                                   // x slice at 0
  L.off_uh = take((size_t)sb * tr_bytes);
  L.off_rrecv = take((size_t)C * s * L.rpb * 4);
  L.off_rown = take((size_t)s * L.rpb * tr_bytes);
  L.off_yown = take((size_t)s * L.rpb * 4);
  L.off_red = take((size_t)(L.rpb > kWarps ? L.rpb : kWarps) * tr_bytes);
  L.off_part = take((size_t)kThreads * 8 * 4);
  L.off_unew = take((size_t)L.rpb * tr_bytes);
  L.total = off;
  return L;
}

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
  TR *unew = reinterpret_cast<TR *>(smem + L.off_unew);

  const TY *Y = static_cast<const TY *>(a.Y);
  for (int c = tid; c < nc; c += kThreads)
    xs[c] = (col0 + c < n) ? a.x[col0 + c] : 0.f;
  const int64_t gsz = b * b * (int64_t)s * (s - 1) / 2;
  // every CTA of the cluster must be running before remote shared writes
  cluster.sync();

  const int V = nc / 8;                    // 8-element vectors in the slice
  const int tpr = V < 32 ? V : 32;         // threads per row in the margin
  const int rpp = kThreads / tpr;          // rows per pass
  const int gi = tid / tpr, li = tid % tpr;

  for (int h = 0; h < a.nouter; ++h) {
    const int sh = (h == a.nouter - 1) ? a.s_last : s;
    const int64_t R = (int64_t)sh * b;
    const int64_t row0 = (int64_t)h * sb;
    const TY *Yh = Y + row0 * a.ldy;

    // ---- A: partial margins over this CTA's column slice ------------------
    for (int64_t rb = 0; rb < R; rb += rpp) {
      const int64_t r = rb + gi;
      float acc = 0.f;
      if (r < R) {
        for (int v = li; v < V; v += tpr) {
          const int64_t col = (int64_t)v * 8;
          if (col0 + col < n) {
            float f[8];
            Vec8<TY>::load(Yh + r * a.ldy + col0 + col, f);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc = fmaf(f[i], xs[col + i], acc);
          }
        }
      }
      for (int off = tpr / 2; off > 0; off >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (li == 0 && r < R) {
        const int64_t j = r / b, l = r - j * b;
        const int owner = (int)(l / rpb);
        const int64_t ll = l - (int64_t)owner * rpb;
        float *dst = cluster.map_shared_rank(rrecv, owner);
        dst[((int64_t)rank * s + j) * rpb + ll] = acc;
      }
    }
    cluster.sync();

    // ---- C: own rows' margins (fixed summation order) and labels ----------
    for (int t = tid; t < sh * nown; t += kThreads) {
      const int j = t / nown, ll = t - j * nown;
      TR sum = 0;
      for (int src = 0; src < C; ++src) sum += (TR)rrecv[((int64_t)src * s + j) * rpb + ll];
      rown[j * rpb + ll] = sum;
      yown[j * rpb + ll] = a.ylab[row0 + (int64_t)j * b + l0 + ll];
    }
    __syncthreads();

    // ---- D: inner s-step recurrence ---------------------------------------
    const int wpr = nown > 0 ? max(1, kWarps / nown) : 1;
    for (int j = 0; j < sh; ++j) {
      if (j > 0 && nown > 0) {
        const int64_t jb = (int64_t)j * b;
        const float *Gj = a.G + (int64_t)h * gsz + b * b * ((int64_t)j * (j - 1) / 2);
        for (int item = warp; item < nown * wpr; item += kWarps) {
          const int rr = item / wpr, pp = item - rr * wpr;
          const float *grow = Gj + (l0 + rr) * jb;
          TR acc = 0;
          for (int64_t c = (int64_t)pp * 32 + lane; c < jb; c += 32 * wpr)
            acc += (TR)__ldg(grow + c) * uh[c];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
          if (lane == 0) red[item] = acc;
        }
      }
      __syncthreads();
      if (tid < nown) {
        TR corr = 0;
        if (j > 0)
          for (int p = 0; p < wpr; ++p) corr += red[tid * wpr + p];
        const TR rj = rown[j * rpb + tid];
        const TR z = (TR)a.cpow[j] * rj -
                     (j > 0 ? (TR)a.alpha * (TR)a.cpow[j - 1] * corr : (TR)0);
        const TR u = dloss<TR>(a.loss, z, (TR)yown[j * rpb + tid]);
        if (!isfinite(z) || !isfinite(u)) atomicOr(a.flag, FLAG_NONFINITE);
        unew[tid] = u * (TR)a.cinv[j];
      }
      __syncthreads();
      for (int t = tid; t < nown * C; t += kThreads) {
        const int rr = t / C, dst = t - rr * C;
        TR *ud = cluster.map_shared_rank(uh, dst);
        ud[(int64_t)j * b + l0 + rr] = unew[rr];
      }
      cluster.sync();
    }

    // ---- E: x <- c^{sh} x - alpha c^{sh-1} Y^T (c^{-j} u), own slice -------
    {
      const int RG = kThreads / V;
      const int g = tid / V, v = tid - (tid / V) * V;
      const int64_t col = (int64_t)v * 8;
      float acc[8], cmp[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) { acc[i] = 0.f; cmp[i] = 0.f; }
      if (g < RG && col0 + col < n) {
        for (int64_t r = g; r < R; r += RG) {
          float f[8];
          Vec8<TY>::load(Yh + r * a.ldy + col0 + col, f);
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
      if (g < RG) {
#pragma unroll
        for (int i = 0; i < 8; ++i) part[(int64_t)g * nc + col + i] = acc[i];
      }
      __syncthreads();
      const float decay = (float)a.cpow[sh];
      const float step = (float)((double)a.alpha * a.cpow[sh - 1]);
      for (int c = tid; c < nc; c += kThreads) {
        float S = 0.f, cS = 0.f;
        for (int gg = 0; gg < RG; ++gg) {
          const float yv = part[(int64_t)gg * nc + c] - cS;
          const float t2 = S + yv;
          cS = (t2 - S) - yv;
          S = t2;
        }
        if (col0 + c < n) {
          const float xn = fmaf(-step, S, decay * xs[c]);
          if (!isfinite(xn)) atomicOr(a.flag, FLAG_NONFINITE);
          xs[c] = xn;
        }
      }
      __syncthreads();
    }
  }
  for (int c = tid; c < nc; c += kThreads)
    if (col0 + c < n) a.x[col0 + c] = xs[c];
  cluster.sync();
}

template <typename TY, typename TR>
int launch_t(const ChainArgs &a, cudaStream_t st) {
  const int C = a.cluster;
  const Layout L = make_layout(a.n, a.b, a.s, C, (int)sizeof(TR));
  if (L.total > 227 * 1024)
    return set_error(GLM_EUNSUPPORTED, "chain: shared-memory need exceeds 227 KB "
                                       "(reduce s*b or raise the cluster size)");
  auto kern = k_chain<TY, TR>;
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

template <typename TY, typename TR>
int max_cluster_t(const ChainArgs &a) {
  auto kern = k_chain<TY, TR>;
  for (int C = 16; C >= 1; C /= 2) {
    const Layout L = make_layout(a.n, a.b, a.s, C, (int)sizeof(TR));
    if (L.total > 227 * 1024) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L.total) != cudaSuccess) { cudaGetLastError(); continue; }
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                      1) != cudaSuccess) { cudaGetLastError(); continue; }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = L.total;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
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
  if (a.cluster < 1 || a.cluster > 16) return set_error(GLM_EINVAL, "chain: cluster size");
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
