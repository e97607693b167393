// glm_api.cu -- the C ABI of libglm (declared in include/glm.h): dataset
// handles, run orchestration (chunked staging of x-independent work, the
// cluster chain, CUDA-graph capture and replay), risk evaluation and the
// kernel-level entry points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <string>
#include <vector>

#include "glm_internal.cuh"
#include "glm_baselines.cuh"

namespace glm {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                 cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? GLM_ENOMEM : GLM_ECUDA;
}

// glm_debug_fail_alloc: allocations left before an injected failure (< 0: off)
static std::atomic<int64_t> g_alloc_countdown{-1};

cudaError_t dev_malloc(void **p, size_t bytes) {
  int64_t c = g_alloc_countdown.load();
  while (c >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
      if (c == 0) {  // this allocation is the injected failure
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

int DevBuf::ensure(size_t need) {
  if (need <= bytes && ptr) return GLM_OK;
  release();
  cudaError_t e = dev_malloc(&ptr, need ? need : 16);
  if (e != cudaSuccess) {
    ptr = nullptr;
    bytes = 0;
    return cuda_error(e, "cudaMalloc(run scratch)");
  }
  bytes = need;
  return GLM_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

bool RunKey::operator==(const RunKey &o) const {
  return s == o.s && gram_dt == o.gram_dt && gemv_dt == o.gemv_dt && rec64 == o.rec64 &&
         kahan == o.kahan && cluster == o.cluster && gram_impl == o.gram_impl &&
         sgd == o.sgd && b == o.b && iters == o.iters && first_iter == o.first_iter &&
         chunk == o.chunk && seed == o.seed && problem == o.problem && eta == o.eta &&
         lambda == o.lambda && x == o.x && timing == o.timing && probe == o.probe &&
         chain == o.chain;
}

int loss_partials_needed();

namespace {

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_handle(Handle *h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    h->ygram[k].release();
    h->ygemv[k].release();
    h->ylab[k].release();
    h->yscale[k].release();
    h->gbuf[k].release();
    if (h->ev_bulk[k]) cudaEventDestroy(h->ev_bulk[k]);
    if (h->ev_chain[k]) cudaEventDestroy(h->ev_chain[k]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  cudaFree(h->A);
  cudaFree(h->y);
  cudaFree(h->colscale);
  cudaFree(h->A8);
  cudaFree(h->rowscale8);
  cudaFree(h->dflag);
  cudaFree(h->loss_partials);
  cudaFree(h->loss_out);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Resolved options of one run.
struct RunPlan {
  int s = 1;
  int64_t b = 1, iters = 0, H = 0, chunk = 1;
  int gram_dt = GLM_F32, gemv_dt = GLM_F32, rec64 = 0, kahan = 1, cluster = 1;
  int gram_impl = 1, sgd = 0, use_graph = 1, timing = 0, chain_impl = 1;
  int64_t chunks = 0, launches = 0;
  int64_t ld_gram = 0, ld_gemv = 0;  // 0 ld_gemv: GEMV reads the Gram copy
  float eta = 0.f, lambda = 0.f, alpha = 0.f;
  double c = 1.0;
  uint64_t seed = 0;
  uint32_t problem = 0;
  int64_t first_iter = 0;
  int64_t probe = 0;
  float *x = nullptr;
};

int resolve(Handle *h, int s, int64_t b, float eta, float lambda, int64_t iters,
            uint64_t seed, float *x, const glm_ca_opts *o, bool sgd, RunPlan &p) {
  if (!h) return set_error(GLM_EINVAL, "null handle");
  if (!x) return set_error(GLM_EINVAL, "x is NULL");
  if (s < 1 || s > 256) return set_error(GLM_EINVAL, "s must be in [1, 256]");
  if (b < 1 || b > 65536) return set_error(GLM_EINVAL, "b must be in [1, 65536]");
  if (iters < 0) return set_error(GLM_EINVAL, "iters must be >= 0");
  if (!(eta > 0.f) || !isfinite(eta)) return set_error(GLM_EINVAL, "eta must be finite and > 0");
  if (!(lambda >= 0.f) || !isfinite(lambda)) return set_error(GLM_EINVAL, "lambda must be >= 0");
  const double c = 1.0 - (double)eta * (double)lambda;
  if (!(c > 0.0)) return set_error(GLM_EINVAL, "eta * lambda must be < 1");
  if ((double)(s - 1) * -log2(c) > 60.0)
    return set_error(GLM_EUNSUPPORTED, "c^-(s-1) exceeds 2^60 (eta*lambda too large for s)");
  glm_ca_opts d;
  glm_ca_opts_default(&d);
  if (!o) o = &d;
  p.s = s;
  p.b = b;
  p.iters = iters;
  p.eta = eta;
  p.lambda = lambda;
  p.alpha = (float)((double)eta / (double)b);
  p.c = c;
  p.seed = seed;
  p.problem = o->problem;
  p.first_iter = o->first_iter;
  if (o->first_iter < 0) return set_error(GLM_EINVAL, "first_iter must be >= 0");
  p.x = x;
  p.sgd = sgd ? 1 : 0;
  p.kahan = o->kahan ? 1 : 0;
  p.use_graph = o->use_graph ? 1 : 0;
  p.timing = o->timing ? 1 : 0;
  if (o->wait_probe_cycles < 0) return set_error(GLM_EINVAL, "wait_probe_cycles must be >= 0");
  p.probe = o->wait_probe_cycles;
  // precision slots
  int gdt = o->gram_dtype < 0 ? h->dtype : o->gram_dtype;
  if (sgd) gdt = (o->gram_dtype < 0) ? GLM_F32 : o->gram_dtype;
  if (gdt != GLM_F32 && gdt != GLM_TF32 && gdt != GLM_BF16 && gdt != GLM_F16 && gdt != GLM_E4M3)
    return set_error(GLM_EINVAL, "gram_dtype must be F32, TF32, BF16, F16 or E4M3");
  if (gdt == GLM_E4M3 && !h->A8)
    return set_error(GLM_EINVAL, "E4M3 Gram needs a handle created with fp8_copy = 1");
  int vdt = o->gemv_dtype;
  if (vdt < 0) vdt = (gdt == GLM_E4M3) ? h->dtype : gdt;
  if (vdt != GLM_F32 && vdt != GLM_TF32 && vdt != GLM_BF16 && vdt != GLM_F16)
    return set_error(GLM_EINVAL, "gemv_dtype must be F32, TF32, BF16 or F16");
  p.gram_dt = gdt;
  p.gemv_dt = vdt;
  if (o->recurrence_f64 < -1 || o->recurrence_f64 > 2)
    return set_error(GLM_EINVAL, "recurrence_f64 must be -1, 0, 1 or 2");
  p.rec64 = o->recurrence_f64 < 0 ? (s >= 32 ? 1 : 0) : o->recurrence_f64;
  if (o->chain_impl < 0 || o->chain_impl > 2)
    return set_error(GLM_EINVAL, "chain_impl must be 0, 1 or 2");
  p.ld_gram = round_up(h->n, gdt == GLM_E4M3 ? 128 : 64);
  p.ld_gemv = (vdt == gdt) ? 0 : round_up(h->n, 64);
  // Gram implementation
  if (o->gram_impl == 2 && !gram_tc_supported(gdt, p.ld_gram))
    return set_error(GLM_EUNSUPPORTED, "tcgen05 Gram does not support this operand type");
  if ((o->gram_impl == 3 || o->gram_impl == 4) && gdt != GLM_F16)
    return set_error(GLM_EINVAL, "gram_impl 3/4 (FP16 accumulation) needs gram_dtype GLM_F16");
  if (o->gram_impl == 4 && !gram_tc_supported(gdt, round_up(h->n, 64)))
    return set_error(GLM_EUNSUPPORTED, "tcgen05 Gram does not support this operand type");
  p.gram_impl = o->gram_impl == 0 ? (gram_tc_supported(gdt, p.ld_gram) ? 2 : 1) : o->gram_impl;
  if (p.gram_impl < 1 || p.gram_impl > 4) return set_error(GLM_EINVAL, "gram_impl");
  // chunking
  p.H = (iters + s - 1) / s;
  const int64_t sb = (int64_t)s * b;
  const int64_t gsz = gram_size(s, b);
  const int64_t per_outer = sb * (p.ld_gram * elem_bytes(gdt) +
                                  (p.ld_gemv ? p.ld_gemv * elem_bytes(vdt) : 0) + 8) +
                            gsz * 4;
  int64_t chunk = o->chunk_outer;
  if (chunk <= 0) {
    const int64_t budget = 64ll << 20;
    chunk = std::max<int64_t>(1, budget / std::max<int64_t>(per_outer, 1));
  }
  chunk = std::min<int64_t>(chunk, std::max<int64_t>(p.H, 1));
  chunk = std::min<int64_t>(chunk, 65535);
  p.chunk = chunk;
  // cluster
  ChainArgs probe = {};
  probe.dt = vdt;
  probe.n = h->n;
  probe.b = b;
  probe.s = s;
  probe.rec64 = p.rec64 == 1 ? 1 : 0;
  probe.prefetch = 1;
  const int cmax_res = chain_max_cluster(probe);
  const int cmax = std::max(cmax_res, 16);  // the streaming chain fits any cluster width
  if (cmax < 1)
    return set_error(GLM_EUNSUPPORTED, "s*b too large for the on-chip recurrence state");
  (void)cmax;
  int C = o->cluster;
  if (C <= 0) {
    // widest cluster that keeps >= 4 rows of each block and >= 32 columns
    // per CTA (16-byte exchanges, full-width slice rows); measured best on
    // the 2^20 x 512 and 8192 x 256 workloads
    C = 1;
    while (C < 16 && b / (2 * C) >= 4 && h->n / (2 * C) >= 32) C *= 2;
  }
  if (C > cmax) C = cmax;
  if (C < 1 || C > 16 || (C & (C - 1)))
    return set_error(GLM_EINVAL, "cluster must be a power of two in [1, 16]");
  while (C > 1 && !chain_cluster_ok(C, b)) C /= 2;
  p.cluster = C;
  // chain kernel: resident when it stages the step (and the recurrence is
  // FP32 / FP64), else streaming
  probe.cluster = C;
  probe.ldy = p.ld_gemv ? p.ld_gemv : p.ld_gram;
  const bool res_ok = cmax_res >= C && p.rec64 != 2 && chain_resident_staged(probe);
  probe.rec64 = p.rec64;
  const bool str_ok = chain_stream_ok(probe);
  if (o->chain_impl == 1) {
    if (p.rec64 == 2) return set_error(GLM_EINVAL, "the resident chain has no compensated FP32 mode");
    if (cmax_res < C) return set_error(GLM_EUNSUPPORTED, "s*b too large for the resident chain");
    p.chain_impl = 1;
  } else if (o->chain_impl == 2) {
    if (!str_ok) return set_error(GLM_EUNSUPPORTED, "shape outside the streaming chain's limits");
    p.chain_impl = 2;
  } else {
    // measured on GB300: the streaming chain wins whenever the resident one
    // cannot stage the step, except with hardware FP64 sums, where the
    // resident chain's FP64 row layout is faster (c5 shape: 5.3 s against
    // 6.6 s per 65,536 iterations)
    const bool res_fp64 = p.rec64 == 1 && cmax_res >= C;
    p.chain_impl = res_ok || res_fp64 || (!str_ok && p.rec64 != 2 && cmax_res >= C) ? 1 : 2;
    if (p.chain_impl == 2 && !str_ok)
      return set_error(GLM_EUNSUPPORTED, "s*b too large for the on-chip recurrence state");
  }
  p.chunks = (p.H + p.chunk - 1) / p.chunk;
  p.launches = p.chunks * (s > 1 ? 3 : 2);
  return GLM_OK;
}

// Record timing event (chunk c, kernel k, edge e) when the run is timed.
int tmark(Handle *h, const RunPlan &p, cudaStream_t st, int64_t c, int k, int e) {
  if (!p.timing) return GLM_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  GLM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  cudaEvent_t ev = h->tev[(size_t)(c * 6 + k * 2 + e)];
  if (cs == cudaStreamCaptureStatusActive)
    GLM_CUDA_TRY(cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal));
  else
    GLM_CUDA_TRY(cudaEventRecord(ev, st));
  return GLM_OK;
}

int ensure_scratch(Handle *h, const RunPlan &p, bool &realloc) {
  const int64_t sb = (int64_t)p.s * p.b;
  const int64_t rows = p.chunk * sb;
  const int64_t gsz = gram_size(p.s, p.b);
  const int nb = p.chunks > 1 ? 2 : 1;
  void *before[10], *after[10];
  for (int k = 0; k < 2; ++k) {
    before[5 * k] = h->ygram[k].ptr; before[5 * k + 1] = h->ygemv[k].ptr;
    before[5 * k + 2] = h->ylab[k].ptr; before[5 * k + 3] = h->yscale[k].ptr;
    before[5 * k + 4] = h->gbuf[k].ptr;
  }
  for (int k = 0; k < nb; ++k) {
    GLM_TRY(h->ygram[k].ensure((size_t)rows * p.ld_gram * elem_bytes(p.gram_dt)));
    if (p.ld_gemv)
      GLM_TRY(h->ygemv[k].ensure((size_t)rows * p.ld_gemv * elem_bytes(p.gemv_dt)));
    GLM_TRY(h->ylab[k].ensure((size_t)p.chunk * round_up(sb, 4) * 4));
    GLM_TRY(h->yscale[k].ensure((size_t)rows * 4));
    GLM_TRY(h->gbuf[k].ensure((size_t)std::max<int64_t>(1, p.chunk * gsz) * 4));
  }
  for (int k = 0; k < 2; ++k) {
    after[5 * k] = h->ygram[k].ptr; after[5 * k + 1] = h->ygemv[k].ptr;
    after[5 * k + 2] = h->ylab[k].ptr; after[5 * k + 3] = h->yscale[k].ptr;
    after[5 * k + 4] = h->gbuf[k].ptr;
  }
  realloc = memcmp(before, after, sizeof(before)) != 0;
  if (!h->side) {
    GLM_CUDA_TRY(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    GLM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    GLM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    for (int k = 0; k < 2; ++k) {
      GLM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_bulk[k], cudaEventDisableTiming));
      GLM_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_chain[k], cudaEventDisableTiming));
    }
  }
  return GLM_OK;
}

// Enqueue a whole run on stream st.
int enqueue_run(Handle *h, const RunPlan &p, cudaStream_t st) {
  const int64_t sb = (int64_t)p.s * p.b;
  if (p.timing) {
    while ((int64_t)h->tev.size() < p.chunks * 6) {
      cudaEvent_t e;
      GLM_CUDA_TRY(cudaEventCreate(&e));
      h->tev.push_back(e);
    }
    h->tev_chunks = p.chunks;
    h->tev_valid = p.s > 1 ? 7 : 5;  // bit k: kernel k was timed
  }
  ChainArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.dt = p.gemv_dt;
  ca.ldy = p.ld_gemv ? p.ld_gemv : p.ld_gram;
  ca.x = p.x;
  ca.flag = h->dflag;
  ca.n = h->n;
  ca.b = p.b;
  ca.s = p.s;
  ca.loss = h->loss;
  ca.alpha = p.alpha;
  ca.rec64 = p.rec64;
  ca.kahan = p.kahan;
  ca.cluster = p.cluster;
  ca.sbp = round_up(sb, 4);
  ca.prefetch = 1;
  ca.probe = p.probe;
  double cp = 1.0;
  for (int j = 0; j <= p.s; ++j) {
    ca.cpow[j] = cp;
    ca.cinv[j] = 1.0 / cp;
    cp *= p.c;
  }
  // the x-independent work (gather, Gram) runs on the side stream, one chunk
  // ahead of the chain on `st`; chunk buffers alternate
  const int nb = p.chunks > 1 ? 2 : 1;
  cudaStream_t side = h->side;
  GLM_CUDA_TRY(cudaEventRecord(h->ev_fork, st));
  GLM_CUDA_TRY(cudaStreamWaitEvent(side, h->ev_fork, 0));
  for (int64_t h0 = 0; h0 < p.H; h0 += p.chunk) {
    const int buf = (int)((h0 / p.chunk) % nb);
    if (h0 / p.chunk >= nb) GLM_CUDA_TRY(cudaStreamWaitEvent(side, h->ev_chain[buf], 0));
    ca.Y = p.ld_gemv ? h->ygemv[buf].ptr : h->ygram[buf].ptr;
    ca.ylab = static_cast<const float *>(h->ylab[buf].ptr);
    ca.G = static_cast<const float *>(h->gbuf[buf].ptr);
    const int64_t nout = std::min<int64_t>(p.chunk, p.H - h0);
    const int64_t it0 = h0 * p.s;                          // first iteration of chunk
    const int64_t it1 = std::min<int64_t>(p.iters, (h0 + nout) * p.s);
    const int64_t rows = (it1 - it0) * p.b;
    const int s_last = (int)(it1 - (h0 + nout - 1) * p.s);
    GatherArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.A = h->A;
    ga.lda = h->lda;
    ga.a_dt = h->dtype;
    ga.colscale = h->colscale;
    ga.A8 = h->A8;
    ga.rs8 = h->rowscale8;
    ga.lda8 = h->lda8;
    ga.y = h->y;
    ga.m = h->m;
    ga.n = h->n;
    ga.rows = rows;
    ga.flag = h->dflag;
    ga.q0 = (uint64_t)((p.first_iter + it0) * p.b);
    ga.seed = p.seed;
    ga.problem = p.problem;
    ga.out1 = h->ygram[buf].ptr;
    ga.dt1 = p.gram_dt;
    ga.ld1 = p.ld_gram;
    if (p.ld_gemv) {
      ga.out2 = h->ygemv[buf].ptr;
      ga.dt2 = p.gemv_dt;
      ga.ld2 = p.ld_gemv;
    }
    ga.ylab = static_cast<float *>(h->ylab[buf].ptr);
    ga.rscale = static_cast<float *>(h->yscale[buf].ptr);
    ga.lab_sb = sb;
    ga.lab_sbp = round_up(sb, 4);
    const int64_t ci = h0 / p.chunk;
    GLM_TRY(tmark(h, p, side, ci, 0, 0));
    GLM_TRY(launch_gather(ga, side));
    GLM_TRY(tmark(h, p, side, ci, 0, 1));
    if (p.s > 1) {
      GramArgs gr;
      gr.Y = h->ygram[buf].ptr;
      gr.dt = p.gram_dt;
      gr.ld = p.ld_gram;
      gr.rs = p.gram_dt == GLM_E4M3 ? static_cast<const float *>(h->yscale[buf].ptr) : nullptr;
      gr.nouter = nout;
      gr.rows = rows;
      gr.s = p.s;
      gr.b = p.b;
      gr.n = h->n;
      gr.G = static_cast<float *>(h->gbuf[buf].ptr);
      gr.flag = h->dflag;
      gr.probe = p.probe;
      gr.tile_n = 0;
      GLM_TRY(tmark(h, p, side, ci, 1, 0));
      if (p.gram_impl == 2) GLM_TRY(launch_gram_tc(gr, side));
      else if (p.gram_impl == 3) GLM_TRY(launch_gram_simt_f16acc(gr, side));
      else if (p.gram_impl == 4) GLM_TRY(launch_gram_tc_f16acc(gr, side));
      else GLM_TRY(launch_gram_simt(gr, side));
      GLM_TRY(tmark(h, p, side, ci, 1, 1));
    }
    GLM_CUDA_TRY(cudaEventRecord(h->ev_bulk[buf], side));
    GLM_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_bulk[buf], 0));
    ca.nouter = (int)nout;
    ca.s_last = s_last;
    GLM_TRY(tmark(h, p, st, ci, 2, 0));
    if (p.chain_impl == 2) GLM_TRY(launch_chain_stream(ca, st));
    else GLM_TRY(launch_chain(ca, st));
    GLM_TRY(tmark(h, p, st, ci, 2, 1));
    GLM_CUDA_TRY(cudaEventRecord(h->ev_chain[buf], st));
  }
  GLM_CUDA_TRY(cudaEventRecord(h->ev_join, side));
  GLM_CUDA_TRY(cudaStreamWaitEvent(st, h->ev_join, 0));
  return GLM_OK;
}

int run_common(Handle *h, int s, int64_t b, float eta, float lambda, int64_t iters,
               uint64_t seed, float *x, const glm_ca_opts *o, bool sgd) {
  RunPlan p;
  GLM_TRY(resolve(h, s, b, eta, lambda, iters, seed, x, o, sgd, p));
  if (iters == 0) return GLM_OK;
  bool realloc = false;
  GLM_TRY(ensure_scratch(h, p, realloc));
  if (!p.use_graph) return enqueue_run(h, p, h->stream);
  RunKey key;
  key.s = p.s; key.gram_dt = p.gram_dt; key.gemv_dt = p.gemv_dt; key.rec64 = p.rec64;
  key.kahan = p.kahan; key.cluster = p.cluster; key.gram_impl = p.gram_impl; key.sgd = p.sgd;
  key.b = p.b; key.iters = p.iters; key.first_iter = p.first_iter; key.chunk = p.chunk;
  key.seed = p.seed; key.problem = p.problem; key.eta = p.eta; key.lambda = p.lambda;
  key.x = p.x; key.timing = p.timing; key.probe = p.probe; key.chain = p.chain_impl;
  if (realloc && h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (!h->graph || !(h->graph_key == key)) {
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
    }
    cudaStream_t cap;
    GLM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_error(e, "cudaStreamBeginCapture");
    }
    const int rc = enqueue_run(h, p, cap);
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != GLM_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->graph = nullptr;
      return cuda_error(e, "cudaGraphInstantiate");
    }
    h->graph_key = key;
  }
  GLM_CUDA_TRY(cudaGraphLaunch(h->graph, h->stream));
  return GLM_OK;
}

}  // namespace

// The precision slots, Gram kernel and stream id a run with these arguments
// resolves to (the column-partitioned steps use the fused path's rules).
int resolve_public(Handle *h, int s, int64_t b, float eta, float lambda, int64_t iters,
                   uint64_t seed, float *x, const glm_ca_opts *o, int &gram_dt, int &gemv_dt,
                   int &rec64, int &kahan, int &gram_impl, int64_t &ld_gram, int64_t &ld_gemv,
                   uint32_t &problem) {
  RunPlan p;
  GLM_TRY(resolve(h, s, b, eta, lambda, iters, seed, x, o, false, p));
  gram_dt = p.gram_dt;
  gemv_dt = p.gemv_dt;
  rec64 = p.rec64;
  kahan = p.kahan;
  gram_impl = p.gram_impl;
  ld_gram = p.ld_gram;
  ld_gemv = p.ld_gemv;
  problem = p.problem;
  return GLM_OK;
}

}  // namespace glm

using namespace glm;

extern "C" {

const char *glm_last_error(void) { return g_last_error.c_str(); }

const char *glm_version(void) { return "libglm 0.1 (sm_103a)"; }

int glm_checked_build(void) {
#ifdef GLM_CHECKED
  return 1;
#else
  return 0;
#endif
}

void glm_create_opts_default(glm_create_opts *o) {
  if (!o) return;
  o->input_dtype = GLM_F32;
  o->input_on_host = 0;
  o->column_scales = 1;
  o->fp8_copy = 0;
  o->stream = nullptr;
}

void glm_ca_opts_default(glm_ca_opts *o) {
  if (!o) return;
  o->gram_dtype = -1;
  o->gemv_dtype = -1;
  o->recurrence_f64 = -1;
  o->kahan = 1;
  o->first_iter = 0;
  o->problem = 0;
  o->use_graph = 1;
  o->cluster = 0;
  o->chunk_outer = 0;
  o->gram_impl = 0;
  o->timing = 0;
  o->accumulate = GLM_F32;
  o->state_dtype = GLM_F32;
  o->chain_impl = 0;
  o->wait_probe_cycles = 0;
}

void glm_debug_fail_alloc(int64_t after) { g_alloc_countdown.store(after < 0 ? -1 : after); }

int glm_create_ex(const void *A, const float *y, int64_t m, int64_t n, int loss, int dtype,
                  const glm_create_opts *opts, glm_handle *out) {
  g_last_error.clear();
  if (!out) return set_error(GLM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!A || !y) return set_error(GLM_EINVAL, "A or y is NULL");
  if (m < 1 || m >= (1ll << 31)) return set_error(GLM_EINVAL, "m must be in [1, 2^31)");
  if (n < 1 || n > 65536) return set_error(GLM_EINVAL, "n must be in [1, 65536]");
  if (loss != GLM_LOGISTIC && loss != GLM_LSQ && loss != GLM_POISSON)
    return set_error(GLM_EINVAL, "unknown loss");
  if (dtype != GLM_F32 && dtype != GLM_BF16 && dtype != GLM_F16)
    return set_error(GLM_EINVAL, "storage dtype must be GLM_F32, GLM_BF16 or GLM_F16");
  glm_create_opts d;
  glm_create_opts_default(&d);
  if (!opts) opts = &d;
  if (opts->input_dtype != GLM_F32 && opts->input_dtype != GLM_BF16)
    return set_error(GLM_EINVAL, "input_dtype must be GLM_F32 or GLM_BF16");
  Handle *h = new Handle();
  h->m = m;
  h->n = n;
  h->loss = loss;
  h->dtype = dtype;
  h->lda = round_up(n, 8);
  int rc = GLM_OK;
  // create-time temporaries: the input uploaded from the host, the column sums
  void *tmpA = nullptr;
  float *tmpy = nullptr;
  double *acc = nullptr;
  auto cleanup_tmp = [&]() {
    if (tmpA) cudaFree(tmpA);
    if (tmpy) cudaFree(tmpy);
    if (acc) cudaFree(acc);
    tmpA = nullptr;
    tmpy = nullptr;
    acc = nullptr;
  };
  auto fail = [&](int code) {
    cleanup_tmp();
    free_handle(h);
    return code;
  };
#define CK(expr)                                                               \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess) return fail(cuda_error(e_, #expr));                 \
  } while (0)
  if (opts->stream) {
    h->stream = static_cast<cudaStream_t>(opts->stream);
  } else {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  cudaStream_t st = h->stream;
  const int ieb = opts->input_dtype == GLM_BF16 ? 2 : 4;
  const int eb = elem_bytes(dtype);
  CK(dev_malloc(&h->A, (size_t)m * h->lda * eb));
  CK(dev_malloc((void **)&h->y, (size_t)m * 4));
  CK(dev_malloc((void **)&h->dflag, 16));
  CK(cudaMemsetAsync(h->dflag, 0, 16, st));
  CK(dev_malloc((void **)&h->loss_partials, (size_t)loss_partials_needed() * 8));
  CK(dev_malloc((void **)&h->loss_out, 8));
  // input in device memory (temporary upload when it lives on the host)
  const void *src = A;
  const float *ysrc = y;
  const bool host_in = opts->input_on_host || !is_device_ptr(A);
  if (host_in) {
    CK(dev_malloc(&tmpA, (size_t)m * n * ieb));
    CK(cudaMemcpyAsync(tmpA, A, (size_t)m * n * ieb, cudaMemcpyHostToDevice, st));
    src = tmpA;
  }
  if (opts->input_on_host || !is_device_ptr(y)) {
    CK(dev_malloc((void **)&tmpy, (size_t)m * 4));
    CK(cudaMemcpyAsync(tmpy, y, (size_t)m * 4, cudaMemcpyHostToDevice, st));
    ysrc = tmpy;
  }
  CK(cudaMemcpyAsync(h->y, ysrc, (size_t)m * 4, cudaMemcpyDeviceToDevice, st));
  // per-column power-of-two scales (BF16 / F16 storage)
  if (dtype != GLM_F32 && opts->column_scales) {
    CK(dev_malloc((void **)&acc, (size_t)n * 8));
    CK(cudaMemsetAsync(acc, 0, (size_t)n * 8, st));
    rc = launch_colsumsq(src, opts->input_dtype, m, n, acc, st);
    if (rc != GLM_OK) return fail(rc);
    std::vector<double> hs(n);
    CK(cudaMemcpyAsync(hs.data(), acc, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(acc);
    acc = nullptr;
    std::vector<float> kappa(h->lda, 1.0f);
    for (int64_t k = 0; k < n; ++k) {
      const double rms = sqrt(hs[k] / (double)m);
      kappa[k] = rms > 0.0 ? (float)ldexp(1.0, (int)nearbyint(log2(rms))) : 1.0f;
    }
    CK(dev_malloc((void **)&h->colscale, (size_t)h->lda * 4));
    CK(cudaMemcpyAsync(h->colscale, kappa.data(), (size_t)h->lda * 4, cudaMemcpyHostToDevice,
                       st));
    CK(cudaStreamSynchronize(st));
  }
  rc = launch_create_convert(h, src, opts->input_dtype, 0, m, st);
  if (rc != GLM_OK) return fail(rc);
  if (opts->fp8_copy) {
    h->lda8 = round_up(n, 16);
    CK(dev_malloc((void **)&h->A8, (size_t)m * h->lda8));
    CK(dev_malloc((void **)&h->rowscale8, (size_t)m * 4));
    rc = launch_fp8_copy(h, src, opts->input_dtype, 0, m, st);
    if (rc != GLM_OK) return fail(rc);
  }
  rc = launch_check_labels(h->y, m, loss, h->dflag, st);
  if (rc != GLM_OK) return fail(rc);
  unsigned flag = 0;
  CK(cudaMemcpyAsync(&flag, h->dflag, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cleanup_tmp();
  if (flag & FLAG_BAD_LABEL)
    return fail(set_error(GLM_EINVAL, loss == GLM_LOGISTIC
                                          ? "logistic labels must be exactly -1 or +1"
                                          : loss == GLM_POISSON
                                                ? "Poisson labels must be finite and >= 0"
                                                : "labels must be finite"));
#undef CK
  *out = reinterpret_cast<glm_handle>(h);
  return GLM_OK;
}

int glm_create(const float *A, const float *y, int64_t m, int64_t n, int loss, int dtype,
               glm_handle *out) {
  return glm_create_ex(A, y, m, n, loss, dtype, nullptr, out);
}

int glm_destroy(glm_handle hh) {
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h) return GLM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_handle(h);
  return GLM_OK;
}

int glm_shape(glm_handle hh, int64_t *m, int64_t *n) {
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h) return set_error(GLM_EINVAL, "null handle");
  if (m) *m = h->m;
  if (n) *n = h->n;
  return GLM_OK;
}

void *glm_stream(glm_handle hh) {
  Handle *h = reinterpret_cast<Handle *>(hh);
  return h ? (void *)h->stream : nullptr;
}

int glm_sync(glm_handle hh) {
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h) return set_error(GLM_EINVAL, "null handle");
  unsigned flag = 0;
  GLM_CUDA_TRY(cudaMemcpyAsync(&flag, h->dflag, 4, cudaMemcpyDeviceToHost, h->stream));
  GLM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (flag) {
    GLM_CUDA_TRY(cudaMemsetAsync(h->dflag, 0, 4, h->stream));
    GLM_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (flag & FLAG_BOUNDS)
      return set_error(GLM_EBOUNDS, "a kernel index fell outside its buffer (checked build)");
    if (flag & FLAG_TIMEOUT) return set_error(GLM_ETIMEOUT, "a bounded device wait gave up");
    return set_error(GLM_ENONFINITE, "a run produced a non-finite margin, residual or iterate");
  }
  return GLM_OK;
}

int glm_sgd_run_ex(glm_handle hh, int64_t b, float eta, float lambda, int64_t iters,
                   uint64_t seed, float *x, const glm_ca_opts *opts) {
  g_last_error.clear();
  return run_common(reinterpret_cast<Handle *>(hh), 1, b, eta, lambda, iters, seed, x, opts,
                    true);
}

int glm_sgd_run(glm_handle h, int64_t b, float eta, float lambda, int64_t iters, uint64_t seed,
                float *x) {
  return glm_sgd_run_ex(h, b, eta, lambda, iters, seed, x, nullptr);
}

int glm_ca_sgd_run_ex(glm_handle hh, int s, int64_t b, float eta, float lambda, int64_t iters,
                      uint64_t seed, float *x, const glm_ca_opts *opts) {
  g_last_error.clear();
  if (opts && (opts->accumulate != GLM_F32 || opts->state_dtype != GLM_F32)) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return set_error(GLM_EINVAL, "null handle");
    return run_recipe(h, s, b, eta, lambda, iters, seed, x, opts);
  }
  return run_common(reinterpret_cast<Handle *>(hh), s, b, eta, lambda, iters, seed, x, opts,
                    false);
}

int glm_ca_sgd_run(glm_handle h, int s, int64_t b, float eta, float lambda, int64_t iters,
                   uint64_t seed, float *x) {
  return glm_ca_sgd_run_ex(h, s, b, eta, lambda, iters, seed, x, nullptr);
}

int glm_sgd_lowp_run(glm_handle hh, int64_t b, float eta, float lambda, int64_t iters,
                     uint64_t seed, float *x, int accumulate, int64_t first_iter) {
  g_last_error.clear();
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h) return set_error(GLM_EINVAL, "null handle");
  if (!x) return set_error(GLM_EINVAL, "x is NULL");
  if (h->dtype != GLM_BF16 && h->dtype != GLM_F16)
    return set_error(GLM_EINVAL, "low-precision SGD needs BF16 or FP16 storage");
  if (accumulate != GLM_F32 && !(accumulate == GLM_F16 && h->dtype == GLM_F16))
    return set_error(GLM_EINVAL, "accumulate must be GLM_F32, or GLM_F16 with FP16 storage");
  if (b < 1 || b > 1024) return set_error(GLM_EINVAL, "b must be in [1, 1024]");
  if (iters < 0) return set_error(GLM_EINVAL, "iters must be >= 0");
  if (first_iter < 0) return set_error(GLM_EINVAL, "first_iter must be >= 0");
  if (!(eta > 0.f) || !isfinite(eta)) return set_error(GLM_EINVAL, "eta must be finite and > 0");
  if (!(lambda >= 0.f) || !isfinite(lambda)) return set_error(GLM_EINVAL, "lambda must be >= 0");
  const double c = 1.0 - (double)eta * (double)lambda;
  if (!(c > 0.0)) return set_error(GLM_EINVAL, "eta * lambda must be < 1");
  if (!lowp_fits(h->n, (int)b))
    return set_error(GLM_EUNSUPPORTED, "n too large for the on-chip low-precision state");
  if (iters == 0) return GLM_OK;
  LowpArgs a = {};
  a.A = h->A;
  a.lda = h->lda;
  a.colscale = h->colscale;
  a.y = h->y;
  a.m = h->m;
  a.n = h->n;
  a.b = (int)b;
  a.loss = h->loss;
  a.seed = seed;
  a.problem = 0;
  a.q0 = (uint64_t)first_iter * (uint64_t)b;
  a.iters = iters;
  a.alpha = (float)((double)eta / (double)b);
  a.c = (float)c;
  a.x = x;
  a.flag = h->dflag;
  return launch_sgd_lowp(a, h->dtype, accumulate == GLM_F16 ? 1 : 0, h->stream);
}

int glm_ca_plan(glm_handle hh, int s, int64_t b, float eta, float lambda, int64_t iters,
                const glm_ca_opts *opts, glm_run_plan *out) {
  g_last_error.clear();
  if (!out) return set_error(GLM_EINVAL, "out is NULL");
  float dummy = 0.f;
  RunPlan p;
  GLM_TRY(resolve(reinterpret_cast<Handle *>(hh), s, b, eta, lambda, iters, 0, &dummy, opts,
                  false, p));
  out->chunk_outer = p.chunk;
  out->chunks = iters > 0 ? p.chunks : 0;
  out->launches = iters > 0 ? p.launches : 0;
  out->cluster = p.cluster;
  out->gram_impl = p.gram_impl;
  out->gram_dtype = p.gram_dt;
  out->gemv_dtype = p.gemv_dt;
  out->recurrence_f64 = p.rec64;
  out->chain_impl = p.chain_impl;
  return GLM_OK;
}

int glm_kernel_times(glm_handle hh, double *ms, int64_t *launches) {
  g_last_error.clear();
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h || !ms || !launches) return set_error(GLM_EINVAL, "null argument");
  if (!h->tev_valid) return set_error(GLM_EINVAL, "no run with opts.timing = 1 yet");
  GLM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < 3; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
    if (!(h->tev_valid & (1 << k))) continue;
    for (int64_t c = 0; c < h->tev_chunks; ++c) {
      float t = 0.f;
      GLM_CUDA_TRY(cudaEventElapsedTime(&t, h->tev[(size_t)(c * 6 + k * 2)],
                                        h->tev[(size_t)(c * 6 + k * 2 + 1)]));
      ms[k] += t;
      launches[k] += 1;
    }
  }
  return GLM_OK;
}

int glm_loss(glm_handle hh, const float *x, float lambda, double *out) {
  g_last_error.clear();
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h || !x || !out) return set_error(GLM_EINVAL, "null argument");
  if (!(lambda >= 0.f)) return set_error(GLM_EINVAL, "lambda must be >= 0");
  GLM_TRY(launch_loss(h, x, lambda, h->stream));
  GLM_CUDA_TRY(cudaMemcpyAsync(out, h->loss_out, 8, cudaMemcpyDeviceToHost, h->stream));
  GLM_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return GLM_OK;
}

int glm_sample_indices(uint64_t seed, uint32_t problem, int64_t first_draw, int64_t count,
                       int64_t m, int32_t *out) {
  g_last_error.clear();
  if (count < 0 || first_draw < 0) return set_error(GLM_EINVAL, "count/first_draw must be >= 0");
  if (m < 1 || m >= (1ll << 31)) return set_error(GLM_EINVAL, "m must be in [1, 2^31)");
  if (count == 0) return GLM_OK;
  if (!out) return set_error(GLM_EINVAL, "out is NULL");
  if (is_device_ptr(out)) {
    GLM_TRY(launch_sample(seed, problem, first_draw, count, m, out, 0));
    GLM_CUDA_TRY(cudaStreamSynchronize(0));
    return GLM_OK;
  }
  int32_t *d = nullptr;
  GLM_CUDA_TRY(dev_malloc((void **)&d, (size_t)count * 4));
  int rc = launch_sample(seed, problem, first_draw, count, m, d, 0);
  if (rc == GLM_OK) {
    cudaError_t e = cudaMemcpy(out, d, (size_t)count * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpy(indices)");
  }
  cudaFree(d);
  return rc;
}

int glm_storage_layout(glm_handle hh, int *dtype, int64_t *lda, int64_t *lda8) {
  g_last_error.clear();
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h) return set_error(GLM_EINVAL, "null handle");
  if (dtype) *dtype = h->dtype;
  if (lda) *lda = h->lda;
  if (lda8) *lda8 = h->A8 ? h->lda8 : 0;
  return GLM_OK;
}

int glm_storage_read(glm_handle hh, int64_t row0, int64_t rows, void *A_out,
                     float *colscale_out, uint8_t *fp8_out, float *rowscale_out) {
  g_last_error.clear();
  Handle *h = reinterpret_cast<Handle *>(hh);
  if (!h) return set_error(GLM_EINVAL, "null handle");
  if (row0 < 0 || rows < 0 || row0 + rows > h->m)
    return set_error(GLM_EINVAL, "rows [row0, row0 + rows) must lie in [0, m)");
  if ((fp8_out || rowscale_out) && !h->A8)
    return set_error(GLM_EINVAL, "the handle keeps no FP8 copy (create it with fp8_copy = 1)");
  for (const void *p : {(const void *)A_out, (const void *)colscale_out, (const void *)fp8_out,
                        (const void *)rowscale_out})
    if (p && is_device_ptr(p)) return set_error(GLM_EINVAL, "outputs must be host memory");
  cudaStream_t st = h->stream;
  const int eb = elem_bytes(h->dtype);
  if (A_out && rows > 0)
    GLM_CUDA_TRY(cudaMemcpyAsync(A_out, static_cast<const char *>(h->A) + row0 * h->lda * eb,
                                 (size_t)rows * h->lda * eb, cudaMemcpyDeviceToHost, st));
  if (colscale_out) {
    if (h->colscale)
      GLM_CUDA_TRY(cudaMemcpyAsync(colscale_out, h->colscale, (size_t)h->n * 4,
                                   cudaMemcpyDeviceToHost, st));
    else
      for (int64_t k = 0; k < h->n; ++k) colscale_out[k] = 1.0f;
  }
  if (fp8_out && rows > 0)
    GLM_CUDA_TRY(cudaMemcpyAsync(fp8_out, h->A8 + row0 * h->lda8, (size_t)rows * h->lda8,
                                 cudaMemcpyDeviceToHost, st));
  if (rowscale_out && rows > 0)
    GLM_CUDA_TRY(cudaMemcpyAsync(rowscale_out, h->rowscale8 + row0, (size_t)rows * 4,
                                 cudaMemcpyDeviceToHost, st));
  GLM_CUDA_TRY(cudaStreamSynchronize(st));
  return GLM_OK;
}

int glm_gram_lower(const void *Y, int dtype, int64_t nouter, int s, int64_t b, int64_t n,
                   int64_t ld, const float *row_scale, float *G, int impl, void *stream) {
  g_last_error.clear();
  if (!Y || !G) return set_error(GLM_EINVAL, "null argument");
  if (nouter < 1 || s < 2 || b < 1 || n < 1 || ld < n || ld % 8)
    return set_error(GLM_EINVAL, "bad Gram shape (need nouter>=1, s>=2, b>=1, n<=ld, ld%8==0)");
  if (dtype != GLM_F32 && dtype != GLM_TF32 && dtype != GLM_BF16 && dtype != GLM_F16 &&
      dtype != GLM_E4M3)
    return set_error(GLM_EINVAL, "bad Gram operand type");
  if (dtype == GLM_E4M3 && (!row_scale || ld % 16))
    return set_error(GLM_EINVAL, "E4M3 Gram needs row scales and ld % 16 == 0");
  GramArgs a;
  a.Y = Y;
  a.dt = dtype;
  a.ld = ld;
  a.rs = dtype == GLM_E4M3 ? row_scale : nullptr;
  a.nouter = nouter;
  a.rows = nouter * s * b;
  a.s = s;
  a.b = b;
  a.n = n;
  a.G = G;
  a.flag = nullptr;
  a.probe = 0;
  a.tile_n = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (impl == 0) impl = gram_tc_supported(dtype, ld) ? 2 : 1;
  if (impl == 2) {
    if (!gram_tc_supported(dtype, ld))
      return set_error(GLM_EUNSUPPORTED, "tcgen05 Gram: unsupported type or ld % 64 != 0");
    return launch_gram_tc(a, st);
  }
  if (impl == 3) {
    if (dtype != GLM_F16) return set_error(GLM_EINVAL, "impl 3 (FP16 accumulation) needs GLM_F16");
    return launch_gram_simt_f16acc(a, st);
  }
  if (impl == 4) {
    if (dtype != GLM_F16) return set_error(GLM_EINVAL, "impl 4 (FP16 accumulation) needs GLM_F16");
    if (!gram_tc_supported(dtype, ld))
      return set_error(GLM_EUNSUPPORTED, "tcgen05 Gram: ld % 64 != 0");
    return launch_gram_tc_f16acc(a, st);
  }
  if (impl != 1) return set_error(GLM_EINVAL, "impl must be 0, 1, 2, 3 or 4");
  return launch_gram_simt(a, st);
}

// ---- batched fits: implemented in glm_batch.cu -----------------------------

}  // extern "C"
