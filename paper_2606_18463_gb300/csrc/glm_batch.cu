// glm_batch.cu -- batched fits (glm_batch_*): many independent problems of
// uneven m, n and lambda, each fit with CA-SGD (paper Algorithm 1), sharing
// the device in one run.
//
// Storage: one dataset handle per problem, made by the same path as
// glm_create_ex (converted storage with per-column scales, labels, loss).
// A run proceeds in rounds of K outer steps of every problem:
//   1. gather: one launch over all problems of the round;
//   2. Gram: one launch per group of problems sharing (s, b, n, operand type),
//      their outer steps stacked (every step holds s b rows, zero-padded);
//   3. chain: one persistent launch over a device work queue (longest first).
// All rounds of a run are captured once as a CUDA graph and replayed; the
// per-problem table lives in device memory, so new iterate pointers only
// rewrite the table.
//
// Autotuner: by default it chooses what leaves the exact-arithmetic iterate
// unchanged -- the s-step length (CA-SGD equals SGD for every s) and the Gram
// kernel and tile -- and never the mini-batch b (part of the problem).  The
// Gram operand type is chosen only under a caller bound on Theorem 1's
// hypothesis figure tau_G (glm_batch_opts.tau_bound), estimated from sampled
// rows, so that no precision is traded without the caller's consent.  For
// every n among the problems left to it, it times one round of each admitted
// candidate on up to 32 of those problems (scratch iterates) and keeps the
// fastest in samples/s (see autotune() below).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "glm_internal.cuh"

namespace glm {
namespace {

constexpr int64_t kRoundBudget = 4ll << 30;    // bytes of round buffers (HBM is plentiful)
constexpr int kMaxBatchN = 16384;              // iterate slice in shared memory

bool dev_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct Prob {
  glm_handle h = nullptr;
  int64_t m = 0, n = 0, b = 1, iters = 0;
  int loss = GLM_LOGISTIC;
  float lambda = 0.f, eta = 0.f;
  uint64_t seed = 0;
  int s = 0;        // chosen s-step length
  int tuned = 0;    // 1: s chosen by the autotuner
  int gk = 0;       // Gram kernel: 0 automatic, 1 SIMT, 2 tcgen05 128 x 128,
                    // 3 tcgen05 128 x 256 (chosen with s by the autotuner)
  double tau = 0.0; // estimated tau_G at the chosen (s, Gram type); 0 if not estimated
};

struct Group {      // problems of one round sharing (s, b, n, Gram kernel): one Gram launch
  int s;
  int64_t b, n, ld, nouter;
  void *Y;
  float *G;
  int gk;
};

struct Plan {
  int64_t K = 1;                       // outer steps per round
  int rounds = 0;
  std::vector<BatchItem> items;        // all rounds, round r at [begin[r], begin[r+1])
  std::vector<int> begin;
  std::vector<int> order;              // per item: position in its round, longest first
  std::vector<std::vector<Group>> groups;
  std::vector<int64_t> max_rows;       // per round: most rows of one item
  size_t y_bytes = 0, lab_bytes = 0, g_bytes = 0;
  int max_n = 8, max_sb = 1, max_s = 1, rec64 = 0;
};

}  // namespace

struct Batch {
  int P = 0;
  int dtype = GLM_BF16;   // storage
  int gdt = GLM_BF16;     // Gram / GEMV operand type (one per batch)
  int gram_impl = 0;      // 0 auto, 1 SIMT, 2 tcgen05
  std::vector<Prob> pr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevBuf ybuf, labbuf, gbuf, itembuf, orderbuf, queuebuf;
  Plan plan;
  bool planned = false;
  cudaGraphExec_t graph = nullptr;
  std::vector<float *> xs;  // iterate pointers the table holds
  unsigned *bflag = nullptr;  // [0]: the Gram launches' flag word, [1]: the
                              // tuner's scratch runs' flag word (every item)
  int64_t probe = 0;          // glm_batch_opts.wait_probe_cycles
  double tau_bound = 0.0;     // glm_batch_opts.tau_bound (0: Gram type not tuned)
  bool gdt_free = false;      // no descriptor fixed the Gram type
};

namespace {

// row pitch of the gathered operand rows: 64 elements for every batched
// operand type (the FP8 Gram is not offered in batches)
int64_t ld_for(int64_t n) { return round_up(n, 64); }

// Plan a run of the problems `sel` (indices) with their s, iterating
// `iters[k]` SGD-equivalent iterations each.
void make_plan(const Batch &B, const std::vector<int> &sel, const std::vector<int64_t> &iters,
               Plan &pl) {
  pl = Plan();
  const int eb = elem_bytes(B.gdt);
  int64_t per_outer = 0, hmax = 0;
  for (size_t k = 0; k < sel.size(); ++k) {
    const Prob &p = B.pr[sel[k]];
    const int64_t sb = (int64_t)p.s * p.b;
    per_outer += sb * (ld_for(p.n) * eb + 4) + gram_size(p.s, p.b) * 4;
    hmax = std::max<int64_t>(hmax, (iters[k] + p.s - 1) / p.s);
    pl.max_n = std::max<int>(pl.max_n, (int)p.n);
    pl.max_sb = std::max<int>(pl.max_sb, (int)sb);
    pl.max_s = std::max(pl.max_s, p.s);
    if (p.s >= 32) pl.rec64 = 1;
  }
  pl.K = std::max<int64_t>(1, kRoundBudget / std::max<int64_t>(per_outer, 1));
  pl.K = std::min<int64_t>(pl.K, std::max<int64_t>(hmax, 1));
  pl.rounds = (int)((hmax + pl.K - 1) / pl.K);
  for (int r = 0; r < pl.rounds; ++r) {
    pl.begin.push_back((int)pl.items.size());
    // group the round's problems by (s, b, n, Gram kernel); each group is contiguous
    std::map<std::tuple<int, int64_t, int64_t, int>, std::vector<std::pair<int, int64_t>>> grp;
    for (size_t k = 0; k < sel.size(); ++k) {
      const Prob &p = B.pr[sel[k]];
      const int64_t H = (iters[k] + p.s - 1) / p.s;
      const int64_t h0 = (int64_t)r * pl.K;
      if (h0 >= H) continue;
      grp[std::make_tuple(p.s, p.b, p.n, p.gk)].push_back({(int)k, std::min<int64_t>(pl.K, H - h0)});
    }
    size_t yoff = 0, loff = 0, goff = 0;
    std::vector<Group> gl;
    int64_t mrows = 0;
    for (auto &kv : grp) {
      const int s = std::get<0>(kv.first);
      const int64_t b = std::get<1>(kv.first), n = std::get<2>(kv.first);
      const int64_t sb = s * b, ld = ld_for(n);
      Group g{s, b, n, ld, 0, reinterpret_cast<void *>(yoff), reinterpret_cast<float *>(goff),
              std::get<3>(kv.first)};
      for (auto &e : kv.second) {
        const int k = e.first;
        const int64_t nout = e.second;
        const Prob &p = B.pr[sel[k]];
        const Handle *h = reinterpret_cast<const Handle *>(p.h);
        const int64_t h0 = (int64_t)r * pl.K;
        const int64_t it0 = h0 * s, it1 = std::min<int64_t>(iters[k], (h0 + nout) * s);
        BatchItem it;
        memset(&it, 0, sizeof(it));
        it.A = h->A; it.lda = h->lda; it.colscale = h->colscale; it.y = h->y;
        it.m = h->m; it.n = (int)h->n; it.a_dt = h->dtype;
        it.seed = p.seed; it.problem = (uint64_t)sel[k]; it.q0 = (uint64_t)(it0 * b);
        it.nouter = (int)nout; it.s = s; it.b = (int)b;
        it.s_last = (int)(it1 - (h0 + nout - 1) * s);
        it.Y = reinterpret_cast<void *>(yoff); it.y_dt = B.gdt; it.ldy = ld;
        it.lab = reinterpret_cast<float *>(loff);
        it.G = reinterpret_cast<float *>(goff);
        it.loss = p.loss; it.kahan = 1;
        it.alpha = (float)((double)p.eta / (double)b);
        it.c = 1.0 - (double)p.eta * (double)p.lambda;
        it.flag = h->dflag;
        pl.items.push_back(it);
        yoff += (size_t)(nout * sb * ld * elem_bytes(B.gdt));
        loff += (size_t)(nout * sb * 4);
        goff += (size_t)(nout * gram_size(s, b) * 4);
        g.nouter += nout;
        mrows = std::max<int64_t>(mrows, nout * sb);
      }
      gl.push_back(g);
    }
    pl.groups.push_back(gl);
    pl.max_rows.push_back(mrows);
    pl.y_bytes = std::max(pl.y_bytes, yoff);
    pl.lab_bytes = std::max(pl.lab_bytes, loff);
    pl.g_bytes = std::max(pl.g_bytes, goff);
    // longest first: work ~ outer steps x rows x (n + s b)
    const int b0 = pl.begin.back(), cnt = (int)pl.items.size() - b0;
    std::vector<int> ord(cnt);
    for (int i = 0; i < cnt; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      const BatchItem &a = pl.items[b0 + x], &c = pl.items[b0 + y];
      const double wa = (double)a.nouter * a.s * a.b * (a.n + a.s * a.b);
      const double wc = (double)c.nouter * c.s * c.b * (c.n + c.s * c.b);
      return wa > wc;
    });
    pl.order.insert(pl.order.end(), ord.begin(), ord.end());
  }
  pl.begin.push_back((int)pl.items.size());
}

// Device table of a plan: offsets become buffer addresses; x[k] is the
// iterate of the k-th selected problem.
int bind(Batch &B, Plan &pl, const std::vector<float *> &x, std::vector<int> *kmap,
         std::vector<BatchItem> &out) {
  GLM_TRY(B.ybuf.ensure(std::max<size_t>(pl.y_bytes, 16)));
  GLM_TRY(B.labbuf.ensure(std::max<size_t>(pl.lab_bytes, 16)));
  GLM_TRY(B.gbuf.ensure(std::max<size_t>(pl.g_bytes, 16)));
  GLM_TRY(B.itembuf.ensure(std::max<size_t>(pl.items.size() * sizeof(BatchItem), 16)));
  GLM_TRY(B.orderbuf.ensure(std::max<size_t>(pl.order.size() * sizeof(int), 16)));
  GLM_TRY(B.queuebuf.ensure(std::max<size_t>((size_t)pl.rounds * sizeof(int), 16)));
  char *yb = static_cast<char *>(B.ybuf.ptr), *gb = static_cast<char *>(B.gbuf.ptr);
  char *lb = static_cast<char *>(B.labbuf.ptr);
  out = pl.items;
  for (auto &it : out) {
    it.Y = yb + reinterpret_cast<size_t>(it.Y);
    it.lab = reinterpret_cast<float *>(lb + reinterpret_cast<size_t>(it.lab));
    it.G = reinterpret_cast<float *>(gb + reinterpret_cast<size_t>(it.G));
    it.x = x[(size_t)(*kmap)[it.problem]];
  }
  return GLM_OK;
}

int upload(Batch &B, const Plan &pl, const std::vector<BatchItem> &items) {
  if (!items.empty())
    GLM_CUDA_TRY(cudaMemcpyAsync(B.itembuf.ptr, items.data(), items.size() * sizeof(BatchItem),
                                 cudaMemcpyHostToDevice, B.stream));
  if (!pl.order.empty())
    GLM_CUDA_TRY(cudaMemcpyAsync(B.orderbuf.ptr, pl.order.data(), pl.order.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, B.stream));
  GLM_CUDA_TRY(cudaStreamSynchronize(B.stream));
  return GLM_OK;
}

// Every round: gather, Gram per group, persistent chain.
int enqueue(Batch &B, const Plan &pl, cudaStream_t st) {
  BatchItem *items = static_cast<BatchItem *>(B.itembuf.ptr);
  int *order = static_cast<int *>(B.orderbuf.ptr);
  int *queue = static_cast<int *>(B.queuebuf.ptr);
  char *yb = static_cast<char *>(B.ybuf.ptr), *gb = static_cast<char *>(B.gbuf.ptr);
  GLM_CUDA_TRY(cudaMemsetAsync(queue, 0, (size_t)pl.rounds * sizeof(int), st));
  for (int r = 0; r < pl.rounds; ++r) {
    const int b0 = pl.begin[r], cnt = pl.begin[r + 1] - b0;
    if (cnt <= 0) continue;
    GLM_TRY(launch_gather_batch(items + b0, cnt, pl.max_rows[r], st, B.dtype));
    for (const Group &g : pl.groups[r]) {
      if (g.s < 2) continue;
      GramArgs ga;
      memset(&ga, 0, sizeof(ga));
      ga.Y = yb + reinterpret_cast<size_t>(g.Y);
      ga.dt = B.gdt;
      ga.ld = g.ld;
      ga.nouter = g.nouter;
      ga.rows = g.nouter * g.s * g.b;
      ga.s = g.s;
      ga.b = g.b;
      ga.n = g.n;
      ga.G = reinterpret_cast<float *>(gb + reinterpret_cast<size_t>(g.G));
      ga.flag = B.bflag;
      ga.probe = B.probe;
      const bool tc_ok = gram_tc_supported(B.gdt, g.ld);
      const bool tc = g.gk >= 2 ? tc_ok : (g.gk == 0 && tc_ok);
      ga.tile_n = g.gk == 2 ? 128 : (g.gk == 3 ? 256 : 0);
      if (tc) GLM_TRY(launch_gram_tc(ga, st));
      else GLM_TRY(launch_gram_simt(ga, st));
    }
    GLM_TRY(launch_chain_batch(items + b0, order + b0, cnt, queue + r, B.gdt, pl.rec64, pl.max_n,
                               pl.max_sb, pl.max_s, st));
  }
  return GLM_OK;
}

// Time one round of candidate s for the problems `sel` (scratch iterates).
int time_candidate(Batch &B, const std::vector<int> &sel, int s, int gk, float *xscratch,
                   double &ms, double &samples) {
  std::vector<int> keep(sel.size()), keepk(sel.size());
  std::vector<int64_t> iters(sel.size());
  std::vector<float *> xp(sel.size());
  std::vector<int> kmap(B.P, -1);
  samples = 0.0;
  int64_t xo = 0;
  for (size_t k = 0; k < sel.size(); ++k) {
    Prob &p = B.pr[sel[k]];
    keep[k] = p.s;
    keepk[k] = p.gk;
    p.s = s;
    p.gk = gk;
    iters[k] = std::min<int64_t>(p.iters, (int64_t)8 * s);  // eight outer steps
    samples += (double)iters[k] * (double)p.b;
    xp[k] = xscratch + xo;
    xo += round_up(p.n, 8);
    kmap[sel[k]] = (int)k;
  }
  Plan pl;
  make_plan(B, sel, iters, pl);
  std::vector<BatchItem> items;
  int rc = bind(B, pl, xp, &kmap, items);
  // scratch runs raise their flags in a word of their own, never in a
  // problem's flag word (which a user run may have set)
  for (auto &it : items) it.flag = B.bflag + 1;
  if (rc == GLM_OK) rc = upload(B, pl, items);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == GLM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = set_error(GLM_ECUDA, "autotune: cudaEventCreate");
  for (int rep = 0; rep < 2 && rc == GLM_OK; ++rep) {  // warm-up, then timed
    if (rep == 1) cudaEventRecord(e0, B.stream);
    rc = enqueue(B, pl, B.stream);
    if (rep == 1) cudaEventRecord(e1, B.stream);
  }
  if (rc == GLM_OK) {
    float t = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      rc = set_error(GLM_ECUDA, "autotune: event timing");
    ms = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (size_t k = 0; k < sel.size(); ++k) {
    B.pr[sel[k]].s = keep[k];
    B.pr[sel[k]].gk = keepk[k];
  }
  return rc;
}

// ---- Theorem 1 prior (paper Sec. 5.2) for the Gram operand type ----------
// tau_G = K_s L_sigma alpha (2 u_A + gamma_G) ||H_L||_2 is the theorem's
// hypothesis figure for the Gram slot: the local budget holds for tau_G <=
// 1/2, and it scales the Gram term E_G.  From one gathered outer step of a
// problem (FP32 values of its stored rows) the tuner bounds
//   ||H_L||_2 <= sqrt(||H_L||_1 ||H_L||_inf),  H_L = strictly block-lower |Y||Y|^T,
// both norms from prefix sums of |rows| over blocks (O(s b n)), and
//   K_s = ||(I - L alpha |G_L|)^-1||_2 <= 1 / (1 - L alpha ||H_L||_2).
double hl_norm_bound(const std::vector<float> &Y, int64_t n, int s, int64_t b) {
  std::vector<double> pre(n, 0.0), suf(n, 0.0), absr(n);
  double ninf = 0.0, none = 0.0;
  // infinity norm: row r of block j against the sum of |rows| of blocks < j
  for (int j = 0; j < s; ++j) {
    for (int64_t l = 0; l < b; ++l) {
      const float *y = Y.data() + ((int64_t)j * b + l) * n;
      double acc = 0.0;
      for (int64_t c = 0; c < n; ++c) acc += std::fabs((double)y[c]) * pre[c];
      ninf = std::max(ninf, acc);
    }
    for (int64_t l = 0; l < b; ++l) {
      const float *y = Y.data() + ((int64_t)j * b + l) * n;
      for (int64_t c = 0; c < n; ++c) pre[c] += std::fabs((double)y[c]);
    }
  }
  // one norm: column (row of Y) c of block i against |rows| of blocks > i
  for (int i = s - 1; i >= 0; --i) {
    for (int64_t l = 0; l < b; ++l) {
      const float *y = Y.data() + ((int64_t)i * b + l) * n;
      double acc = 0.0;
      for (int64_t c = 0; c < n; ++c) acc += std::fabs((double)y[c]) * suf[c];
      none = std::max(none, acc);
    }
    for (int64_t l = 0; l < b; ++l) {
      const float *y = Y.data() + ((int64_t)i * b + l) * n;
      for (int64_t c = 0; c < n; ++c) suf[c] += std::fabs((double)y[c]);
    }
  }
  return std::sqrt(ninf * none);
}

double unit_roundoff(int dt) {
  switch (dt) {
  case GLM_BF16: return std::ldexp(1.0, -8);
  case GLM_F16: case GLM_TF32: return std::ldexp(1.0, -11);
  }
  return 0.0;  // FP32 storage values are the data
}

// Rounding of stored values to Gram operands of type `gdt`: none when every
// stored value is representable (FP32 operands; TF32 holds BF16 and FP16).
double operand_roundoff(int gdt, int storage) {
  if (gdt == storage || gdt == GLM_F32) return 0.0;
  if (gdt == GLM_TF32 && (storage == GLM_BF16 || storage == GLM_F16)) return 0.0;
  return unit_roundoff(gdt);
}

double tau_g(double hl, double alpha, int loss, double u_A, double u_in, int64_t n) {
  if (loss == GLM_POISSON) return u_in > 0.0 ? INFINITY : 0.0;  // no Lipschitz bound
  const double L = loss == GLM_LOGISTIC ? 0.25 : 1.0;
  const double q = (double)n * std::ldexp(1.0, -24);
  const double gamma_G = 2.0 * u_in + q / (1.0 - q);
  const double a = L * alpha * hl;
  if (a >= 1.0) return INFINITY;
  return (1.0 / (1.0 - a)) * L * alpha * (2.0 * u_A + gamma_G) * hl;
}

// FP32 values of the stored rows of problem p's first outer step of `rows`
// rows (its own index stream), on the host.
int sample_rows(Batch &B, int p, int64_t rows, std::vector<float> &out) {
  const Handle *h = reinterpret_cast<const Handle *>(B.pr[p].h);
  const int64_t ld = round_up(h->n, 8);
  float *d = nullptr, *lab = nullptr;
  GLM_CUDA_TRY(dev_malloc((void **)&d, (size_t)rows * ld * 4));
  if (dev_malloc((void **)&lab, (size_t)round_up(rows, 4) * 4) != cudaSuccess) {
    cudaFree(d);
    return set_error(GLM_ENOMEM, "autotune: sample buffer");
  }
  GatherArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.A = h->A; ga.lda = h->lda; ga.a_dt = h->dtype; ga.colscale = h->colscale;
  ga.y = h->y; ga.m = h->m; ga.n = h->n; ga.rows = rows;
  ga.flag = h->dflag;
  ga.q0 = 0; ga.seed = B.pr[p].seed; ga.problem = (uint64_t)p;
  ga.out1 = d; ga.dt1 = GLM_F32; ga.ld1 = ld;
  ga.ylab = lab; ga.lab_sb = rows; ga.lab_sbp = round_up(rows, 4);
  int rc = launch_gather(ga, B.stream);
  std::vector<float> tmp((size_t)rows * ld);
  if (rc == GLM_OK && cudaMemcpyAsync(tmp.data(), d, tmp.size() * 4, cudaMemcpyDeviceToHost,
                                      B.stream) != cudaSuccess)
    rc = set_error(GLM_ECUDA, "autotune: sample copy");
  if (rc == GLM_OK && cudaStreamSynchronize(B.stream) != cudaSuccess)
    rc = set_error(GLM_ECUDA, "autotune: sample sync");
  cudaFree(d);
  cudaFree(lab);
  if (rc != GLM_OK) return rc;
  out.resize((size_t)rows * h->n);
  for (int64_t r = 0; r < rows; ++r)
    memcpy(out.data() + r * h->n, tmp.data() + r * ld, (size_t)h->n * 4);
  return GLM_OK;
}

// The autotuner.  For every n among the problems left to it (up to 32 of
// them timed, up to 4 sampled for the prior) and, under a caller bound on
// tau_G, for every admissible Gram operand type of the batch, it times one
// round of each candidate (s, Gram kernel) -- s in {1, 2, 4, 8, 16}; SIMT,
// tcgen05 128 x 128 or 128 x 256 tiles -- and keeps the fastest in samples
// per second.  With a bound, (s, type) pairs whose estimated tau_G exceeds it
// are not timed; s = 1 (no Gram) runs only on the storage type's operands, so
// a narrower type must have an admitted s > 1 for every n; and the type kept
// is the one with the shortest estimated run over all problems.
int autotune(Batch &B) {
  std::map<int64_t, std::vector<int>> by_n;  // problems left to the tuner, by n
  for (int p = 0; p < B.P; ++p)
    if (B.pr[p].tuned && B.pr[p].iters > 0) by_n[B.pr[p].n].push_back(p);
  if (by_n.empty()) return GLM_OK;
  float *xs = nullptr;
  size_t xcount = 0;
  for (auto &kv : by_n) xcount = std::max(xcount, std::min<size_t>(kv.second.size(), 32) *
                                                      (size_t)round_up(kv.first, 8));
  GLM_CUDA_TRY(dev_malloc((void **)&xs, xcount * 4));
  const int svals[5] = {1, 2, 4, 8, 16};
  // ||H_L|| bounds per (problem sampled, s): prefixes of one 16-step sample
  std::map<int, std::vector<double>> hl;  // problem -> bound for each s value
  int rc = GLM_OK;
  if (B.tau_bound > 0.0) {
    for (auto &kv : by_n) {
      for (size_t k = 0; k < kv.second.size() && k < 4 && rc == GLM_OK; ++k) {
        const int p = kv.second[k];
        // up to 16 outer-step blocks (64 M values at most): longer s is not admitted
        const int steps = (int)std::max<int64_t>(
            1, std::min<int64_t>(16, (64ll << 20) / (B.pr[p].b * B.pr[p].n)));
        std::vector<float> Y;
        rc = sample_rows(B, p, (int64_t)steps * B.pr[p].b, Y);
        if (rc != GLM_OK) break;
        std::vector<double> v;
        for (int si : svals)
          v.push_back(si <= steps ? hl_norm_bound(Y, B.pr[p].n, si, B.pr[p].b) : INFINITY);
        hl[p] = v;
      }
    }
  }
  std::vector<int> types = {B.gdt};
  if (B.tau_bound > 0.0 && B.gdt_free) {
    if (B.dtype == GLM_F32) types = {GLM_F32, GLM_TF32, GLM_F16, GLM_BF16};
    else types = {B.dtype};  // narrower storage: its own type is exact and fastest
  }
  struct Choice { int s = 1, gk = 0; double rate = -1.0; };
  double best_total = INFINITY;
  int best_type = B.gdt;
  std::map<int64_t, Choice> best_choice;
  for (int T : types) {
    if (rc != GLM_OK) break;
    B.gdt = T;
    const double u_in = operand_roundoff(T, B.dtype), u_A = unit_roundoff(B.dtype);
    // a type narrower than the storage is chosen for its Gram only: plain SGD
    // (s = 1, no Gram) keeps the storage type's exact operands, so such a type
    // needs an admitted s > 1 for every n
    const bool narrowed = B.tau_bound > 0.0 && B.gdt_free && u_in > 0.0;
    std::map<int64_t, Choice> ch;
    double total = 0.0;
    for (auto &kv : by_n) {
      std::vector<int> sel(kv.second.begin(),
                           kv.second.begin() + std::min<size_t>(kv.second.size(), 32));
      const bool tc_ok = gram_tc_supported(T, round_up(kv.first, 64));
      Choice c;
      for (int si = 0; si < 5 && rc == GLM_OK; ++si) {
        const int sv = svals[si];
        if (narrowed && sv == 1) continue;
        if (B.tau_bound > 0.0 && sv > 1) {  // the prior: every sampled problem admits it
          double tmax = 0.0;
          for (size_t k = 0; k < kv.second.size() && k < 4; ++k) {
            const Prob &q = B.pr[kv.second[k]];
            tmax = std::max(tmax, tau_g(hl[kv.second[k]][si], (double)q.eta / (double)q.b,
                                        q.loss, u_A, u_in, q.n));
          }
          if (!(tmax <= B.tau_bound)) continue;
        }
        std::vector<int> kernels = {0};
        if (sv > 1) kernels = tc_ok ? std::vector<int>{1, 2, 3} : std::vector<int>{1};
        for (int gk : kernels) {
          if (cudaMemsetAsync(xs, 0, xcount * 4, B.stream) != cudaSuccess) {
            rc = set_error(GLM_ECUDA, "autotune: cudaMemsetAsync");
            break;
          }
          double ms = 0.0, samples = 0.0;
          rc = time_candidate(B, sel, sv, gk, xs, ms, samples);
          if (rc != GLM_OK) break;
          const double rate = samples / std::max(ms, 1e-6);
          if (rate > c.rate) { c.rate = rate; c.s = sv; c.gk = gk; }
        }
      }
      ch[kv.first] = c;
      double work = 0.0;  // samples of all this n's problems at the chosen rate
      for (int p : kv.second) work += (double)B.pr[p].iters * (double)B.pr[p].b;
      total += c.rate > 0.0 ? work / c.rate : INFINITY;  // no admitted candidate
    }
    if (rc == GLM_OK && total < best_total) {
      best_total = total;
      best_type = T;
      best_choice = ch;
    }
  }
  if (rc == GLM_OK) {
    B.gdt = best_type;
    for (auto &kv : by_n)
      for (int p : kv.second) {
        B.pr[p].s = best_choice[kv.first].s;
        B.pr[p].gk = best_choice[kv.first].gk;
        const int si = (int)(std::find(svals, svals + 5, B.pr[p].s) - svals);
        auto it = hl.find(kv.second[0]);
        B.pr[p].tau = (it != hl.end() && B.pr[p].s > 1)
                          ? tau_g(it->second[si], (double)B.pr[p].eta / (double)B.pr[p].b,
                                  B.pr[p].loss, unit_roundoff(B.dtype),
                                  operand_roundoff(B.gdt, B.dtype), B.pr[p].n)
                          : 0.0;
      }
  }
  // the scratch runs' flags (a diverging candidate, a timed-out Gram) say
  // nothing about the problems' own runs: clear both words
  cudaMemsetAsync(B.bflag, 0, 2 * sizeof(unsigned), B.stream);
  cudaStreamSynchronize(B.stream);
  cudaFree(xs);
  return rc;
}

void drop_graph(Batch &B) {
  if (B.graph) cudaGraphExecDestroy(B.graph);
  B.graph = nullptr;
}

}  // namespace
}  // namespace glm

using namespace glm;

extern "C" {

void glm_batch_opts_default(glm_batch_opts *o) {
  if (!o) return;
  o->dtype = GLM_BF16;
  o->input_dtype = GLM_F32;
  o->input_on_host = 1;
  o->stream = nullptr;
  o->wait_probe_cycles = 0;
  o->tau_bound = 0.0;
}

int glm_batch_destroy(glm_batch bt) {
  Batch *B = reinterpret_cast<Batch *>(bt);
  if (!B) return GLM_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  drop_graph(*B);
  for (auto &p : B->pr)
    if (p.h) glm_destroy(p.h);
  B->ybuf.release(); B->labbuf.release(); B->gbuf.release();
  B->itembuf.release(); B->orderbuf.release(); B->queuebuf.release();
  if (B->bflag) cudaFree(B->bflag);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
  return GLM_OK;
}

int glm_batch_create(int P, const glm_problem_desc *descs, const glm_batch_opts *opts,
                     glm_batch *out) {
  set_error(GLM_OK, "");
  if (!out) return set_error(GLM_EINVAL, "out is NULL");
  *out = nullptr;
  if (P < 1 || !descs) return set_error(GLM_EINVAL, "need P >= 1 problem descriptors");
  glm_batch_opts dflt;
  glm_batch_opts_default(&dflt);
  if (!opts) opts = &dflt;
  if (opts->dtype != GLM_F32 && opts->dtype != GLM_BF16 && opts->dtype != GLM_F16)
    return set_error(GLM_EINVAL, "batch storage dtype must be F32, BF16 or F16");
  if (opts->wait_probe_cycles < 0) return set_error(GLM_EINVAL, "wait_probe_cycles must be >= 0");
  if (!(opts->tau_bound >= 0.0)) return set_error(GLM_EINVAL, "tau_bound must be >= 0");
  int gdt = -1;
  for (int p = 0; p < P; ++p) {
    const glm_problem_desc &d = descs[p];
    if (!d.A || !d.y) return set_error(GLM_EINVAL, "problem with a NULL A or y");
    if (d.m < 1 || d.m >= (1ll << 31)) return set_error(GLM_EINVAL, "m must be in [1, 2^31)");
    if (d.n < 1 || d.n > kMaxBatchN) return set_error(GLM_EINVAL, "batched n must be in [1, 16384]");
    if (d.b < 1 || d.b > 1024) return set_error(GLM_EINVAL, "batched b must be in [1, 1024]");
    if (d.s < 0 || d.s > 64) return set_error(GLM_EINVAL, "s must be 0 (autotuned) or in [1, 64]");
    if (d.iters < 0) return set_error(GLM_EINVAL, "iters must be >= 0");
    if (d.loss != GLM_LOGISTIC && d.loss != GLM_LSQ && d.loss != GLM_POISSON)
      return set_error(GLM_EINVAL, "bad loss");
    if (!(d.eta > 0.f) || !isfinite(d.eta)) return set_error(GLM_EINVAL, "eta must be > 0");
    if (!(d.lambda >= 0.f) || !isfinite(d.lambda)) return set_error(GLM_EINVAL, "lambda must be >= 0");
    const double c = 1.0 - (double)d.eta * (double)d.lambda;
    if (!(c > 0.0)) return set_error(GLM_EINVAL, "eta * lambda must be < 1");
    const int smax = d.s > 0 ? d.s : 16;
    if ((double)(smax - 1) * -log2(c) > 60.0)
      return set_error(GLM_EUNSUPPORTED, "c^-(s-1) exceeds 2^60 (eta*lambda too large for s)");
    if ((int64_t)smax * d.b > 8192) return set_error(GLM_EINVAL, "batched s*b must be <= 8192");
    if (d.gram_dtype >= 0) {
      if (d.gram_dtype != GLM_F32 && d.gram_dtype != GLM_TF32 && d.gram_dtype != GLM_BF16 &&
          d.gram_dtype != GLM_F16)
        return set_error(GLM_EINVAL, "batched gram_dtype must be F32, TF32, BF16 or F16");
      if (gdt >= 0 && gdt != d.gram_dtype)
        return set_error(GLM_EINVAL, "every problem of a batch uses the same gram_dtype");
      gdt = d.gram_dtype;
    }
  }
  Batch *B = new Batch;
  B->P = P;
  B->dtype = opts->dtype;
  B->gdt = gdt >= 0 ? gdt : opts->dtype;  // default: the storage type (exact operands)
  if (opts->stream) {
    B->stream = static_cast<cudaStream_t>(opts->stream);
  } else {
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete B;
      return set_error(GLM_ECUDA, "cudaStreamCreateWithFlags");
    }
    B->own_stream = true;
  }
  B->probe = opts->wait_probe_cycles;
  B->tau_bound = opts->tau_bound;
  B->gdt_free = gdt < 0;
  if (dev_malloc((void **)&B->bflag, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemsetAsync(B->bflag, 0, 4 * sizeof(unsigned), B->stream) != cudaSuccess) {
    cudaGetLastError();
    glm_batch_destroy(reinterpret_cast<glm_batch>(B));
    return set_error(GLM_ENOMEM, "batch flag words: device allocation failed");
  }
  B->pr.resize(P);
  for (int p = 0; p < P; ++p) {
    const glm_problem_desc &d = descs[p];
    glm_create_opts co;
    glm_create_opts_default(&co);
    co.input_dtype = opts->input_dtype;
    co.input_on_host = opts->input_on_host || !dev_ptr(d.A);
    co.stream = B->stream;
    const int rc = glm_create_ex(d.A, d.y, d.m, d.n, d.loss, B->dtype, &co, &B->pr[p].h);
    if (rc != GLM_OK) {
      const std::string msg = std::string("problem ") + std::to_string(p) + ": " + glm_last_error();
      glm_batch_destroy(reinterpret_cast<glm_batch>(B));
      return set_error(rc, msg);
    }
    Prob &q = B->pr[p];
    q.m = d.m; q.n = d.n; q.b = d.b; q.iters = d.iters; q.loss = d.loss;
    q.lambda = d.lambda; q.eta = d.eta; q.seed = d.seed;
    q.s = d.s > 0 ? d.s : 8;
    q.tuned = d.s == 0;
  }
  const int rc = autotune(*B);
  if (rc != GLM_OK) {
    const std::string msg = glm_last_error();
    glm_batch_destroy(reinterpret_cast<glm_batch>(B));
    return set_error(rc, msg);
  }
  *out = reinterpret_cast<glm_batch>(B);
  return GLM_OK;
}

int glm_batch_run(glm_batch bt, float *const *xs, int *status) {
  set_error(GLM_OK, "");
  Batch *B = reinterpret_cast<Batch *>(bt);
  if (!B || !xs) return set_error(GLM_EINVAL, "null argument");
  std::vector<int> sel;
  std::vector<int64_t> iters;
  std::vector<int> kmap(B->P, -1);
  std::vector<float *> x;
  for (int p = 0; p < B->P; ++p) {
    if (B->pr[p].iters <= 0) continue;
    if (!xs[p]) return set_error(GLM_EINVAL, "iterate pointer of a problem is NULL");
    kmap[p] = (int)sel.size();
    sel.push_back(p);
    iters.push_back(B->pr[p].iters);
    x.push_back(xs[p]);
  }
  if (!B->planned) {
    make_plan(*B, sel, iters, B->plan);
    B->planned = true;
    drop_graph(*B);
  }
  void *before[3] = {B->ybuf.ptr, B->gbuf.ptr, B->itembuf.ptr};
  std::vector<BatchItem> items;
  GLM_TRY(bind(*B, B->plan, x, &kmap, items));
  void *after[3] = {B->ybuf.ptr, B->gbuf.ptr, B->itembuf.ptr};
  if (memcmp(before, after, sizeof(before))) drop_graph(*B);
  if (x != B->xs || !B->graph) {
    GLM_TRY(upload(*B, B->plan, items));
    B->xs = x;
  }
  if (!B->graph) {
    cudaStream_t cap;
    GLM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_error(e, "cudaStreamBeginCapture");
    }
    const int rc = enqueue(*B, B->plan, cap);
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != GLM_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      B->graph = nullptr;
      return cuda_error(e, "cudaGraphInstantiate");
    }
  }
  GLM_CUDA_TRY(cudaGraphLaunch(B->graph, B->stream));
  GLM_CUDA_TRY(cudaStreamSynchronize(B->stream));
  unsigned gflag = 0;
  GLM_CUDA_TRY(cudaMemcpy(&gflag, B->bflag, sizeof(unsigned), cudaMemcpyDeviceToHost));
  int worst = GLM_OK;
  if (gflag) {  // a Gram launch gave up a bounded wait: every problem's G is suspect
    GLM_CUDA_TRY(cudaMemset(B->bflag, 0, sizeof(unsigned)));
    for (int p = 0; p < B->P; ++p) glm_sync(B->pr[p].h);  // clear the problems' flags
    const int code = (gflag & FLAG_BOUNDS) ? GLM_EBOUNDS : GLM_ETIMEOUT;
    if (status)
      for (int p = 0; p < B->P; ++p) status[p] = code;
    return set_error(code, code == GLM_EBOUNDS
                               ? "a Gram launch of the batch indexed outside G (checked build)"
                               : "a Gram launch of the batch gave up a bounded device wait");
  }
  for (int p = 0; p < B->P; ++p) {
    const int rc = glm_sync(B->pr[p].h);  // reads and clears the problem's flag
    if (status) status[p] = rc;
    if (rc != GLM_OK && rc != GLM_ENONFINITE) worst = rc;
  }
  if (worst != GLM_OK) return set_error(worst, "a problem's device flag reported a failure");
  return GLM_OK;
}

int glm_batch_loss(glm_batch bt, float *const *xs, double *out) {
  set_error(GLM_OK, "");
  Batch *B = reinterpret_cast<Batch *>(bt);
  if (!B || !xs || !out) return set_error(GLM_EINVAL, "null argument");
  for (int p = 0; p < B->P; ++p) {
    if (!xs[p]) return set_error(GLM_EINVAL, "iterate pointer of a problem is NULL");
    GLM_TRY(glm_loss(B->pr[p].h, xs[p], B->pr[p].lambda, &out[p]));
  }
  return GLM_OK;
}

int glm_tau_prior(const float *Y, int64_t n, int s, int64_t b, double alpha, int loss,
                  double u_A, double u_in, double *hl_bound, double *tau) {
  set_error(GLM_OK, "");
  if (!Y || n < 1 || s < 1 || b < 1) return set_error(GLM_EINVAL, "bad arguments");
  if (loss != GLM_LOGISTIC && loss != GLM_LSQ && loss != GLM_POISSON)
    return set_error(GLM_EINVAL, "bad loss");
  std::vector<float> v(Y, Y + (size_t)s * b * n);
  const double hl = hl_norm_bound(v, n, s, b);
  if (hl_bound) *hl_bound = hl;
  if (tau) *tau = tau_g(hl, alpha, loss, u_A, u_in, n);
  return GLM_OK;
}

int glm_batch_choice_kernel(glm_batch bt, int p, int *gram_kernel, double *tau_g) {
  set_error(GLM_OK, "");
  Batch *B = reinterpret_cast<Batch *>(bt);
  if (!B || p < 0 || p >= B->P) return set_error(GLM_EINVAL, "bad batch or problem index");
  if (gram_kernel) *gram_kernel = B->pr[p].gk;
  if (tau_g) *tau_g = B->pr[p].tau;
  return GLM_OK;
}

int glm_batch_choice(glm_batch bt, int p, int *s, int64_t *b, int *gram_dtype) {
  set_error(GLM_OK, "");
  Batch *B = reinterpret_cast<Batch *>(bt);
  if (!B || p < 0 || p >= B->P) return set_error(GLM_EINVAL, "bad batch or problem index");
  if (s) *s = B->pr[p].s;
  if (b) *b = B->pr[p].b;
  if (gram_dtype) *gram_dtype = B->gdt;
  return GLM_OK;
}

}  // extern "C"
