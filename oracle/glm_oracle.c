/*
 * glm_oracle.c -- plain, slow, FP64 CPU oracle for mini-batch SGD and
 * s-step (communication-avoiding) SGD on generalized linear models.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Every function follows the paper (Mixed-Precision Communication-Avoiding
 * SGD for Generalized Linear Models on GPUs) step by step, in FP64, with no
 * blocking, fusion or reordering beyond what the definitions state:
 *   - GLM risk and losses ........................ Sec. 2.1
 *   - residual delta = -dL/dr ..................... Sec. 3.1
 *   - mini-batch SGD step ......................... Sec. 2.1, Sec. 3.1
 *   - CA-SGD outer iteration ...................... Algorithm 1, Sec. 2.2
 *   - sampling: i.i.d. uniform with replacement ... Algorithm 1 (sampling step)
 * The paper does not name its random number generator.  The index stream
 * is Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11), keyed by (seed, problem), counter (k,0,0,0)
 * for block k; draw q uses word q mod 4 of block q div 4, and maps the
 * 64-bit word U to the row floor(U * m / 2^64).
 *
 * The ridge term lambda is absent from the paper.  The objective here is
 * F(x) = m^-1 sum_i L(a_i^T x, y_i) + (lambda/2) ||x||^2, so one SGD step is
 * x <- c x - alpha Y^T u with c = 1 - eta*lambda, alpha = eta/b and
 * u = dL/dr (u = -delta in the paper's notation).
 *
 * Conventions: A is row-major m x n, given as FP32 values (converted to FP64
 * exactly on use), labels y are FP32, iterates x are FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LOGISTIC 0
#define ORC_LSQ 1
#define ORC_POISSON 2

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (SC'11, Sec. 4): 10 rounds of two 64x64->128 multiplies.   */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_MUL0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_MUL1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_WEYL0 = 0x9E3779B97F4A7C15ULL; /* golden ratio   */
static const uint64_t PHILOX_WEYL1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1    */

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                       uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: Weyl sequence */
      k0 += PHILOX_WEYL0;
      k1 += PHILOX_WEYL1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul_hi_lo(PHILOX_MUL0, x0, &hi0, &lo0);
    mul_hi_lo(PHILOX_MUL1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Raw 64-bit word for global draw q of stream (seed, problem). */
uint64_t orc_draw_word(uint64_t seed, uint64_t problem, int64_t q) {
  uint64_t ctr[4] = {(uint64_t)q >> 2, 0, 0, 0};
  uint64_t key[2] = {seed, problem};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[(uint64_t)q & 3u];
}

/* Row index in [0, m): floor(U * m / 2^64). */
static int64_t draw_row(uint64_t seed, uint64_t problem, int64_t q, int64_t m) {
  uint64_t U = orc_draw_word(seed, problem, q);
  uint64_t hi, lo;
  mul_hi_lo(U, (uint64_t)m, &hi, &lo);
  return (int64_t)hi;
}

/* Algorithm 1, sampling step: `count` draws starting at global draw index
 * first_draw, i.i.d. uniform over {0..m-1} with replacement. */
void orc_sample_indices(uint64_t seed, uint64_t problem, int64_t first_draw,
                        int64_t count, int64_t m, int64_t *out) {
  for (int64_t i = 0; i < count; ++i)
    out[i] = draw_row(seed, problem, first_draw + i, m);
}

/* ------------------------------------------------------------------------ */
/* Losses and residuals, Sec. 2.1 and Sec. 3.1                               */
/* ------------------------------------------------------------------------ */
/* sigma(t) = 1/(1+e^-t), evaluated without overflow. */
static double sigmoid(double t) {
  if (t >= 0.0) return 1.0 / (1.0 + exp(-t));
  double e = exp(t);
  return e / (1.0 + e);
}

/* u = dL/dr (r, y); the paper's residual is delta = -u. */
double orc_dloss(int loss, double r, double y) {
  switch (loss) {
  case ORC_LOGISTIC: /* L = log(1+e^{-y r}) ; dL/dr = -y sigma(-y r) */
    return -y * sigmoid(-y * r);
  case ORC_LSQ: /* L = (r-y)^2/2 */
    return r - y;
  case ORC_POISSON: /* L = e^r - y r */
    return exp(r) - y;
  }
  return NAN;
}

double orc_loss_one(int loss, double r, double y) {
  switch (loss) {
  case ORC_LOGISTIC: { /* log(1+e^{-t}) = max(-t,0) + log1p(e^{-|t|}) */
    double t = y * r;
    return fmax(-t, 0.0) + log1p(exp(-fabs(t)));
  }
  case ORC_LSQ:
    return 0.5 * (r - y) * (r - y);
  case ORC_POISSON:
    return exp(r) - y * r;
  }
  return NAN;
}

static double dot_row(const float *a, const double *x, int64_t n) {
  double acc = 0.0;
  for (int64_t k = 0; k < n; ++k) acc += (double)a[k] * x[k];
  return acc;
}

/* Pairwise (recursive halving) sum of v[0..len). */
static double pairwise_sum(const double *v, int64_t len) {
  if (len <= 8) {
    double acc = 0.0;
    for (int64_t i = 0; i < len; ++i) acc += v[i];
    return acc;
  }
  int64_t half = len / 2;
  return pairwise_sum(v, half) + pairwise_sum(v + half, len - half);
}

/* Sec. 2.1: F(x) = m^-1 sum_i L(a_i^T x, y_i) + (lambda/2) ||x||^2. */
double orc_loss(const float *A, const float *y, int64_t m, int64_t n,
                int loss, double lambda, const double *x) {
  double *terms = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  if (!terms) return NAN;
  for (int64_t i = 0; i < m; ++i)
    terms[i] = orc_loss_one(loss, dot_row(A + i * n, x, n), (double)y[i]);
  double risk = pairwise_sum(terms, m) / (double)m;
  free(terms);
  double xx = 0.0;
  for (int64_t k = 0; k < n; ++k) xx += x[k] * x[k];
  return risk + 0.5 * lambda * xx;
}

/* ------------------------------------------------------------------------ */
/* Mini-batch SGD, Sec. 2.1 / Sec. 3.1, with the ridge decay c = 1 - eta*lambda.
 * Iteration t (counted from first_iter) uses draws [(first_iter+t) b, +b).   */
/* ------------------------------------------------------------------------ */
int orc_sgd(const float *A, const float *y, int64_t m, int64_t n, int loss,
            int64_t b, double eta, double lambda, int64_t iters, uint64_t seed,
            uint64_t problem, int64_t first_iter, double *x) {
  if (m <= 0 || n <= 0 || b <= 0 || iters < 0) return 1;
  const double alpha = eta / (double)b;
  const double c = 1.0 - eta * lambda;
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)b);
  double *u = (double *)malloc(sizeof(double) * (size_t)b);
  double *g = (double *)malloc(sizeof(double) * (size_t)n);
  if (!idx || !u || !g) { free(idx); free(u); free(g); return 2; }
  for (int64_t t = 0; t < iters; ++t) {
    orc_sample_indices(seed, problem, (first_iter + t) * b, b, m, idx);
    /* margins and residuals at the current iterate */
    for (int64_t l = 0; l < b; ++l) {
      const float *a = A + idx[l] * n;
      u[l] = orc_dloss(loss, dot_row(a, x, n), (double)y[idx[l]]);
    }
    /* g = Y^T u */
    for (int64_t k = 0; k < n; ++k) g[k] = 0.0;
    for (int64_t l = 0; l < b; ++l) {
      const float *a = A + idx[l] * n;
      for (int64_t k = 0; k < n; ++k) g[k] += (double)a[k] * u[l];
    }
    for (int64_t k = 0; k < n; ++k) x[k] = c * x[k] - alpha * g[k];
  }
  free(idx); free(u); free(g);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* CA-SGD, Algorithm 1 (exact FP64), extended with the ridge decay.
 * Outer block h covers iterations [h s, h s + s_h), s_h = min(s, iters - h s),
 * i.e. draws [(first_iter + h s) b, +s_h b).  With x_0 the block's start:
 *   r   = Y x_0                                   (margin, Alg. 1)
 *   G   = Y Y^T, only blocks G_{j,i}, i < j used  (Gram, Alg. 1)
 *   z_j = c^j r_j - alpha sum_{i<j} c^{j-1-i} G_{j,i} u_i   (correction)
 *   u_j = dL/dr(z_j, y_{I_j})                     (residual)
 *   x  <- c^{s_h} x_0 - alpha sum_j c^{s_h-1-j} Y_j^T u_j   (update)
 * With lambda = 0 (c = 1) this is Algorithm 1 with delta = -u.           */
/* ------------------------------------------------------------------------ */
int orc_ca_sgd(const float *A, const float *y, int64_t m, int64_t n, int loss,
               int64_t s, int64_t b, double eta, double lambda, int64_t iters,
               uint64_t seed, uint64_t problem, int64_t first_iter, double *x) {
  if (m <= 0 || n <= 0 || b <= 0 || s <= 0 || iters < 0) return 1;
  const double alpha = eta / (double)b;
  const double c = 1.0 - eta * lambda;
  const int64_t sb = s * b;
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)sb);
  double *r = (double *)malloc(sizeof(double) * (size_t)sb);
  double *u = (double *)malloc(sizeof(double) * (size_t)sb);
  double *G = (double *)malloc(sizeof(double) * (size_t)(sb * sb));
  double *cpow = (double *)malloc(sizeof(double) * (size_t)(s + 1));
  if (!idx || !r || !u || !G || !cpow) {
    free(idx); free(r); free(u); free(G); free(cpow);
    return 2;
  }
  cpow[0] = 1.0;
  for (int64_t p = 1; p <= s; ++p) cpow[p] = cpow[p - 1] * c;

  for (int64_t t0 = 0; t0 < iters; t0 += s) {
    const int64_t sh = (iters - t0 < s) ? (iters - t0) : s;
    const int64_t rows = sh * b;
    orc_sample_indices(seed, problem, (first_iter + t0) * b, rows, m, idx);
    /* base margin r = Y x */
    for (int64_t p = 0; p < rows; ++p) r[p] = dot_row(A + idx[p] * n, x, n);
    /* strictly block-lower Gram blocks G_{j,i} = Y_j Y_i^T, i < j */
    for (int64_t p = 0; p < rows; ++p) {
      const int64_t j = p / b;
      for (int64_t q = 0; q < j * b; ++q) {
        const float *ap = A + idx[p] * n, *aq = A + idx[q] * n;
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += (double)ap[k] * (double)aq[k];
        G[p * sb + q] = acc;
      }
    }
    /* inner s-step recurrence */
    for (int64_t j = 0; j < sh; ++j) {
      for (int64_t l = 0; l < b; ++l) {
        const int64_t p = j * b + l;
        double corr = 0.0;
        for (int64_t i = 0; i < j; ++i) {
          double blk = 0.0;
          for (int64_t l2 = 0; l2 < b; ++l2)
            blk += G[p * sb + i * b + l2] * u[i * b + l2];
          corr += cpow[j - 1 - i] * blk;
        }
        const double z = cpow[j] * r[p] - alpha * corr;
        u[p] = orc_dloss(loss, z, (double)y[idx[p]]);
      }
    }
    /* outer update x <- c^{s_h} x - alpha sum_j c^{s_h-1-j} Y_j^T u_j */
    for (int64_t k = 0; k < n; ++k) {
      double gk = 0.0;
      for (int64_t p = 0; p < rows; ++p)
        gk += cpow[sh - 1 - p / b] * (double)A[idx[p] * n + k] * u[p];
      x[k] = cpow[sh] * x[k] - alpha * gk;
    }
  }
  free(idx); free(r); free(u); free(G); free(cpow);
  return 0;
}
