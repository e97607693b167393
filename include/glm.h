/*
 * glm.h -- C ABI of libglm: s-step (communication-avoiding) mini-batch SGD
 * for binary logistic regression and least squares / ridge on one GB300
 * (sm_103a), after "Mixed-Precision Communication-Avoiding SGD for
 * Generalized Linear Models on GPUs".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status (GLM_OK on success).  On failure,
 *    glm_last_error() returns a thread-local, NUL-terminated description.
 *  - Pointers are DEVICE pointers unless the argument says "host".  The
 *    caller owns every buffer it passes; the library owns what a handle
 *    allocates and frees it in glm_destroy / glm_batch_destroy.
 *  - Matrices are row-major, with contiguous rows (stride = number of
 *    columns) unless a leading dimension is given.
 *  - Work is enqueued on the handle's stream and returns without waiting,
 *    except glm_create*, glm_loss, glm_sample_indices with a host output
 *    and glm_sync, which block.  Device-side checks (non-finite iterates)
 *    raise a flag that glm_sync reports as GLM_ENONFINITE.
 *  - Argument errors return GLM_EINVAL before anything is enqueued.
 *
 * Notation (paper Sec. 3.1): A in R^{m x n}, labels y, mini-batch b, s-step
 * length s, step size eta, ridge weight lambda, alpha = eta / b,
 * c = 1 - eta * lambda.  The objective is
 *     F(x) = m^-1 sum_i L(a_i^T x, y_i) + (lambda/2) ||x||^2
 * with L the logistic loss log(1 + exp(-y r)), the squared loss (r - y)^2 / 2
 * or the Poisson loss e^r - y r (its constant log y! dropped) (paper Sec. 2.1;
 * the ridge term is this library's addition).
 */
#ifndef GLM_H_
#define GLM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define GLM_OK 0
#define GLM_EINVAL 1        /* invalid argument                                */
#define GLM_ENOMEM 2        /* device allocation failed                        */
#define GLM_ECUDA 3         /* a CUDA runtime / driver call failed             */
#define GLM_ENONFINITE 4    /* a NaN or Inf was produced on the device         */
#define GLM_ETIMEOUT 5      /* a bounded device wait gave up                   */
#define GLM_EUNSUPPORTED 6  /* valid request the library does not support      */
#define GLM_EBOUNDS 7       /* checked builds only: a kernel's computed index
                               fell outside its buffer; the access was skipped */

/* ---- losses (paper Sec. 2.1) -------------------------------------------- */
#define GLM_LOGISTIC 0      /* labels must be -1 or +1 */
#define GLM_LSQ 1           /* least squares / ridge   */
#define GLM_POISSON 2       /* Poisson counts y >= 0, log link (Sec. 2.1 lists the GLM family) */

/* ---- element types (paper Table 1 storage slots u_A, u_G, u_r, u_g) ------ */
#define GLM_F32 0
#define GLM_BF16 1
#define GLM_F16 2
#define GLM_TF32 3          /* FP32 container rounded to 10 mantissa bits      */
#define GLM_E4M3 4          /* FP8 E4M3 with one power-of-two scale per row    */
#define GLM_F64 5

typedef struct glm_handle_s *glm_handle;

/* Last error message of the calling thread ("" if none). */
const char *glm_last_error(void);

/* Library version string. */
const char *glm_version(void);

/* 1 when this library was built with -DGLM_CHECKED (every kernel tests its
 * computed indices against their buffers, records an index outside them as
 * GLM_EBOUNDS at the next glm_sync or glm_batch_run and skips the access),
 * else 0.  The checked build is a test instrument: slower, same results. */
int glm_checked_build(void);

/* ---- dataset handles ----------------------------------------------------- */

typedef struct {
  int input_dtype;   /* element type behind the A pointer: GLM_F32 (float)
                        or GLM_BF16 (uint16 bit patterns).  Default GLM_F32. */
  int input_on_host; /* 1: A and y are host pointers; 0 (default): device.    */
  int column_scales; /* 1 (default): BF16/F16 storage keeps one power-of-two
                        scale per column (the value nearest the column RMS)
                        and stores A/scale.                                    */
  int fp8_copy;      /* 1: also keep an FP8-E4M3 copy of A with one
                        power-of-two scale per row (needed by GLM_E4M3 Gram). */
  void *stream;      /* cudaStream_t the handle enqueues on; NULL creates a
                        private non-blocking stream owned by the handle (pass
                        cudaStreamLegacy, 0x1, for the legacy default stream). */
} glm_create_opts;

/* Fill *o with the defaults documented above. */
void glm_create_opts_default(glm_create_opts *o);

/*
 * Copy the dataset (A: m x n row-major, y: m labels) into handle-owned
 * device storage of element type `dtype` (GLM_F32, GLM_BF16 or GLM_F16),
 * paper Table 1 slot u_A; labels stay FP32.  The caller keeps ownership of
 * A and y.  Requires 1 <= m < 2^31, 1 <= n <= 65536, loss GLM_LOGISTIC
 * (labels exactly +-1), GLM_LSQ (finite labels) or GLM_POISSON (finite
 * labels >= 0); other labels give GLM_EINVAL.  Blocks until the copy and
 * conversion are done.  glm_create takes device FP32 pointers.
 */
int glm_create(const float *A, const float *y, int64_t m, int64_t n, int loss,
               int dtype, glm_handle *out);
int glm_create_ex(const void *A, const float *y, int64_t m, int64_t n,
                  int loss, int dtype, const glm_create_opts *opts,
                  glm_handle *out);

/* Release everything the handle owns.  NULL is accepted. */
int glm_destroy(glm_handle h);

/* Shape / stream queries. */
int glm_shape(glm_handle h, int64_t *m, int64_t *n);
void *glm_stream(glm_handle h);

/* Wait for the handle's stream; returns GLM_ENONFINITE if a run since the
 * previous glm_sync produced a non-finite value (the flag is then cleared). */
int glm_sync(glm_handle h);

/* ---- runs ---------------------------------------------------------------- */

typedef struct {
  int gram_dtype;     /* u_G: GLM_F32, GLM_TF32, GLM_BF16, GLM_F16 or GLM_E4M3;
                         -1 (default) = the storage type.  Accumulation is
                         always FP32 (paper Eq. for BF16-in/FP32-acc).       */
  int gemv_dtype;     /* u_r = u_g (margin and outer-gradient operands);
                         -1 (default) = gram_dtype, or the storage type when
                         gram_dtype is GLM_E4M3.                              */
  int recurrence_f64; /* u_c: -1 (default) FP64 iff s >= 32, 0 FP32, 1 FP64,
                         2 compensated FP32.  In FP64 the correction sums and
                         residual history are FP64 and each residual
                         (u_sigma) is the FP32 loss derivative of the FP64
                         margin; in FP32 the residual uses the fast
                         exponential and division.  Compensated FP32 (the
                         streaming chain only): FP32 products with per-lane
                         Kahan sums combined in FP64, residual as in FP64
                         mode -- the correction's error stays near
                         2 u_32 sum |G| |u| whatever its length, like FP64
                         sums, at FP32 rates (GB300's FP64 rate is 1/64).     */
  int kahan;          /* 1 (default): Kahan-compensated FP32 Y^T u sums.      */
  int64_t first_iter; /* SGD-equivalent iteration the run starts at; draws
                         continue the counter-based stream from there, so a
                         run of k+l iterations equals a run of k followed by
                         a run of l with first_iter = k.  Default 0.         */
  uint32_t problem;   /* stream id (second Philox key word).  Default 0.     */
  int use_graph;      /* 1 (default): capture the run as a CUDA graph once
                         per shape and replay it.                            */
  int cluster;        /* CTAs cooperating on the x-dependent chain:
                         0 (default) = automatic, else 1..16.                */
  int64_t chunk_outer;/* outer iterations staged per chunk; 0 = automatic.   */
  int gram_impl;      /* 0 (default) automatic, 1 SIMT FP32 kernel,
                         2 tcgen05 tensor-core kernel, 3 SIMT kernel with
                         FP16 accumulation, 4 tcgen05 kernel with an FP16
                         accumulator (3 and 4: Recipe F's Gram slot, FP16
                         input and accumulation; gram_dtype GLM_F16 only,
                         else GLM_EINVAL; never chosen automatically).       */
  int timing;         /* 1: record CUDA events around every kernel of the run
                         (read back with glm_kernel_times).  Default 0.       */
  int accumulate;     /* GLM_F32 (default) or GLM_F16: FP16 accumulation in
                         the margin and gradient GEMVs (Recipe F's h_a slots;
                         FP16 GEMV operands required; pair it with gram_impl
                         3 or 4 for the FP16-accumulate Gram).               */
  int state_dtype;    /* GLM_F32 (default), GLM_BF16 (Recipe I) or GLM_F16
                         (Recipe H): CA-SGD end to end in that type -- the
                         margins, the Gram output, each correction, residual
                         and history entry, the gradient and the weights are
                         rounded to it once each (x is rounded on entry and
                         holds values of the type on return); Gram and GEMV
                         operands must be that type; the correction sums
                         accumulate in FP16 when accumulate is GLM_F16.
                         Either field away from GLM_F32 runs a per-step
                         numerical baseline (one kernel per stage and outer
                         iteration, no graph), not the fused chain.          */
  int chain_impl;     /* x-dependent chain kernel: 0 (default) automatic, 1
                         resident (the step's Y and G staged whole in the
                         cluster's shared memory), 2 streaming (Y and G
                         streamed through shared-memory rings: wide rows,
                         long blocks).  Automatic takes the streaming kernel
                         when the resident one cannot stage the step (except
                         with FP64 sums, which stay resident), and for
                         recurrence_f64 = 2.                                  */
  int64_t wait_probe_cycles;
                      /* Failure-path test hook; 0 (default) = off.  When > 0,
                         one thread of every CTA of the chain and tcgen05
                         Gram kernels first waits, for at most this many SM
                         cycles, on a barrier that nothing signals; the wait
                         gives up, and the kernels unwind as after any device
                         timeout before any data moves between CTAs (copies
                         in flight are drained, TMEM is freed, x is left as
                         it was).  glm_sync then returns GLM_ETIMEOUT.      */
} glm_ca_opts;

void glm_ca_opts_default(glm_ca_opts *o);

/* What a run with these arguments will do (no work is enqueued). */
typedef struct {
  int64_t chunk_outer;  /* outer iterations staged per chunk                  */
  int64_t chunks;       /* number of chunks                                   */
  int64_t launches;     /* kernels launched by the run                        */
  int cluster;          /* CTAs in the chain cluster                          */
  int gram_impl;        /* 1 SIMT, 2 tcgen05, 3 SIMT FP16 accumulation       */
  int gram_dtype, gemv_dtype, recurrence_f64;
  int chain_impl;       /* 1 resident, 2 streaming                            */
} glm_run_plan;

int glm_ca_plan(glm_handle h, int s, int64_t b, float eta, float lambda,
                int64_t iters, const glm_ca_opts *opts, glm_run_plan *out);

/*
 * Per-kernel device time of the most recent run made with opts.timing = 1,
 * from CUDA events recorded on the handle's stream (inside the captured
 * graph when graphs are used).  ms[0..2] = summed milliseconds of the
 * gather, Gram and chain kernels; launches[0..2] = their launch counts.
 * Blocks until that run has finished.
 */
int glm_kernel_times(glm_handle h, double *ms, int64_t *launches);

/*
 * Plain mini-batch SGD (paper Sec. 2.1 / Sec. 3.1) in FP32 with FP32 master
 * weights: per iteration t, draw b rows, z = Y x, u = dL/dr(z, y_I),
 * x <- c x - alpha Y^T u.  x: device FP32[n], read as x_0 and overwritten
 * with x_T.  iters >= 0, b >= 1, 0 <= eta*lambda < 1.
 */
int glm_sgd_run(glm_handle h, int64_t b, float eta, float lambda,
                int64_t iters, uint64_t seed, float *x);
int glm_sgd_run_ex(glm_handle h, int64_t b, float eta, float lambda,
                   int64_t iters, uint64_t seed, float *x,
                   const glm_ca_opts *opts);

/*
 * End-to-end low-precision mini-batch SGD: the paper's end-to-end BF16 and
 * FP16 baselines (Recipes I and H of the precision-symbol table, Sec. 5.3,
 * run as plain mini-batch SGD as in the end-to-end check of Sec. 7,
 * "Accuracy gap").  The state type T is the handle's storage type (GLM_BF16
 * or GLM_F16).  Per iteration t it draws b rows from the same index stream as
 * glm_sgd_run (draws (first_iter + t) b .. + b - 1, stream id 0), then
 *     z = T(Y x),  u = T(dL/dr(z, y_I)),  g = T(Y^T u),
 *     x <- T(c x - alpha g),   alpha = eta / b, c = 1 - eta lambda,
 * where T(.) rounds to nearest even once.  The residual and the update are
 * evaluated in FP32; the inner products accumulate in FP32 (accumulate =
 * GLM_F32) or, with FP16 storage only, in FP16 by fused multiply-adds
 * (accumulate = GLM_F16, Recipe H's FP16 accumulation).  Power-of-two
 * column scales of the storage fold into the weights exactly.
 * x: device FP32[n], read as x_0 (each entry rounded to T first) and
 * overwritten with x_T (values of T).  iters >= 0, 1 <= b <= 1024,
 * 0 <= eta*lambda < 1, first_iter >= 0; n up to about 27,000
 * (GLM_EUNSUPPORTED beyond the on-chip state).  Runs on one SM (a baseline,
 * not a fast path), allocates nothing and returns once the work is enqueued
 * on the handle's stream; non-finite values raise the handle's flag.
 */
int glm_sgd_lowp_run(glm_handle h, int64_t b, float eta, float lambda,
                     int64_t iters, uint64_t seed, float *x, int accumulate,
                     int64_t first_iter);

/*
 * CA-SGD (paper Algorithm 1, with the ridge decay c).  Each outer iteration
 * draws s*b indices, gathers Y (s b x n), forms r = Y x and the strictly
 * block-lower Gram blocks G_{j,i} = Y_j Y_i^T (i < j), runs
 *     z_j = c^j r_j - alpha sum_{i<j} c^{j-1-i} G_{j,i} u_i,
 *     u_j = dL/dr(z_j, y_{I_j}),                       j = 0..s-1,
 * and applies x <- c^s x - alpha sum_j c^{s-1-j} Y_j^T u_j.  In exact
 * arithmetic this equals s SGD iterations on the same draws (paper
 * Assumption 6).  If iters % s != 0 the last outer iteration has
 * iters % s inner steps.  x: device FP32[n], in/out.  0 <= eta*lambda < 1;
 * the recurrence carries the residual history scaled by c^-j, so a request
 * with c^-(s-1) > 2^60 (eta*lambda near 1 with a long s, e.g. eta*lambda
 * above about 0.48 at s = 64) returns GLM_EUNSUPPORTED before any work.
 */
int glm_ca_sgd_run(glm_handle h, int s, int64_t b, float eta, float lambda,
                   int64_t iters, uint64_t seed, float *x);
int glm_ca_sgd_run_ex(glm_handle h, int s, int64_t b, float eta, float lambda,
                      int64_t iters, uint64_t seed, float *x,
                      const glm_ca_opts *opts);

/*
 * F(x) = m^-1 sum_i L(a_i^T x, y_i) + (lambda/2) ||x||^2 over the stored
 * data (paper Sec. 2.1), FP32 margins, Kahan-compensated FP32 per-thread
 * sums, FP64 block totals.  x: device FP32[n]; *out: host double.  Blocks.
 */
int glm_loss(glm_handle h, const float *x, float lambda, double *out);

/*
 * Index stream (paper Algorithm 1, sampling step): out[i] = row of global
 * draw first_draw + i, i.i.d. uniform on [0, m) with replacement.  Draw q
 * takes 64-bit word q mod 4 of Philox4x64-10 block (q div 4, 0, 0, 0) under
 * key (seed, problem) and maps it to floor(U m / 2^64).  out may be host or
 * device memory (detected); count >= 0, 1 <= m < 2^31.  Blocks.
 */
int glm_sample_indices(uint64_t seed, uint32_t problem, int64_t first_draw,
                       int64_t count, int64_t m, int32_t *out);

/*
 * No counterpart in the paper: a form of glm_sample_indices for a HOST
 * output that allocates nothing.  The draws are staged in a fixed device
 * array of GLM_SAMPLE_NOALLOC_MAX int32 (4 MiB, one per device) instead of a
 * per-call cudaMalloc/cudaFree; results equal glm_sample_indices'.
 * out: host int32[count].  count > GLM_SAMPLE_NOALLOC_MAX returns GLM_EINVAL
 * before any device work.  Calls whose work overlaps on the same GPU race on
 * the shared staging array: serialise them.  The first call on a device
 * resolves the array's address (cudaGetSymbolAddress, with that device
 * current): make it before any stream capture.  The address is kept for the
 * life of the process, so do not call this on a device after a
 * cudaDeviceReset of it.  A device (or managed) out pointer returns
 * GLM_EINVAL.  Blocks.
 */
#define GLM_SAMPLE_NOALLOC_MAX 1048576
int glm_sample_indices_noalloc(uint64_t seed, uint32_t problem, int64_t first_draw,
                               int64_t count, int64_t m, int32_t *out);

/* ---- kernel-level entry points (tests, micro-benchmarks) ----------------- */

/*
 * Failure-path test hook (host side): the next `after` device allocations the
 * library makes succeed and the one after them fails as if the device were
 * out of memory, so the call making it returns GLM_ENOMEM after releasing
 * what it had allocated.  A negative value disarms the hook (the default).
 * Affects every thread of the process.
 */
void glm_debug_fail_alloc(int64_t after);

/*
 * Layout of the dataset a handle stores (Table 1 slot u_A, created by
 * glm_create_ex): *dtype = GLM_F32, GLM_BF16 or GLM_F16; *lda = row stride in
 * elements (n rounded up to a multiple of 8; columns n..lda-1 hold zeros);
 * *lda8 = row stride in bytes of the optional FP8-E4M3 copy (n rounded up to
 * a multiple of 16; 0 when there is none).  Any output may be NULL.
 */
int glm_storage_layout(glm_handle h, int *dtype, int64_t *lda, int64_t *lda8);

/*
 * Copy rows [row0, row0 + rows) of what glm_create_ex stored to HOST memory,
 * so that the create-time quantisation can be checked value by value.  Each
 * output may be NULL (skipped):
 *   A_out         rows x lda elements of the storage type, as stored (A / kappa
 *                 rounded to nearest even, kappa the column scale);
 *   colscale_out  n floats: the power-of-two column scales kappa_j (all 1
 *                 when the handle keeps none, e.g. FP32 storage);
 *   fp8_out       rows x lda8 E4M3 bytes (E4M3(a / rho_i), nearest even,
 *                 saturating); GLM_EINVAL if the handle has no FP8 copy;
 *   rowscale_out  rows floats: the FP8 copy's power-of-two row scales rho_i;
 *                 GLM_EINVAL if the handle has no FP8 copy.
 * Requires 0 <= row0, rows >= 0, row0 + rows <= m.  Blocks.
 */
int glm_storage_read(glm_handle h, int64_t row0, int64_t rows, void *A_out,
                     float *colscale_out, uint8_t *fp8_out, float *rowscale_out);

/*
 * Strictly block-lower Gram (paper Algorithm 1, Gram step; Sec. 5.2 G_L) of
 * `nouter` consecutive row groups of Y.  Y: device, `nouter * s * b` rows of
 * `ld` elements of type `dtype` (GLM_F32, GLM_TF32 (FP32 container),
 * GLM_BF16, GLM_F16, GLM_E4M3 bytes); only the first n columns are read and
 * columns n..ld-1 must be zero.  row_scale: device FP32 per row (E4M3 only,
 * else NULL).  G: device FP32, for each group g the s(s-1)/2 blocks stored
 * row-block by row-block with 16-byte aligned rows: with ld_t =
 * 4 ceil(t b / 4), row l of block row j (1 <= j < s) holds the j*b values
 * G[j b + l][0 .. j b) at float offset g Z + b (ld_1 + ... + ld_{j-1}) +
 * l ld_j, where Z = b (ld_1 + ... + ld_{s-1}) floats per group; the padding
 * floats of a row hold no result.  impl: 0 auto, 1 SIMT FP32, 2 tcgen05, 3
 * SIMT with FP16 accumulation, 4 tcgen05 with an FP16 accumulator (3 and 4:
 * GLM_F16 only, else GLM_EINVAL).  ld must be a multiple of 64 for impl 2
 * and 4.  With impl 2 (or 0 choosing it) a shape with fewer 128 x 256 tiles
 * than SMs and at least 4,096 bytes of K per row splits K across SMs: the
 * whole G range is zeroed on the stream first (padding included) and the
 * partial sums are added atomically, so the last bits of an entry can differ
 * between runs; each entry stays within the FP32-accumulation bound.
 * stream: cudaStream_t or NULL (legacy default stream).
 */
int glm_gram_lower(const void *Y, int dtype, int64_t nouter, int s, int64_t b,
                   int64_t n, int64_t ld, const float *row_scale, float *G,
                   int impl, void *stream);

/* ---- column-partitioned CA-SGD (P ranks) ---------------------------------- */
/*
 * Paper Algorithm 1 on P ranks with the 1D block-column partition (Sec. 4):
 * rank p holds a column slab A_p of A (its own handle, created from those
 * columns with every row and the same labels) and the matching slab x_p of
 * the iterate.  Every rank draws the same rows (same seed and stream id).
 * One outer iteration of sh inner steps (1 <= sh <= s; sh < s only for a
 * run's last, shorter block) is:
 *   glm_slab_partial(rank p)   red_p = [ r_p | G_p ]
 *   red = sum over p of red_p  (the grouped AllReduce of Sec. 6, done by the
 *                               caller: NCCL/gloo across processes, or
 *                               glm_sum_buffers across ranks emulated on one
 *                               device)
 *   glm_slab_finish(rank p)    recurrence on red, update of x_p
 * red holds glm_slab_reduce_floats(s, b) floats: the partial margins
 * r_p = Y_p x_p in red[0 .. round_up(s b, 4)) (zeros past sh b), then the
 * strictly block-lower Gram of the step's rows over the slab's columns in the
 * packed row-block layout of glm_gram_lower (zeros for blocks >= sh).  The
 * recurrence is the same on every rank, so the slabs stay one iterate; in
 * exact arithmetic P ranks equal one rank (and SGD).  Precision options are
 * those of glm_ca_opts (gram_dtype, gemv_dtype, recurrence_f64, kahan,
 * gram_impl, problem; first_iter and the graph/cluster/chunk/timing options
 * are ignored).  s b <= 8192.  Both calls enqueue on the handle's stream; a
 * finish must follow its partial on the same handle with the same s, b, sh.
 */
int glm_slab_reduce_floats(int s, int64_t b, int64_t *count);
/* Gather the step's rows (SGD-equivalent iterations first_iter .. first_iter
 * + sh - 1, draws first_iter b ..), write red.  x: device FP32[n_p] (read);
 * red: device FP32[glm_slab_reduce_floats] (written). */
int glm_slab_partial(glm_handle h, int s, int64_t b, int sh, uint64_t seed, int64_t first_iter,
                     const float *x, float *red, const glm_ca_opts *opts);
/* Run the recurrence on the summed red (read) and update x (device FP32[n_p],
 * in/out): x <- c^sh x - alpha sum_j c^{sh-1-j} Y_{j,p}^T u_j. */
int glm_slab_finish(glm_handle h, int s, int64_t b, int sh, float eta, float lambda,
                    const float *red, float *x, const glm_ca_opts *opts);
/* dst[i] = srcs[0][i] + srcs[1][i] + ... + srcs[P-1][i] in rank order, FP32
 * (the reduction of ranks emulated on one device).  srcs: host array of P
 * device pointers, 1 <= P <= 64; dst may be one of them.  stream: cudaStream_t
 * or NULL (legacy default stream).  Enqueues and returns. */
int glm_sum_buffers(float *dst, const float *const *srcs, int P, int64_t count, void *stream);

/* ---- batched fits -------------------------------------------------------- */
/*
 * No counterpart in the paper (its experiments fit one problem at a time):
 * many independent fits of uneven m, n and lambda share the device.  Every
 * problem is fit with CA-SGD (paper Algorithm 1) on its own index stream:
 * problem p draws from Philox key (desc[p].seed, p), so it reproduces a
 * single-problem run with glm_ca_opts.problem = p.
 */
typedef struct {
  const void *A;     /* m x n, element type input_dtype, host or device    */
  const float *y;    /* m labels                                           */
  int64_t m, n;      /* 1 <= m < 2^31, 1 <= n <= 16384                     */
  int loss;          /* GLM_LOGISTIC, GLM_LSQ or GLM_POISSON              */
  float lambda, eta;
  int64_t iters;     /* SGD-equivalent iterations (0: the problem is idle) */
  uint64_t seed;
  int s;             /* 1..64, or 0: chosen by the autotuner (1..16)       */
  int64_t b;         /* mini-batch size, 1..1024, s*b <= 8192 (required:
                        b is part of the problem, the tuner never picks it) */
  int gram_dtype;    /* -1: the storage type; else GLM_F32, GLM_TF32,
                        GLM_BF16 or GLM_F16, the same for every problem     */
} glm_problem_desc;

typedef struct glm_batch_s *glm_batch;

typedef struct {
  int dtype;          /* storage type for every problem (default GLM_BF16) */
  int input_dtype;    /* GLM_F32 (default) or GLM_BF16                      */
  int input_on_host;  /* 1 (default): descriptors point to host memory      */
  void *stream;       /* as glm_create_opts.stream                          */
  int64_t wait_probe_cycles; /* as glm_ca_opts.wait_probe_cycles, for the
                         batch's tcgen05 Gram launches (glm_batch_run then
                         returns GLM_ETIMEOUT); 0 (default) = off            */
  double tau_bound;   /* 0 (default): the Gram operand type is the one the
                         descriptors give (else the storage type).  > 0 and
                         no descriptor fixes it: the autotuner also chooses
                         the batch's Gram type among FP32, TF32, FP16 and
                         BF16 (FP32 storage; narrower storage keeps its own,
                         already exact, type), admitting an (s, type) pair
                         only if Theorem 1's hypothesis figure
                         tau_G = K_s L_sigma alpha (2 u_A + gamma_G) ||H_L||
                         (paper Sec. 5.2), bounded from one gathered outer
                         step of up to four problems of each n, is at most
                         tau_bound (the theorem needs <= 1/2).  A narrower
                         type serves the Gram only: s = 1 keeps the storage
                         type, so a narrower type is kept only if every n
                         has an admitted s > 1.                             */
} glm_batch_opts;

void glm_batch_opts_default(glm_batch_opts *o);

/*
 * Upload P independent problems (each converted like glm_create_ex, with
 * per-column scales) and run the autotuner for every problem with s = 0: for
 * each n among them it times one round of each (s, Gram kernel) -- s in
 * {1, 2, 4, 8, 16}; the SIMT kernel or tcgen05 tiles of 128 x 128 or
 * 128 x 256 -- on up to 32 of those problems (scratch iterates) and keeps the
 * fastest in samples per second.  Without opts.tau_bound the tuner only
 * chooses what leaves the exact-arithmetic iterate unchanged (s and the
 * kernel); with it, also the Gram operand type under that accuracy bound.
 * It never chooses b (part of the problem).  Returns GLM_EINVAL on a bad
 * descriptor (the message names the problem).  Blocks.
 */
int glm_batch_create(int P, const glm_problem_desc *descs,
                     const glm_batch_opts *opts, glm_batch *out);

/*
 * Run every problem's fit.  The run proceeds in rounds of K outer steps of
 * every problem: one gather launch, one Gram launch per group of problems
 * sharing (s, b, n), and one persistent chain launch whose CTAs take problems
 * from a device work queue, longest first; all rounds are captured once as a
 * CUDA graph and replayed by later runs.  xs: host array of P device FP32[n_p]
 * pointers, read as x0 and written with x_T.  status: host int[P] or NULL,
 * filled with GLM_OK or GLM_ENONFINITE per problem (flags are then cleared).
 * If a Gram launch gave up a bounded device wait, every entry is
 * GLM_ETIMEOUT and so is the return value (the iterates are then not
 * meaningful).  Blocks.
 */
int glm_batch_run(glm_batch bt, float *const *xs, int *status);

/* Per-problem risk F_p(x_p) (as glm_loss) into host double[P].  Blocks. */
int glm_batch_loss(glm_batch bt, float *const *xs, double *out);

/* The s, b and Gram operand type used for problem p. */
int glm_batch_choice(glm_batch bt, int p, int *s, int64_t *b, int *gram_dtype);

/* The autotuner's Theorem 1 prior (paper Sec. 5.2) on host data: for the
 * s b x n rows Y (host FP32, row-major, blocks of b rows) an upper bound on
 * ||H_L||_2 (H_L the strictly block-lower part of |Y| |Y|^T), from
 * sqrt(||H_L||_1 ||H_L||_inf), and the hypothesis figure
 *   tau_G = K_s L_sigma alpha (2 u_A + gamma_G) ||H_L||_2,
 * with K_s <= 1 / (1 - L_sigma alpha ||H_L||_2), gamma_G = 2 u_in +
 * gamma_n(2^-24), L_sigma 1/4 (logistic) or 1 (least squares); Poisson has
 * no Lipschitz bound (tau_G infinite unless u_in = 0).  Either output may be
 * NULL.  Host only, no device work. */
int glm_tau_prior(const float *Y, int64_t n, int s, int64_t b, double alpha, int loss,
                  double u_A, double u_in, double *hl_bound, double *tau);

/* The Gram kernel chosen for problem p (0 automatic, 1 SIMT, 2 tcgen05
 * 128 x 128 tiles, 3 tcgen05 128 x 256 tiles) and the estimated tau_G at the
 * chosen s and type (0 when not estimated: no tau_bound, or s = 1).  Host
 * outputs, either may be NULL. */
int glm_batch_choice_kernel(glm_batch bt, int p, int *gram_kernel, double *tau_g);

int glm_batch_destroy(glm_batch bt);

#ifdef __cplusplus
}
#endif
#endif /* GLM_H_ */
