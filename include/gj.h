/*
 * gj.h -- C ABI of the GB300 (sm_103a) Gauss-Jordan inversion library.
 *
 * The method is the Gauss-Jordan inversion of arXiv:1401.7962, Section 2: the pair
 * [A | D], initialised to [A | I] (eqs. 1-2), is reduced in n steps to [I | A^-1]
 * (eqs. 11-12).  Step k divides the pivot row by the pivot (eq. 14) and subtracts
 * multiples of it from every other row (eq. 15); the pivot is the entry of largest
 * magnitude among the candidates (observations 2-3) and the interchanges are undone
 * at the end; det A is the product of the pivots (eq. 13) with one sign change per
 * interchange.
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major.  Element (i, j) of A is A[i + j * lda].  The inverse
 *     is written with leading dimension n.
 *   - Floating point is IEEE binary64 unless an entry point says otherwise.
 *   - Pointers the caller passes are owned by the caller.  The library allocates only
 *     internal workspace (stream-ordered, freed before the call returns or, for
 *     stream-ordered calls, in stream order) and never frees caller memory.
 *   - Where a pointer is documented "host or device" the library inspects it
 *     (cudaPointerGetAttributes) and stages host buffers through device memory.
 *   - Steps are numbered from 0 (the paper numbers them from 1).  Pivot positions
 *     returned by the library are 0-based positions at the time of the step, i.e.
 *     the index of the row (column) interchanged with row (column) k at step k, as
 *     in the paper's program, which records the row it swaps with row k.
 *   - Errors are reported by return value.  Argument errors are detected before any
 *     launch.  A CUDA error is returned as GJ_ERR_CUDA; gj_last_error() then gives
 *     the CUDA error text.  There is no CPU fallback: every step of the inversion
 *     runs in the library's CUDA kernels.
 */
#ifndef GJ_H
#define GJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Result codes. */
typedef enum gj_status {
  GJ_OK = 0,
  GJ_SINGULAR = 1,       /* every candidate of some step was 0 or <= tau (obs. 2: "all
                            possibilities fail"); det_sign = 0, det_log2 = -inf */
  GJ_ZERO_PIVOT = 2,     /* pivot mode NONE met a pivot with |a_kk| <= tau; obs. 2 notes
                            this does not imply that A is singular */
  GJ_NONFINITE = 3,      /* a candidate of some step was NaN or infinite */
  GJ_NOT_CONVERGED = 4,  /* iterative refinement did not reach the tolerance */
  GJ_ERR_ARG = -1,       /* invalid argument; nothing was launched */
  GJ_ERR_CUDA = -2,      /* a CUDA call failed; see gj_last_error() */
  GJ_ERR_NOMEM = -3,     /* workspace allocation failed */
  GJ_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up (grid or cluster barrier) */
  GJ_ERR_UNSUPPORTED = -5 /* the combination of sizes and options has no kernel */
} gj_status;

/* Pivot selection (observations 2-3). */
typedef enum gj_pivot {
  GJ_PIVOT_NONE = 0,     /* pivot a_kk as it stands (eqs. 3-15 without interchanges) */
  GJ_PIVOT_PARTIAL = 1,  /* largest |a_ik| over the rows not yet used; ties to the
                            smallest row position */
  GJ_PIVOT_FULL = 2      /* largest |a_ij| over unused rows and columns; ties to the
                            smallest column position, then the smallest row position */
} gj_pivot;

/* Options for gj_invert_ex.  Zero-initialise and set what you need. */
typedef struct gj_opts {
  void* stream;          /* cudaStream_t to run on; NULL = the legacy default stream */
  double tau;            /* zero threshold of obs. 2: a step fails when the largest
                            candidate magnitude is <= tau.  Must be >= 0.  Default 0 */
  int32_t panel;         /* panel width b of the blocked path (16, 32 or 64); 0 = library
                            choice.  Ignored by the single-CTA path */
  int32_t path;          /* 0 = automatic; 1 = single-CTA shared-memory kernel (n <= 128);
                            2 = blocked panel + rank-b update (partial / none pivoting);
                            3 = unblocked multi-CTA (any pivoting, any n); 4 = one
                            thread-block cluster, rows spread over its CTAs (n <= 128) */
  int32_t update;        /* blocked path rank-b update engine: 0 = automatic (tensor cores for
                            n >= 512), 1 = FP64 FMA, 2 = FP64 emulated on BF16 tcgen05 tensor
                            cores (digit-split operands, exact FP32 partial sums, FP64
                            recombination; 128-column panels) */
  int32_t slices;        /* digit slices per operand for update 2: 1..8, 0 = 7 (8 bits per
                            slice; 7 slices round below 2^-56 of each row / column scale) */
  int32_t* piv_rows;     /* optional out [n], host or device: row position interchanged
                            with position k at step k */
  int32_t* piv_cols;     /* optional out [n], host or device: same for columns */
  double* pivots;        /* optional out [n], host or device: pivot value of step k (the
                            eq. 13 factors) */
  int64_t* fail_step;    /* optional out, host: failing step, -1 on success */
  int32_t lookahead;     /* blocked path with tensor-core update: 0 = automatic (on for
                            n >= 2048), 1 = off, 2 = on.  On: the next 128-column panel is
                            reduced on a second stream while the rank-128 update of the
                            other columns runs (same arithmetic, same results) */
  int32_t update_sms;    /* look-ahead: SMs of the persistent grid of the wide rank-128 update;
                            the panel stream keeps the others.  0 = library choice */
} gj_opts;

/*
 * gj_invert -- invert one n x n matrix (eqs. 1-15, obs. 2-3).
 *   n          order, n >= 0.  n == 0 returns GJ_OK with det_sign = 1, det_log2 = 0.
 *   A          [lda * n] input, host or device.  Not modified unless Ainv == A.
 *   lda        leading dimension of A, lda >= max(1, n).
 *   Ainv       [n * n] output, host or device, leading dimension n.  Ainv == A is allowed
 *              when lda == n (in-place inversion).  Contents are unspecified when the
 *              status is not GJ_OK.
 *   pivot_mode a gj_pivot value.
 *   det_sign   out (host, may be NULL): sign of det A, one of -1, +1; 0 on failure.
 *   det_log2   out (host, may be NULL): log2 |det A|; -inf on failure.
 * Synchronous: returns after the result is in Ainv.  Runs on the legacy default stream.
 */
gj_status gj_invert(int64_t n, const double* A, int64_t lda, double* Ainv, int pivot_mode, int* det_sign,
                    double* det_log2);

/* gj_invert_ex -- gj_invert with options (stream, tau, path, pivot record).  opts may be
 * NULL (same as gj_invert).  Synchronous with respect to the host: it waits on
 * opts->stream before returning, because det_sign / det_log2 are host values. */
gj_status gj_invert_ex(const gj_opts* opts, int64_t n, const double* A, int64_t lda, double* Ainv,
                       int pivot_mode, int* det_sign, double* det_log2);

/*
 * gj_solve -- solve A X = B by one Gauss-Jordan sweep of [A | B]: eqs. 3-10 of Section 2
 * with the columns of B in the place of D (each step scales the pivot row of A and B by
 * the pivot and eliminates the pivot column from every other row), pivoting as in
 * obs. 2-3 on the columns of A, exchanged unknowns restored at the end (obs. 3).  The
 * inverse itself is not formed.  det A (eq. 13) is returned as for gj_invert.
 *   n          order of A, n >= 0.  n == 0 returns GJ_OK with det_sign = 1, det_log2 = 0.
 *   nrhs       number of right-hand sides m >= 0 (m == 0: only det A is computed).
 *   A          [lda * n] input, host or device, column-major.  Not modified.
 *   B          [ldb * m] right-hand sides, host or device, column-major.  Not modified
 *              unless X == B.
 *   X          [ldx * m] output A^-1 B, host or device, column-major.  X == B is allowed
 *              when ldx == ldb.  Contents unspecified when the status is not GJ_OK.
 *   lda, ldb, ldx >= max(1, n).
 *   pivot_mode a gj_pivot value: none / partial run the blocked path (cluster panels and
 *              rank-b updates of the columns right of each panel and of B; tensor-core
 *              update for n >= 512 unless opts->update says otherwise), full runs the
 *              unblocked path.
 *   det_sign, det_log2  as for gj_invert.
 * Synchronous.  Status codes as for gj_invert; GJ_ERR_ARG also for opts->path == 1 (the
 * single-CTA kernel does not take right-hand sides).
 */
gj_status gj_solve(int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* B, int64_t ldb, double* X,
                   int64_t ldx, int pivot_mode, int* det_sign, double* det_log2);

/* gj_solve_ex -- gj_solve with options (stream, tau, path 2 or 3, update engine, pivot
 * record).  opts may be NULL.  Synchronous with respect to the host. */
gj_status gj_solve_ex(const gj_opts* opts, int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* B,
                      int64_t ldb, double* X, int64_t ldx, int pivot_mode, int* det_sign, double* det_log2);

/*
 * gj_invert_batched -- invert `count` independent matrices of uneven orders in one
 * persistent launch (one CTA per matrix; work items taken largest order first).  Each
 * matrix gets the method of Section 2 as gj_invert does: [A | I] reduced to [I | A^-1]
 * (eqs. 1-12) by pivot-row scaling (eq. 14) and elimination (eq. 15), pivots of largest
 * magnitude (obs. 2-3) with the interchanges undone at the end (obs. 3), det A as the
 * signed product of the pivots (eq. 13).  Batching itself is not in the paper.
 *   count      number of matrices, >= 0.
 *   nmax       host: upper bound of the orders (sizes the launch); 0 means 128.  Must
 *              be <= 128 (GJ_ERR_UNSUPPORTED otherwise).
 *   n          [count] device: orders, 0 <= n[m] <= nmax (a matrix outside that range
 *              gets status[m] = GJ_ERR_ARG and is not touched).
 *   A          [count] device array of device pointers: matrix m, column-major, ld n[m].
 *   Ainv       [count] device array of device pointers: output m, column-major, ld n[m].
 *              Ainv[m] == A[m] is allowed.
 *   pivot_mode a gj_pivot value, shared by all matrices.
 *   status     [count] device out: per-matrix gj_status.
 *   det_sign   [count] device out (may be NULL): -1, +1, or 0 on failure.
 *   det_log2   [count] device out (may be NULL): log2 |det|, -inf on failure.
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Stream-ordered: returns after enqueueing; no host synchronisation.  Needs a device
 * workspace of (count + 130) int32 taken from the stream-ordered allocator.
 */
gj_status gj_invert_batched(int64_t count, int32_t nmax, const int32_t* n, const double* const* A,
                            double* const* Ainv, int pivot_mode, int32_t* status, int8_t* det_sign,
                            double* det_log2, void* stream);

/*
 * gj_invert_batched_noalloc -- gj_invert_batched without any device allocation.
 * The paper has no counterpart.  Some callers cannot allocate device memory at the point
 * where they invert: real-time loops that must not take the allocator's locks or risk its
 * latency or an out-of-memory failure in the middle of a frame; programs that handed all
 * device memory to their own pool at start-up, so that a library allocation fails or
 * fragments it; code that by its own rules allocates only during initialisation.  This
 * entry point serves them.  Arguments, results and stream ordering are those of
 * gj_invert_batched.
 *   - Scratch (work order, histogram, queue counter) lives in a static device array of
 *     GJ_NOALLOC_MAX_COUNT + 131 int32 (about 4 MiB) that every GPU loading the library
 *     holds until the process exits.  count > GJ_NOALLOC_MAX_COUNT returns
 *     GJ_ERR_UNSUPPORTED before any launch (gj_last_error() says why).
 *   - The first call on a device looks up the array's device address (with that device
 *     current) and keeps it for later calls; the lookup is repeated when the device's
 *     context has changed since (after cudaDeviceReset, for instance).  Make that first
 *     call before any stream capture.
 *   - Every call shares the one array, which keeps the last call's contents: each call
 *     clears what must start at zero, and calls whose execution overlaps on the GPU (other
 *     streams, other host threads) race on it and must be serialised by the caller.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine.
 */
#define GJ_NOALLOC_MAX_COUNT 1048576
gj_status gj_invert_batched_noalloc(int64_t count, int32_t nmax, const int32_t* n, const double* const* A,
                                    double* const* Ainv, int pivot_mode, int32_t* status, int8_t* det_sign,
                                    double* det_log2, void* stream);

/*
 * gj_gemm_update_emulated -- C += L U in FP64 with the inner dimension K <= 128, computed
 * on BF16 tcgen05 tensor cores by exact digit splitting (the kernel of the blocked path's
 * rank-b update, the product form of eqs. 14-15 applied b steps at a time).
 *   M, N, K    sizes, M, N >= 0, 0 <= K <= 128.
 *   L          [ldl * K] device, column-major M x K, ldl >= M.
 *   U          [ldu * N] device, column-major K x N, ldu >= K.
 *   C          [ldc * N] device, column-major M x N, ldc >= M; updated in place.
 *   slices     balanced base-256 digits per operand entry, 1..8 (8 bits each; 7 or 8 reach
 *              FP64-level error: below 2^-8*slices relative to each row / column scale).
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Synchronous (waits for the stream: it reports device-side wait expiry as
 * GJ_ERR_TIMEOUT).  Uses a stream-ordered workspace of about
 * slices * (M + N) * 256 bytes.
 */
gj_status gj_gemm_update_emulated(int64_t M, int64_t N, int64_t K, const double* L, int64_t ldl, const double* U,
                                  int64_t ldu, double* C, int64_t ldc, int slices, void* stream);

/*
 * gj_invert_mixed -- inverse of an FP32 matrix by reduced-precision Gauss-Jordan plus
 * Newton-Schulz refinement (not in the paper; an accelerated variant of eqs. 14-15).
 *   X0: blocked Gauss-Jordan (partial pivoting) whose rank-128 updates run on the BF16
 *       tensor cores with x0_slices balanced 8-bit digit slices per operand (1: 8 bits,
 *       2: 16, 3: 24 bits of each row / column scale; 7: FP64 level); pivot search,
 *       division and log2|det| stay FP64.
 *   refinement: R = I - A X formed to FP64 level (exact 128-wide chunks of the emulated
 *       update), X <- X + X R with corr_slices slices, until
 *       ||A X - I||_F / (||A||_F ||X||_F) <= tol.  A rung that does not contract is
 *       replaced by the next (x0_slices -> max(x0_slices, 5) -> 7, each capped at 7); the
 *       middle rung is skipped when the first ||I - A X0||_F of the failed rung, times
 *       2^-8 per extra slice, stays above 1/4.
 *   n, A, lda   FP32 column-major input, device memory, lda >= max(1, n).
 *   X           [n * n] FP64 output, device memory, leading dimension n.
 *   x0_slices, corr_slices   1..8.   tol > 0.   max_iter >= 0 refinement steps per rung.
 *   resid_out, iters_out, rung_out   host outputs (may be NULL): final normalised residual,
 *               refinement steps of the last rung, index of that rung (0..2).
 *   det_sign, det_log2   host outputs (may be NULL): from the pivots of the last X0 (eq. 13),
 *               so as accurate as that X0: relative error of log2|det| about
 *               n kappa 2^-8S for S slices (FP64 level at S = 7 for a well-conditioned A).
 * Returns GJ_NOT_CONVERGED when no rung reaches tol (X holds the last iterate).
 * Synchronous.  Workspace: about 4 n^2 doubles plus the blocked path's.
 */
gj_status gj_invert_mixed(int64_t n, const float* A, int64_t lda, double* X, int x0_slices, int corr_slices,
                          double tol, int max_iter, double* resid_out, int* iters_out, int* rung_out, int* det_sign,
                          double* det_log2, void* stream);

/* Arithmetic of the reduced-precision first inverse of the mixed path (gj_invert_mixed_prec).
 * The update's operands are cut into S balanced 8-bit digits of each row / column scale and
 * the digit products with s + t <= S - 1 are summed exactly on the BF16 tensor cores, so S
 * sets how many significant bits of each operand take part: */
typedef enum gj_prec {
  GJ_PREC_FP64 = 0,          /* S = 7: 56 bits, the FP64-level update (no reduced precision) */
  GJ_PREC_BF16 = 1,          /* S = 1: 8 bits, BF16's significand; one product per term */
  GJ_PREC_FP16 = 2,          /* S = 2: 16 bits, covering FP16's 11-bit significand */
  GJ_PREC_SPLIT_BF16_3 = 3,  /* S = 2: a hi + lo pair of 8-bit digits and the three products
                                hi*hi + hi*lo + lo*hi (the split-BF16 3-term scheme) */
  GJ_PREC_TF32x3 = 4         /* S = 3: 24 bits, FP32's significand, as three TF32 products reach */
} gj_prec;
/* The digits are fixed point relative to the largest entry of their row (column), not
 * floating point per entry: an entry far below its row's largest keeps fewer significant
 * bits than BF16 / FP16 / TF32 rounding would leave it, with the same normwise error. */

/*
 * gj_invert_mixed_prec -- gj_invert_mixed with the first inverse's arithmetic named by a
 * gj_prec value (and correction products of 4 slices, 32 bits).  Not in the paper.
 * Arguments, outputs, ladder and status as for gj_invert_mixed; GJ_ERR_ARG for an unknown
 * prec.  GJ_PREC_FP64 inverts at the FP64 level first, so refinement only polishes.
 */
gj_status gj_invert_mixed_prec(int64_t n, const float* A, int64_t lda, double* X, int prec, double tol, int max_iter,
                               double* resid_out, int* iters_out, int* rung_out, int* det_sign, double* det_log2,
                               void* stream);

/*
 * gj_invert_mixed_batched -- gj_invert_mixed over a batch of FP32 matrices of different
 * orders (not in the paper: batching and the precision ladder are outside its method).
 * A pool of host workers, each with its own CUDA stream and workspace, takes the
 * matrices largest first; each matrix climbs its own ladder from its own residuals.
 *   count      number of matrices (>= 0).
 *   n, lda     [count] host arrays: order (>= 0) and leading dimension (>= max(1, n)).
 *   A          [count] host array of device pointers: FP32 column-major matrices.
 *   X          [count] host array of device pointers: FP64 outputs, leading dimension n.
 *              A and X of different matrices must not overlap.
 *   x0_slices, corr_slices, tol, max_iter   as gj_invert_mixed, for every matrix.
 *   workers    host workers (= concurrent streams), 0..64; 0 chooses min(count, 16).
 *   status     [count] host out (may be NULL): gj_invert_mixed's status per matrix.
 *   resid, iters, rung, det_sign, det_log2   [count] host outs (may be NULL): per-matrix
 *              values of gj_invert_mixed's outputs.
 *   stream     the batch starts after the work queued on it before the call.
 * Returns GJ_ERR_ARG (nothing launched) for a bad count, order, leading dimension, null
 * pointer of a non-empty matrix or option; otherwise the first negative per-matrix status in
 * matrix order, else the first non-OK one (e.g. GJ_NOT_CONVERGED), else GJ_OK.
 * Synchronous.  Workspace: gj_invert_mixed's, per worker, for the matrix it holds.
 */
gj_status gj_invert_mixed_batched(int64_t count, const int32_t* n, const int32_t* lda, const float* const* A,
                                  double* const* X, int x0_slices, int corr_slices, double tol, int max_iter,
                                  int workers, int32_t* status, double* resid, int32_t* iters, int32_t* rung,
                                  int8_t* det_sign, double* det_log2, void* stream);

/* A batched plan fixes the orders (host copy given at creation), precomputes the
 * largest-first work order and launch shape, and can be replayed as a CUDA graph.  Every
 * matrix of a planned batch is inverted by the method of Section 2 (eqs. 1-15, obs. 2-3,
 * det by eq. 13), as in gj_invert_batched; the plan only schedules that work. */
typedef struct gj_plan gj_plan;

/*
 * gj_batched_plan_create -- plan a batch.
 *   plan     out: the new plan.
 *   count    number of matrices.
 *   n_host   [count] host: orders (0 <= n <= 128).
 *   pivot_mode  gj_pivot value.
 * The plan owns device copies of the orders and the work order.
 */
gj_status gj_batched_plan_create(gj_plan** plan, int64_t count, const int32_t* n_host, int pivot_mode);

/* Kernel variants of a planned batch (one per order bin). */
typedef enum {
  GJ_BATCHED_WARP4 = 0,   /* one warp per matrix, 4 warps per CTA (orders <= 32, not full pivoting) */
  GJ_BATCHED_WARP8 = 1,   /* one warp per matrix, 8 warps per CTA (same limits) */
  GJ_BATCHED_CTA64 = 2,   /* one CTA of 64 threads per matrix, matrix in shared memory */
  GJ_BATCHED_CTA128 = 3,  /* ... 128 threads */
  GJ_BATCHED_CTA256 = 4,  /* ... 256 threads */
  GJ_BATCHED_CTA512 = 5   /* ... 512 threads */
} gj_batched_variant;

/*
 * gj_batched_plan_create_ex -- plan a batch with the kernel variant of each order bin
 * (orders 0-8, 9-16, 17-24, 25-32, 33-48, 49-64, 65-96, 97-128) chosen by an autotuner.
 * The paper has no counterpart (batching is outside its method).
 *   tune_cache  host path of a text file (may be NULL): choices recorded there for this
 *               device, pivot mode and bin are used first; new measurements are appended
 *               (one line per bin: "gj-tune-v1 <device>_sm<SMs> <mode> <lo> <hi>
 *               <variant> <microseconds>").  Within a process, measured choices are also
 *               remembered in memory and reused by later plans.
 *   variant     -1: autotune (time every applicable gj_batched_variant on up to 2048
 *               synthetic matrices of the bin's orders, keep the fastest); otherwise that
 *               variant for every bin it applies to (CTA128 / CTA256 elsewhere).
 * Synchronous (it runs and times kernels on the legacy default stream while tuning).
 * Other arguments and errors as for gj_batched_plan_create; GJ_ERR_ARG for a variant
 * >= 6.
 */
gj_status gj_batched_plan_create_ex(gj_plan** plan, int64_t count, const int32_t* n_host, int pivot_mode,
                                    const char* tune_cache, int32_t variant);

/*
 * gj_batched_plan_bins -- describe a plan's order bins (host arrays of max_bins entries,
 * each may be NULL): orders lo..hi, number of matrices, chosen gj_batched_variant and the
 * tuning time of that variant on the sample in microseconds (-1 when not measured in
 * this call).  Returns the number of non-empty bins (0 for a NULL plan).
 */
int32_t gj_batched_plan_bins(const gj_plan* plan, int32_t* lo, int32_t* hi, int64_t* count, int32_t* variant,
                             float* tuned_us, int32_t max_bins);

/*
 * gj_batched_plan_execute -- run a planned batch on `stream`: every matrix is inverted by
 * eqs. 1-15 with the pivoting of obs. 2-3 and its determinant formed by eq. 13, as in
 * gj_invert_batched.  Argument meaning as in gj_invert_batched (device arrays).  With use_graph != 0 the launch sequence is
 * captured once into a CUDA graph for these pointer arrays and replayed afterwards
 * (re-captured if the pointers or stream change).
 */
gj_status gj_batched_plan_execute(gj_plan* plan, const double* const* A, double* const* Ainv, int32_t* status,
                                  int8_t* det_sign, double* det_log2, void* stream, int use_graph);

/* gj_batched_plan_destroy -- free a plan (NULL is allowed). */
void gj_batched_plan_destroy(gj_plan* plan);

/* Kernel timing for benchmarks (no counterpart in the paper).  Between
 * gj_profile_begin() and gj_profile_end() the library records a CUDA event pair on the
 * launching stream around each launch of its dominant kernels and counts every kernel
 * it launches.  gj_profile_end() waits for those events and fills up to max_entries
 * aggregates (one per kernel name, `kernel` points to static text); it returns the
 * number of aggregates and stores the total number of kernel launches in *launches.
 * Process-wide state; not meant to be used from several threads at once. */
typedef struct gj_profile_entry {
  const char* kernel;
  int64_t launches;
  double total_ms;   /* summed device time of those launches */
  double flops;      /* summed algorithmic FLOP count declared by the launch site */
  double bytes;      /* summed algorithmic DRAM bytes declared by the launch site */
} gj_profile_entry;

gj_status gj_profile_begin(void);
int gj_profile_end(gj_profile_entry* out, int max_entries, int64_t* launches);

/*
 * gj_trim_memory -- return the device memory the library keeps between calls.  Workspace
 * is taken, stream-ordered, from a memory pool of the library's own on each device that
 * keeps freed memory for later calls (up to the largest amount one call has needed).  The
 * paper has no counterpart.  Call it with no library work in flight.
 */
gj_status gj_trim_memory(void);

/*
 * gj_set_wait_limit_ns -- limit, in nanoseconds, of the pipeline waits of the tensor-core
 * update kernel (gj_gemm_update_emulated, and the update of the blocked path and of
 * gj_invert_mixed); 0 restores the default of 2 s.  The paper has no counterpart: the limit
 * exists so that a test can make such a wait expire and check what follows.  On expiry
 * the kernel stops issuing work, waits (with the full 2 s limit) for the tile loads and
 * MMAs it already issued, frees its tensor memory and exits; the call returns
 * GJ_ERR_TIMEOUT.  Process-wide, read at every launch; set it with no library work in
 * flight.  The waits of the cluster kernels keep their fixed 2 s limit.
 */
gj_status gj_set_wait_limit_ns(uint64_t ns);

/*
 * gj_measure_peaks -- arithmetic throughput of the current GPU, measured with probe kernels
 * of independent chains on every SM (no memory traffic): FP64 FMA, FP64 mma.sync (m8n8k4)
 * and FP32 FMA, in GFLOP/s (best of five timed launches after a warm-up).  The paper has no
 * counterpart; these are the denominators of the benchmark's rooflines for FP64 work.
 * Synchronous; allocates 64 bytes of device memory for the duration of the call.
 */
typedef struct gj_peaks {
  double fp64_fma_gflops;
  double fp64_mma_gflops;
  double fp32_fma_gflops;
  int32_t sm_count;
  double max_clock_mhz;
} gj_peaks;
gj_status gj_measure_peaks(gj_peaks* out);

/* gj_status_string -- static text for a status code. */
const char* gj_status_string(int status);

/* gj_last_error -- text of the last CUDA error seen by this thread ("" if none). */
const char* gj_last_error(void);

/* gj_version -- library version string. */
const char* gj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GJ_H */
