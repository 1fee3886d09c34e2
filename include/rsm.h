/*
 * rsm.h - C ABI of the GB300 Random SubMatrix (RSM) library (librsm.so).
 *
 * RSM (Y. Liu, arXiv 1411.0814) computes a rank-r decomposition Y ~ U V^T of an
 * m x n matrix Y with missing entries (eq. problem, Section I):
 *   step 2 (Section IV-A): repeatedly draw l columns (method M1, Section III),
 *          keep the rows known in all of them, and take the l - r right singular
 *          vectors of the smallest singular values of that submatrix;
 *   step 3: accumulate M = Xi Xi^T = sum xi xi^T (eq. XI and the text after
 *          eq. solve.barV_L2_norm), take V = the r smallest eigenvectors of M,
 *          then solve U row by row by least squares (eq. solve.barU).
 *
 * Conventions shared by every entry point:
 *   - Matrices are column-major.  "device" pointers are CUDA device memory of
 *     the handle's (or the current) device; "host" pointers are ordinary host
 *     memory.  The caller owns every pointer it passes; the library never frees
 *     or retains one past the call (rsm_submit: past completion, see there).
 *   - No C++ exception crosses this boundary; every failure is a status code.
 *   - Arguments are validated before any launch; on RSM_ERR_INVALID_ARG nothing
 *     was launched and no output was written.
 *   - A "stream" argument is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Stage entry points are asynchronous on that stream.
 */
#ifndef RSM_H_
#define RSM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rsm_status {
  RSM_OK = 0,
  RSM_ERR_INVALID_ARG = 1,          /* a size, pointer, leading dimension or enum is out of range */
  RSM_ERR_NO_MEMORY = 2,            /* footprint above the handle's HBM budget, or cudaMalloc failed */
  RSM_ERR_UNDERDETERMINED = 3,      /* no accepted trial, or M has more than r numerically zero
                                       eigenvalues (rank(Xi) < n - r, Section III before eq.
                                       solve.barV); V and U are not written */
  RSM_ERR_ROWS_UNDERDETERMINED = 4, /* V and U are written, but some rows of Y have fewer than r
                                       known entries; those rows got the minimum-norm solution */
  RSM_ERR_TIMEOUT = 5,              /* a bounded device-side or host-side wait ran out */
  RSM_ERR_CANCELLED = 6,            /* the request was cancelled before it ran */
  RSM_ERR_CUDA = 7,                 /* a CUDA runtime call failed (message: rsm_last_error) */
  RSM_ERR_NOT_IMPLEMENTED = 8,      /* the requested option exists in the ABI but not in this build */
  RSM_PENDING = 9,                  /* rsm_poll: the request has not finished */
  RSM_ERR_QUEUE_FULL = 10           /* rsm_submit: the admission queue is full; retry later */
} rsm_status;

/* Element type of Y. */
typedef enum rsm_dtype { RSM_F64 = 0, RSM_F32 = 1 } rsm_dtype;

/* Arithmetic of the two bulk contractions: the per-trial Gram A^T A of step 2
 * (gram_prec) and the accumulation of the per-row normal equations
 * N_i = sum v_j v_j^T, b_i = sum y_ij v_j of step 3 (solve_prec).
 *   RSM_PREC_F64:   FP64 multiply-add throughout.
 *   RSM_PREC_F32X2: products and sums carried as unevaluated pairs of FP32
 *                   values (about 48 significant bits) on the FP32 pipes
 *                   (gram_prec only).
 *   RSM_PREC_F32:   FP32 multiply-add (the reduced-precision form); for FP32 Y
 *                   and r <= 21 the N_i accumulate on the tensor cores (TF32
 *                   head + tail of v_a v_b, FP32 accumulation, ~2^-22).
 * In every mode: the l x l eigenproblems (minor vectors) are refined in FP64;
 * M is summed in 64-bit fixed point and stored in FP64; the eigensolve of M
 * iterates with M X in FP32 pairs (~2^-44) and ends with a refinement pass
 * (two with the FP64 factor) whose products M X, Rayleigh-Ritz step and
 * residual are IEEE FP64;
 * the r x r Cholesky factorisations and triangular solves for U are FP64. */
typedef enum rsm_prec { RSM_PREC_F64 = 0, RSM_PREC_F32X2 = 1, RSM_PREC_F32 = 2 } rsm_prec;

/* Submatrix sampler (Section III, methods M1 and M2). */
typedef enum rsm_variant {
  RSM_COLS_RANDOM = 0,   /* M1: l distinct columns, uniform without replacement (Floyd's algorithm) */
  RSM_COLS_ADJACENT = 1, /* M1: l contiguous columns s..s+l-1, s uniform in [0, n-l] */
  RSM_ROWS_RANDOM = 2    /* M2: k distinct rows (the same sampler over m), then the columns known in all */
} rsm_variant;

typedef struct rsm_config {
  int32_t device;            /* CUDA device ordinal */
  int32_t max_slots;         /* requests the serving loop runs concurrently (0 -> 4) */
  size_t hbm_budget_bytes;   /* library-owned device memory the handle may hold (0 -> 80% of free) */
  uint64_t wait_timeout_ns;  /* bound on every blocking wait of the serving loop (0 -> 10 s) */
  void* stream;              /* cudaStream_t used by rsm_decompose and rsm_decompose_batch (NULL -> a
                                stream the handle creates; see rsm_decompose for the ordering) */
  uint32_t fault_inject;     /* host-side fault injection for tests (RSM_FAULT_* bits); 0 in production */
  uint32_t reserved;
} rsm_config;

/* Fault injection bits for tests (rsm_config.fault_inject).  No kernel is
 * ever made to fault, trap or hang: the first three act on the host; the last
 * gives one bounded device-side wait a condition that nothing meets, so that
 * the wait runs out exactly as a lost dependency would. */
#define RSM_FAULT_ADMISSION 0x1u    /* every admission check reports the budget exhausted */
#define RSM_FAULT_ALLOC 0x2u        /* the next workspace allocation reports failure */
#define RSM_FAULT_STALL 0x4u        /* the scheduler withholds work, so waits run out (TIMEOUT) */
#define RSM_FAULT_DEVICE_WAIT 0x8u  /* the eigen stage's factor launch waits (with a short bound) for a
                                       state word nothing sets: the launch is abandoned and the result
                                       is RSM_ERR_TIMEOUT; the handle stays usable */

typedef struct rsm_problem {
  int64_t m, n;          /* Y is m x n; the paper assumes m >= n (Section II) */
  int32_t r;             /* target rank, 1 <= r < n */
  int32_t l;             /* columns per submatrix, r < l <= n; 0 -> r + 1 (Section IV-A step 1) */
  int32_t n_minor;       /* minor vectors kept per submatrix, 1..l-r; 0 -> l - r (Section III) */
  int32_t variant;       /* rsm_variant */
  int64_t trials;        /* number of submatrix draws I >= 1 (rejected draws count) */
  uint64_t seed;         /* Philox key of the column sampler */
  uint32_t problem_id;   /* second counter word of the sampler, distinguishes problems */
  int32_t y_dtype;       /* rsm_dtype of Y */
  int32_t gram_prec;     /* rsm_prec of the per-trial Gram */
  int32_t solve_prec;    /* rsm_prec of the per-row normal equations */
  const void* Y;         /* device, m x n column-major, leading dimension ldy >= m; read only */
  int64_t ldy;
  const uint8_t* W;      /* device, m x n column-major bytes, 1 = known (eq. problem); read only */
  int64_t ldw;
  double* U;             /* device output m x r (ldu >= m), or NULL to stop after V */
  int64_t ldu;
  double* V;             /* device output n x r (ldv >= n), orthonormal columns */
  int64_t ldv;
  /* Optional device outputs for inspection (NULL = not written). */
  int32_t* debug_cols;       /* trials x l, row-major: the sorted column set of each trial */
  int32_t* debug_row_counts; /* trials: rows kept by each trial (p_t), rejected trials included */
  double* debug_Z;           /* trials x l x n_minor: minor vectors (zero for rejected trials) */
  double* debug_M;           /* n x n: the accumulated M */
  /* Trial planning and coverage (Section III, Theorem 3; Section IV-A step 1). */
  double epsilon;            /* used when trials == 0: the library counts the known entries (density rho)
                                and draws ceil(rsm_plan_trials(...).trials) submatrices, so that each known
                                entry is visited with probability >= epsilon (0 < epsilon < 1); debug_cols,
                                debug_row_counts and debug_Z must then be NULL.  rsm_submit needs trials >= 1. */
  int32_t coverage;          /* 1: count the known entries that the accepted draws visit (rsm_result.coverage) */
  int32_t norm;              /* 2 (or 0): the L2 forms of eqs. solve.barV and solve.barU; 1: their L1 forms
                                (Section IV-A eq. solve.barV_L1_norm; column variants, r <= 8), read as
                                min sum_j ||V^T xi_j||_2 over the null vectors (rotation-invariant) and
                                per-row least absolute deviations, each by irls_iters steps of iteratively
                                reweighted least squares from the L2 solution.  All problems of a batch
                                share it. */
  int32_t irls_iters;        /* L1 forms: reweighting steps of V-hat and of U-hat (0 -> 8) */
  int32_t reserved;
  double irls_delta_v;       /* L1 form of V-hat: weights delta / max(||V^T xi||, delta) (0 -> 1e-4); a
                                smaller delta is more robust to outliers but leaves the reweighted M less
                                well conditioned */
  double irls_delta_u;       /* L1 form of U-hat: delta = irls_delta_u * e of the L2 solution (0 -> 1e-3) */
  uint32_t* debug_visited;   /* optional device output with coverage = 1: the visited entries as a packed
                                mask, n columns of ldb = 4 ceil(ceil(m / 32) / 4) uint32 words, bit (i mod 32)
                                of word i / 32 of column j set iff entry (i, j) was visited */
} rsm_problem;

typedef struct rsm_result {
  int32_t status;                /* rsm_status of the decomposition */
  int32_t n_eig;                 /* eigenvalues of M reported in eig_M */
  int64_t accepted_trials;       /* trials that kept at least l rows */
  int64_t rows_underdetermined;  /* rows with fewer than r known entries */
  int64_t rows_selected;         /* sum over all trials of the rows kept (p_t) */
  int64_t kernel_launches;       /* CUDA kernels this call launched (whole batch) */
  int32_t eig_factor_bits;       /* 32 or 64: precision of the Cholesky preconditioner used for M */
  int32_t eig_iterations;        /* preconditioned block iterations of the eigensolve of M (last attempt) */
  double eig_M[32];              /* smallest eigenvalues of M, ascending: the first r to FP64 working
                                    accuracy; the rest are Ritz values of the solver's extra block
                                    vectors (upper bounds on lambda_{r+1}, ..., loosely converged) */
  double eig_residual;           /* largest ||M v - lambda v|| over the r returned vectors */
  double e_known_rms;            /* eq. (ep): RMS residual over the known entries (NaN if U is NULL) */
  float stage_ms[12];            /* device time per stage (CUDA events on the launching stream):
                                    0 setup (plan upload, zeroing), 1 pack_mask and sample_cols
                                    (one launch), 2 empty (0),
                                    3 select+Gram, 4 minor vectors + scatter into M, 5 eigensolve of M,
                                    6 solve U, 7 residual e, 8 total; 9-11 reserved.  A batch reports
                                    the batch's times in every result. */
  double queue_ms;               /* serving: submit -> start */
  double run_ms;                 /* serving: start -> finish */
  double coverage;               /* with rsm_problem.coverage: visited / known entries, else NaN */
  int64_t trials;                /* submatrix draws made (the planned count when rsm_problem.trials was 0) */
} rsm_result;

typedef struct rsm_handle rsm_handle;

/* Library version string (static storage). */
const char* rsm_version(void);
/* sizeof of the ABI structs, for bindings to check their layout:
 * which = 0 rsm_config, 1 rsm_problem, 2 rsm_result; 0 for other values. */
size_t rsm_struct_size(int32_t which);
/* Trial-count plan (Section III, Theorem 3 and the first line of its proof):
 * the probability that one draw visits a given known entry, and the number of
 * draws that visits every known entry with probability at least epsilon. */
typedef struct rsm_trial_plan {
  double p_visit;          /* exact per-draw visit probability for density rho (binomial expectation) */
  double trials;           /* ln(1 / (1 - epsilon)) / p_visit */
  double p_visit_theorem3; /* Theorem 3's closed-form lower bound of p_visit (through Lemma 1) */
  double trials_theorem3;  /* Theorem 3's upper bound ln(1 / (1 - epsilon)) / p_visit_theorem3 */
} rsm_trial_plan;

/* Plan the number of draws for an m x n Y with known density rho, rank r and
 * submatrix size `size` (l columns for M1 variants, k rows for M2), so that each
 * known entry is visited with probability at least epsilon (Section IV-A step 1).
 * Pure host arithmetic.  RSM_ERR_INVALID_ARG unless 0 < rho <= 1, r < size,
 * size <= n (M1) or <= m (M2), 0 < epsilon < 1. */
int32_t rsm_plan_trials(int64_t m, int64_t n, double rho, int32_t r, int32_t size, int32_t variant, double epsilon,
                        rsm_trial_plan* out);

/* Text for a status code (static storage). */
const char* rsm_status_string(int32_t status);
/* Message of the last failure on the calling thread (thread-local storage). */
const char* rsm_last_error(void);

/* Create a handle bound to config->device (config may be NULL for defaults).
 * On success *out owns the device workspace and the serving threads. */
int32_t rsm_create(const rsm_config* config, rsm_handle** out);
/* Wait for in-flight work (bounded by the wait timeout), then free everything
 * the handle owns.  NULL is ignored. */
void rsm_destroy(rsm_handle* h);

/* Device bytes a problem needs beyond the caller's Y, W, U and V: the packed
 * mask, the sampled columns, per-trial Grams and minor vectors, M and the
 * eigensolver workspace.  0 if the problem is invalid.  Pure host arithmetic. */
size_t rsm_footprint_bytes(const rsm_problem* p);

/* Synchronous decomposition (Section IV-A steps 1-3).  Runs every stage on the
 * handle's stream and returns after the stream is synchronised.  res (host)
 * may be NULL.  Returns the same status as res->status.
 * Ordering: the first read of Y and W comes after all work already enqueued
 * on the handle's stream (rsm_config.stream).  A handle that created its own
 * stream instead starts after all work enqueued so far on the legacy default
 * stream, which covers the caller's blocking streams but NOT streams created
 * with cudaStreamNonBlocking: inputs produced on such a stream must be
 * complete (or the handle created on that stream).  U, V and the debug
 * outputs are complete when the call returns. */
int32_t rsm_decompose(rsm_handle* h, const rsm_problem* p, rsm_result* res);

/* Batched decomposition of count independent problems (host array ps).  The
 * problems share the launches of every stage (one launch covers all trials of
 * all problems).  res (host) holds count results or is NULL.  Returns RSM_OK if
 * every problem succeeded, else the first failing status. */
int32_t rsm_decompose_batch(rsm_handle* h, const rsm_problem* ps, int32_t count, rsm_result* res);

/* Gram-stage autotuning.  The Gram stage (Section IV-A steps 2-3: the rows
 * known in all drawn columns and the Gram matrix of each submatrix) has two
 * schedules: row slabs of Y small enough to stay in L2 while every draw reads
 * them (the default, 32 MiB), and one warp per submatrix reading Y directly.
 * rsm_autotune times, on the caller's problem p, the default, the slab
 * schedule at 8, 16, 32 and 64 MiB of Y per slab with the kernel's register-
 * derived CTAs per SM (and one fewer, where that build has more registers per
 * thread), and the per-submatrix schedule: `reps`
 * timed runs each (0 -> 3) after one untimed run, a 256 MiB write between runs
 * to evict L2, the Gram stage's device time (stage_ms[3]) minimum over reps.
 * The fastest becomes the handle's choice for every later problem with the same
 * key (gram_prec, y_dtype, l, n, and ceil(log2 m)), in rsm_decompose, the
 * batch and the serving calls.  The results do not depend on the choice beyond
 * rounding: M is accumulated in fixed point, but the per-submatrix schedule
 * sums the Gram in another order.
 * p's V is overwritten (U and the debug outputs are not touched); trials == 0
 * is planned as in rsm_decompose.  Runs on the handle's stream like
 * rsm_decompose and synchronises it.  RSM_ERR_INVALID_ARG for the rows variant
 * (it has no Gram stage) or an invalid problem; the status of a failing run
 * otherwise.  *out (may be NULL) receives the choice and its timings. */
typedef struct rsm_tune {
  int32_t schedule;   /* 0: L2-resident row slabs, 1: one warp per submatrix */
  int32_t slab_mib;   /* MiB of Y per slab (schedule 0) */
  int32_t variant;    /* 0: register-derived CTAs per SM, 1: one fewer (schedule 0) */
  int32_t candidates; /* choices timed */
  double gram_ms;     /* Gram-stage time of the choice (ms) */
  double default_ms;  /* Gram-stage time of the default (ms) */
} rsm_tune;
int32_t rsm_autotune(rsm_handle* h, const rsm_problem* p, int32_t reps, rsm_tune* out);
/* 1 and *out (may be NULL) filled when the handle holds a choice for p's key,
 * 0 when not, -RSM_ERR_INVALID_ARG for a NULL handle or problem. */
int32_t rsm_autotune_lookup(rsm_handle* h, const rsm_problem* p, rsm_tune* out);
/* Forget every choice (later problems take the defaults). */
int32_t rsm_autotune_clear(rsm_handle* h);
/* Write the handle's choices to a text file (one line per key), or add those
 * of a file written so to the handle (an entry replaces one with the same
 * key).  A malformed file loads nothing: RSM_ERR_INVALID_ARG, message names
 * the line.  Choices are per device model and build: a file is a cache, not a
 * portable setting. */
int32_t rsm_autotune_save(rsm_handle* h, const char* path);
int32_t rsm_autotune_load(rsm_handle* h, const char* path);

/* Serving: enqueue a problem.  The problem struct is copied; Y, W, U, V and the
 * debug buffers must stay valid until rsm_poll reports a final status.  A
 * request is admitted when a slot is free and its footprint fits the budget;
 * requests run concurrently on separate streams.  *ticket identifies it.
 * Ordering: the request's first read of Y and W comes after all work that was
 * enqueued on `stream` (a cudaStream_t of the handle's device; NULL = the
 * legacy default stream) before this call; its outputs are complete once
 * rsm_poll / rsm_wait report a final status. */
int32_t rsm_submit_on(rsm_handle* h, const rsm_problem* p, void* stream, uint64_t* ticket);
/* rsm_submit_on with the legacy default stream. */
int32_t rsm_submit(rsm_handle* h, const rsm_problem* p, uint64_t* ticket);
/* Non-blocking: RSM_PENDING while queued or running, else the final status
 * (res filled).  A finished ticket can be polled again until rsm_release. */
int32_t rsm_poll(rsm_handle* h, uint64_t ticket, rsm_result* res);
/* Blocking form of rsm_poll, bounded by timeout_ns (0 -> the handle's wait
 * timeout); returns RSM_ERR_TIMEOUT if the request is still pending then. */
int32_t rsm_wait(rsm_handle* h, uint64_t ticket, uint64_t timeout_ns, rsm_result* res);
/* Cancel a request that has not started (RSM_ERR_CANCELLED becomes its status);
 * a running request is not interrupted and RSM_ERR_INVALID_ARG is returned. */
int32_t rsm_cancel(rsm_handle* h, uint64_t ticket);
/* Forget a finished ticket. */
int32_t rsm_release(rsm_handle* h, uint64_t ticket);

/* ---- Stage entry points: one hot-path kernel each, asynchronous on stream ---- */

/* Pack the mask (Section IV-A: submatrix extraction needs only logical tests on
 * W).  W: device m x n bytes (ldw >= m), nonzero = known.  bits: device
 * n x ldb uint32 words, column c at bits + c*ldb, bit (i mod 32) of word i/32 is
 * W[i, c] != 0; ldb >= ceil(m/32); words past the last row are zero. */
int32_t rsm_pack_mask(const uint8_t* W, int64_t ldw, int64_t m, int64_t n, uint32_t* bits, int64_t ldb,
                      void* stream);

/* Draw the column sets of trials t0..t0+count-1 (Section III, M1; Section II:
 * the indices of a list are distinct).  Word w of trial t is lane (w mod 4) of
 * Philox4x32-10 with key (seed mod 2^32, seed >> 32) and counter
 * (t mod 2^32, problem_id, w div 4, t >> 32); a draw in [0, k) is
 * (word * k) >> 32.  RANDOM: Floyd's algorithm, draw number d = 0..l-1 picks x
 * in [0, n-l+d] from word d and inserts n-l+d if x is already taken; ADJACENT:
 * s from word 0 in [0, n-l].  cols: device count x l int32, each row ascending. */
int32_t rsm_sample_columns(int64_t n, int32_t l, int64_t t0, int64_t count, uint64_t seed, uint32_t problem_id,
                           int32_t variant, int32_t* cols, void* stream);

/* Row lists R_t (Section III, M1: the rows whose entries in all chosen columns
 * are known) for count trials.  bits/ldb: packed mask (rsm_pack_mask).  cols:
 * device count x l.  row_offsets: device count+1 int64, exclusive prefix of the
 * caller's capacity per trial; rows: device int32 array of row_offsets[count]
 * entries.  row_counts: device count int32, receives p_t; a trial whose p_t
 * exceeds its capacity writes only the first rows (ascending). */
int32_t rsm_select_rows(const uint32_t* bits, int64_t ldb, int64_t m, const int32_t* cols, int32_t l, int64_t count,
                        const int64_t* row_offsets, int32_t* rows, int32_t* row_counts, void* stream);

/* The eigen stage alone (row a7; Section III, eq. solve.barV_L2_norm: V-hat =
 * the eigenvectors of M for its r smallest eigenvalues) on a caller-supplied
 * M, with the same solver, precision and acceptance as rsm_decompose.
 * M: device n x n symmetric (FP64, leading dimension n), read only, copied
 * into the handle's workspace.  V: device output n x r (ldv >= n), orthonormal
 * columns.  res (host, may be NULL): status, eig_M (the kx smallest
 * eigenvalues, ascending), eig_residual (largest ||M v - lambda v|| of the r
 * returned vectors, FP64), eig_factor_bits, eig_iterations, stage_ms.  The
 * status is RSM_ERR_UNDERDETERMINED when lambda_{r+1} <= 1e-12 trace(M) (more
 * than r numerically zero eigenvalues); V is written either way.
 * 2 <= n <= 32768, 1 <= r < min(n, 32).  Synchronous on the handle's stream,
 * ordered like rsm_decompose. */
int32_t rsm_eig_smallest(rsm_handle* h, const double* M, int64_t n, int32_t r, double* V, int64_t ldv,
                         rsm_result* res);

/* The FP64 reciprocal, inverse square root and square root that the library's
 * small dense kernels use (pivots, rotations, substitutions; the r x r solves
 * of Section III eq. solve.barU): each is seeded by the FP32 hardware
 * approximation and refined by Newton-Raphson steps in FP64, so the result may
 * differ from the correctly rounded one in the last bits.  Evaluated for tests
 * that bound that difference.  x: device array of count doubles; out: device
 * array of 3 count doubles receiving 1/x, then 1/sqrt(x) (0 for x <= 0), then
 * sqrt(x) (0 for x < 0).  Asynchronous on stream. */
int32_t rsm_check_fp64_math(const double* x, int64_t count, double* out, void* stream);

/* Gather probe (measurement only; the paper has no counterpart): the ceilings of
 * the row-slab Gram's access pattern.  blocks x 256 threads each issue
 * per_thread (a multiple of 16) 4-byte loads; each group of per_line (1 or 4)
 * consecutive lanes reads distinct 32-byte sectors of one pseudo-random
 * 128-byte line of buf (device, elems floats, a power of two >= 1024; size it to
 * stay in L2).  per_line = 1: every load is its own line (the L1's per-line
 * rate); per_line = 4: four sectors per line (the L2's sector rate).  out:
 * device, blocks x 256 floats, written only to keep the loads alive.  Time it
 * with events on `stream`: loads per second = blocks 256 per_thread / time. */
int32_t rsm_probe_gather(const float* buf, int64_t elems, int64_t blocks, int32_t per_thread, int32_t per_line,
                         float* out, void* stream);

/* e = sqrt(sum over known (y_ij - u_i . v_j)^2 / number of known entries) for a
 * given U and V, computed without allocating device memory.  The paper has no
 * counterpart: this entry point is for callers that cannot allocate at the
 * point where they need the error - a process whose device memory is owned by
 * its own pool and may not be taken through the CUDA runtime allocator, or a
 * latency-bound loop that must not pay the device synchronisation that
 * cudaMalloc / cudaFree can cause.
 * Y: device m x n (ldy >= m) of y_dtype; W: device m x n bytes (ldw >= m),
 * nonzero = known; U: device m x r FP64 (ldu >= m); V: device n x r FP64
 * (ldv >= n); 1 <= r <= 32.  e: device pointer to one double that receives e.
 * Asynchronous on stream.  Scratch is a fixed array inside the library (256 KiB
 * per device, held until the process exits): m above 4,194,304 rows returns
 * RSM_ERR_INVALID_ARG.  All calls share that array, so calls that overlap on the
 * GPU race and give wrong results.  The first call on a device resolves the
 * array's address (cudaGetSymbolAddress, device current); make it before any
 * stream capture.  No cudaMalloc, cudaFree or allocating library call is made. */
int32_t rsm_residual_noalloc(const void* Y, int64_t ldy, int32_t y_dtype, const uint8_t* W, int64_t ldw,
                             const double* U, int64_t ldu, const double* V, int64_t ldv, int64_t m, int64_t n,
                             int32_t r, double* e, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSM_H_ */
