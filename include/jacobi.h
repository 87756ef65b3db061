/*
 * jacobi.h - C ABI of the GB300 (sm_103a) dense Jacobi solver.
 *
 * The method is the Jacobi iteration of Margaris, Souravlas & Roumeliotis, "Parallel Implementations
 * of the Jacobi Linear Algebraic Systems Solver" (arXiv:1403.5805), Section 2: split A = D - L - U,
 * iterate X^(k) = T X^(k-1) + C with T = D^-1 (L + U) and C = D^-1 B, stop when the change between
 * consecutive iterates drops below a tolerance or after a maximum number of sweeps.
 *
 * Every sweep runs on the GPU inside one persistent kernel per solve: the matrix is streamed from HBM
 * once per sweep, the convergence reduction is fused into the sweep and decided on the device, so no
 * host round trip happens between sweeps.
 *
 * Conventions shared by all calls
 *   - A is row-major n x n: element (i, j) at A[i*lda + j] (lda = n in the host-pointer calls).
 *   - B and X are column-major n x nrhs: element (i, c) at B[c*ldb + i] (one right-hand side per
 *     column; ldb = n in the host-pointer calls).
 *   - Return value: a jacobi_status.  Values > 0 are warnings with a valid X, values < 0 are errors.
 *   - All calls use the CUDA device that is current on the calling thread when the handle is created.
 *   - A handle is not thread-safe: use one handle per thread (handles are independent).
 */
#ifndef JACOBI_H
#define JACOBI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JACOBI_API __attribute__((visibility("default")))
#else
#define JACOBI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum jacobi_status {
  JACOBI_OK = 0,                  /* converged */
  JACOBI_NOT_CONVERGED = 1,       /* iteration cap reached; X holds the last iterate X^(L) */
  JACOBI_ERR_INVALID_ARG = -1,    /* null pointer, n < 1, max_iter < 1, tol <= 0 or NaN, bad enum */
  JACOBI_ERR_ZERO_DIAGONAL = -2,  /* some a_ii == 0: the method is undefined (Section 2) */
  JACOBI_ERR_NONFINITE = -3,      /* non-finite diagonal, or the iteration produced inf/NaN */
  JACOBI_ERR_OUT_OF_MEMORY = -4,  /* device allocation failed or workspace too small */
  JACOBI_ERR_CUDA = -5,           /* a CUDA runtime call failed (see jacobi_last_cuda_error) */
  JACOBI_ERR_TIMEOUT = -6,        /* a bounded device-side wait expired; the context stays usable */
  JACOBI_ERR_UNSUPPORTED = -8     /* valid request the library does not implement (e.g. Gauss-Seidel, FP32
                                     or E4M3 inner sweeps with nrhs > 1; BF16 sweeps for an nrhs other than
                                     16, 32, 64 or 128) */
} jacobi_status;

/* Arithmetic of the solve.
 *   JACOBI_FP64     plain Jacobi in FP64 (Section 2 iteration exactly; the stopping test is `change < tol`).
 *   JACOBI_*_IR     mixed precision: inner Jacobi sweeps read the off-diagonal part of A stored as FP32,
 *                   BF16 or FP8 E4M3 (with an FP32 scale per row) and accumulate in FP32; an outer FP64
 *                   iterative refinement (r = B - A X in FP64, X += delta) runs until
 *                   ||B - A X||_inf / ||B||_inf <= tol.  The paper does not discuss precision; this
 *                   refinement is the library's own design around the Section 2 sweep. */
typedef enum jacobi_precision {
  JACOBI_FP64 = 0,
  JACOBI_FP32_IR = 1,
  JACOBI_BF16_IR = 2,
  JACOBI_FP8_IR = 3
} jacobi_precision;

/* Stopping norm of the FP64 path (the change between consecutive iterates, Section 2 algorithm).
 *   JACOBI_NORM_INF    max_i |x_i^(k) - x_i^(k-1)|
 *   JACOBI_NORM_2      sqrt(sum_i (x_i^(k) - x_i^(k-1))^2), the paper's Euclidean test (Section 3.1)
 *   JACOBI_NORM_RESID  max_i |a_ii (x_i^(k) - x_i^(k-1))| / ||B||_inf, which is the relative residual
 *                      ||B - A X^(k-1)||_inf / ||B||_inf of the previous iterate. */
typedef enum jacobi_norm { JACOBI_NORM_INF = 0, JACOBI_NORM_2 = 1, JACOBI_NORM_RESID = 2 } jacobi_norm;

/* Result record of one solve. */
typedef struct jacobi_stats {
  int64_t sweeps;       /* FP64: Jacobi sweeps executed (k of the returned X^(k)); IR: inner sweeps */
  int64_t outer_steps;  /* IR: FP64 residual evaluations; FP64 path: 0 */
  double final_delta;   /* FP64: stopping norm of the last sweep; IR: last inner max-norm change */
  double rel_residual;  /* IR: ||B - A X||_inf / ||B||_inf of the returned X (FP64, on the device);
                           FP64 path: NaN */
  int32_t status;       /* jacobi_status of the solve */
  int32_t converged;    /* 1 if status == JACOBI_OK */
} jacobi_stats;

typedef struct jacobi_handle jacobi_handle;

/* ------------------------------------------------------------------------------------------------
 * Host-pointer interface (the problem statement of Section 2: inputs A, B, X^0, tol, L; output X).
 * ------------------------------------------------------------------------------------------------ */

/* Copy A (n x n, row-major, host) and B (n, host) to the device and prepare the FP64 sweep.
 * The library allocates the device memory (cudaMalloc) and owns it until jacobi_destroy; A and B may be
 * freed when the call returns.  Fails with JACOBI_ERR_ZERO_DIAGONAL / JACOBI_ERR_NONFINITE if some
 * a_ii is 0 or not finite (the handle is then not created; *out is set to NULL). */
JACOBI_API int jacobi_setup(const double* A, const double* B, int64_t n, jacobi_handle** out);

/* Run the FP64 Jacobi iteration from X0 (n, host; NULL means zeros) for at most max_iter sweeps with
 * the max-norm test `max|X^(k) - X^(k-1)| < tol` (Section 2).  On return X_out (n, host, caller-owned)
 * holds X^(k) (the new iterate of the converging sweep, or X^(L) at the cap), *iters_out = k and
 * *final_delta_out = max|X^(k) - X^(k-1)|.  iters_out / final_delta_out may be NULL.  Blocks until done. */
JACOBI_API int jacobi_solve(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                 int64_t* iters_out, double* final_delta_out);

/* Release every resource of the handle (NULL is a no-op). */
JACOBI_API void jacobi_destroy(jacobi_handle* h);

/* Short English description of a status value (static storage). */
JACOBI_API const char* jacobi_status_string(int status);

/* Last CUDA error string seen by the library on this thread ("" if none). */
JACOBI_API const char* jacobi_last_cuda_error(void);

/* ------------------------------------------------------------------------------------------------
 * Device-pointer interface (PyTorch or any other owner of device memory and streams).
 * ------------------------------------------------------------------------------------------------ */

typedef struct jacobi_desc {
  int64_t n;              /* system size, >= 1 */
  int64_t nrhs;           /* right-hand sides, >= 1 (B and X column-major, one column per right-hand side) */
  int32_t precision;      /* jacobi_precision */
  int32_t norm;           /* jacobi_norm (FP64 path; with nrhs > 1 each column is tested on its own and
                             the solve stops when every column has met the test) */
  const double* A;        /* row-major, A[i*lda + j], device or host memory.  Borrowed (read by every
                             solve, so it must stay unchanged and alive until jacobi_destroy) when it is
                             16-byte aligned device memory with n and lda even and JACOBI_FLAG_COPY_A is
                             not set; otherwise copied into the workspace during setup (host memory:
                             a host-to-device copy, fastest from pinned memory) and not referenced
                             afterwards */
  int64_t lda;            /* >= n */
  const double* B;        /* column-major, B[c*ldb + i], device or host memory; read during setup only */
  int64_t ldb;            /* >= n */
  void* workspace;        /* device buffer of >= jacobi_workspace_size() bytes, 256-byte aligned,
                             owned by the caller and borrowed until jacobi_destroy; NULL: the library
                             allocates it with cudaMalloc */
  size_t workspace_bytes; /* size of workspace when given */
  void* stream;           /* cudaStream_t every call of this handle is ordered on; NULL: legacy default */
  int32_t grid;           /* CTAs of the persistent kernels; 0: one per SM (capped by the row count) */
  int32_t max_outer;      /* IR: cap on FP64 residual evaluations (0: 60) */
  double inner_rtol;      /* IR: stop inner sweeps when max|delta change| <= inner_rtol * max|delta|
                             (0: 2^-10 for FP32/BF16, 2^-6 for FP8) */
  int32_t max_inner;      /* IR: cap on inner sweeps per outer step (0: 1000) */
  int32_t flags;          /* JACOBI_FLAG_* */
  int32_t method;         /* jacobi_method (0: the Jacobi iteration) */
  int32_t reserved;
  double omega;           /* JACOBI_METHOD_SOR: relaxation factor, 0 < omega < 2 (0: 1, Gauss-Seidel) */
} jacobi_desc;

/* Iteration of the FP64 single-right-hand-side path.
 * JACOBI_METHOD_SOR: the Gauss-Seidel / SOR sweep, the relaxed relative of the Section 2 iteration that
 *   uses each new component as soon as it is computed,
 *     x_i^(k) = x_i^(k-1) + omega ((beta_i - sum_{j<i} alpha_ij x_j^(k) - sum_{j>i} alpha_ij x_j^(k-1))
 *               / alpha_ii - x_i^(k-1)),
 *   run as a chain over the CTAs' row blocks (each block waits for the earlier blocks' new values), so the
 *   iterates are those of the sequential sweep whatever the grid.  Stopping test, norms (max-norm or
 *   Euclidean) and return conventions as for the Jacobi iteration.  Requires JACOBI_FP64, one right-hand
 *   side and n <= 112 * (co-resident CTAs); otherwise JACOBI_ERR_UNSUPPORTED from the setup. */
typedef enum { JACOBI_METHOD_JACOBI = 0, JACOBI_METHOD_SOR = 1 } jacobi_method;

#define JACOBI_FLAG_COPY_A 1 /* always copy A into the workspace (never borrow it) */
/* IR precisions (one or many right-hand sides): compute the FP64 residual r = B - A X with split-float
 * arithmetic on the FP32 units (each a_ij as two FP32 words after a per-row power-of-two scale, each
 * x_j as two FP32 words after a power-of-two scale of its column, products with exact FMA errors,
 * float-float sums, FP64 combination at the end) instead of FP64 FMAs.  Accuracy ~2^-46 relative per
 * product; GB300's FP64 FMA rate makes the FP64-instruction residual arithmetic-bound.  The column
 * scale comes from max_i |b_i / a_ii| (one right-hand side) or from max_i |x_ic| of each residual's X
 * (many), so X may have any magnitude that stays within 2^100 of that scale. */
#define JACOBI_FLAG_SPLIT_RESIDUAL 2
/* Every device-side wait of this handle's solves gives up after 50 ms instead of 4 s. */
#define JACOBI_FLAG_SHORT_WAITS 4
/* Test only: the first ring item of each solve is announced to the consumers but never copied, so their
 * bounded wait expires; the solve then returns JACOBI_ERR_TIMEOUT and the context stays usable. */
#define JACOBI_FLAG_TEST_DROP_COPY 8
/* Test only.  Sparse handle: CTA 0 never arrives at the grid barrier of the first sweep and raises the
 * error word instead.  Gauss-Seidel handle: block 0 never publishes its first sweep (no flag, no mailbox)
 * and raises the error word.  Either way the other CTAs leave their bounded waits, the solve returns
 * JACOBI_ERR_TIMEOUT and the context stays usable. */
#define JACOBI_FLAG_TEST_SKIP_ARRIVAL 32
/* Many right-hand sides: retire each column as soon as it meets the stopping test on its own (the
 * FP64 path: its change norm below tol; the BF16 path: its relative residual at or below tol) instead of
 * iterating every column until the worst one does.  A retired column keeps the iterate that met the test
 * (so each column equals the single-right-hand-side solve of that column), and later passes skip it:
 * the FP64 sweeps and FP64 residual evaluations only touch the columns still active.  Per-column counts
 * come from jacobi_column_stats. */
#define JACOBI_FLAG_RETIRE_COLUMNS 16
/* Sparse handle: keep T in sliced ELL even when its entries lie on a few diagonals (see jacobi_csr_format). */
#define JACOBI_FLAG_CSR_ELL 64
/* BF16 inner sweeps with many right-hand sides (nrhs 16, 32, 64 or 128): compute each residual
 * r = B - A X on the tcgen05 tensor cores with FP64 accuracy instead of FP64 FMAs.  Setup splits the off-
 * diagonal part of A (each row scaled by a power of two from its largest entry) into 7 balanced base-256
 * digits stored as BF16 matrices (14 bytes per entry of A in the workspace), and each residual splits X
 * (each column scaled by its largest entry) the same way; the products of digit pairs whose levels add up
 * to at most 8 are summed by tcgen05.mma in FP32, exactly (1024-column chunks of integer products of at
 * most 2^14), the chunk sums in float-float, the diagonal term in FP64.  When the 128-row tiles alone would
 * leave part of the last wave of CTAs idle, each tile's K range is split into up to 8 parts whose float-
 * float sums a second launch adds in part order (the workspace holds 8 x 8 bytes per entry of X for them).
 * The representation and dropped-pair errors are below 2^-50 of sum_j |a_ij| max |x_jc| per entry.  Not
 * with JACOBI_FLAG_SPLIT_RESIDUAL;
 * JACOBI_ERR_UNSUPPORTED for other precisions or one right-hand side.  Also a server flag
 * (jacobi_server_desc.flags), for requests of any size and right-hand-side count. */
#define JACOBI_FLAG_TC_RESIDUAL 128
/* BF16 / FP32 inner sweeps, one right-hand side: A is symmetric, so the narrow copy of its off-diagonal part
 * keeps only the 128 x 128 tiles on and above the diagonal (packed), half the bytes of every inner sweep.
 * Each off-diagonal tile (I, J) gives the row dots of block I and, through a_ji = a_ij, the column dots of
 * block J in one read; per-row partial sums go to fixed slots that a second launch adds in slot order.  The
 * lower triangle of A is not read for the narrow copy (the FP64 residual reads all of A, so a non-symmetric
 * A refines slowly or not at all).  The refinement loop runs on the host (one small device-to-host read per
 * phase); the per-phase trace (jacobi_last_trace) comes from CUDA events.  Not with the split-float or
 * tensor-core residual; JACOBI_ERR_UNSUPPORTED for other precisions, several right-hand sides or SOR.
 * jacobi_get_narrow returns JACOBI_ERR_UNSUPPORTED (the copy is not row-major). */
#define JACOBI_FLAG_SYMMETRIC 256

/* Fill *d with defaults (n = 0 and null pointers: the caller sets those). */
JACOBI_API void jacobi_desc_init(jacobi_desc* d);

/* Bytes of device workspace a handle for *d needs (written to *bytes). */
JACOBI_API int jacobi_workspace_size(const jacobi_desc* d, size_t* bytes);

/* Prepare a solver from device-resident A and B, on d->stream: reads the diagonal (rejecting zero or
 * non-finite entries), stores 1/a_ii, copies B, copies A into the padded streaming layout unless it is
 * borrowed (see jacobi_desc.A) and, for the IR precisions, writes the FP32/BF16/E4M3 copy of the
 * off-diagonal part of A.  Synchronises the stream once, to read the diagonal check.  B is not
 * referenced after the call returns. */
JACOBI_API int jacobi_setup_ex(const jacobi_desc* d, jacobi_handle** out);

/* Solve asynchronously on the handle's stream.  X0 (device, n x nrhs column-major, ld = n; NULL means
 * zeros) and X_out (device, same layout) may alias.  stats_dev, if not NULL, is a device jacobi_stats
 * the kernel fills.  For JACOBI_FP64, tol is the stopping threshold of the handle's norm (strict <);
 * for the IR precisions, tol is the relative-residual target (<=) and max_iter caps inner sweeps.
 * Returns an error only for invalid arguments or launch failures; the solve's own status lands in
 * stats_dev and in the handle (jacobi_last_stats). */
JACOBI_API int jacobi_solve_async(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                       jacobi_stats* stats_dev);

/* jacobi_solve_async, then wait for the stream and return the solve's status; *stats (host) filled if
 * not NULL. */
JACOBI_API int jacobi_solve_ex(jacobi_handle* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                    jacobi_stats* stats);

/* Stats of the handle's last solve (waits for its stream). */
JACOBI_API int jacobi_last_stats(jacobi_handle* h, jacobi_stats* stats);

/* Relative residual ||B - A X||_inf / ||B||_inf of a device X (n, ld = n) against the handle's FP64 A and
 * B, computed on the device in FP64 with the handle's streaming kernel; waits for the stream. */
JACOBI_API int jacobi_residual(jacobi_handle* h, const double* X, double* rel_out);

/* Per-column record of the last solve of a many-right-hand-side handle (host arrays of nrhs entries,
 * either may be NULL): iters[c] = sweeps (FP64) or residual evaluations (BF16 IR) after which column c
 * finished (retired, or the solve ended), value[c] = its last change norm (FP64) or relative residual
 * (BF16 IR).  JACOBI_ERR_INVALID_ARG for a single-right-hand-side handle. */
JACOBI_API int jacobi_column_stats(jacobi_handle* h, int64_t* iters, double* value);

/* Copy the narrow off-diagonal matrix that the inner sweeps of an IR handle read to host memory:
 * dst_host is row-major n x ld_dst (ld_dst >= n) of the precision's element type (FP32 values, BF16
 * codes as uint16, E4M3 codes as uint8; the diagonal holds zero codes), scale_host (n floats, may be
 * NULL) the per-row E4M3 scales (1.0 for FP32/BF16).  JACOBI_ERR_INVALID_ARG for an FP64 handle.
 * Waits for the stream. */
JACOBI_API int jacobi_get_narrow(jacobi_handle* h, void* dst_host, int64_t ld_dst, float* scale_host);

/* Trace of the last solve: for each phase (one sweep or one residual evaluation) its end time in
 * nanoseconds since the solve started and its kind (JACOBI_PHASE_*).  Single right-hand side: recorded
 * by the persistent kernel from %globaltimer at each grid-wide barrier (the first 512 phases).  Many
 * right-hand sides: CUDA events around each phase's kernel.  Writes min(cap, phases) entries and the
 * phase count to *count.  Waits for the stream. */
#define JACOBI_PHASE_SWEEP64 0  /* FP64 Jacobi sweep over A */
#define JACOBI_PHASE_RESID64 1  /* FP64 residual r = B - A X over A */
#define JACOBI_PHASE_RESID0 2   /* residual of a zero start vector (r = B, no matrix pass) */
#define JACOBI_PHASE_INNER 3    /* inner sweep over the narrow copy of A */
#define JACOBI_PHASE_NARROW_INNER 4 /* first inner sweep of a handle's first solve (BF16 / FP32 inner sweeps):
                                       reads FP64 A, writes the narrow copy and sweeps over the rounded values */
#define JACOBI_PHASE_HOST_GAP 5     /* host-driven solves (JACOBI_FLAG_SYMMETRIC): the stream's idle time while the
                                       host reads a phase's result and queues the next; not a phase of work */
JACOBI_API int jacobi_last_trace(jacobi_handle* h, int64_t* t_end_ns, int32_t* kinds, int32_t cap,
                                 int32_t* count);

/* ------------------------------------------------------------------------------------------------
 * Batched solves of many independent systems of uneven size.
 *
 * Section 2's Jacobi iteration applied to `count` independent systems A_k X_k = B_k (n_k <=
 * JACOBI_BATCH_MAX_N) in one persistent kernel: each CTA takes a whole system from a device work queue
 * (largest first), keeps its iterates in shared memory, and sweeps its rows with its warps (the
 * row-wise distribution of Section 3.1 applied to systems over SMs and rows over warps).  The launch
 * is captured once into a CUDA graph and replayed.
 * ------------------------------------------------------------------------------------------------ */

#define JACOBI_BATCH_MAX_N 4096

typedef struct jacobi_batch jacobi_batch;

typedef struct jacobi_batch_desc {
  int64_t count;              /* number of systems, >= 1 */
  const int64_t* n;           /* host array [count]: sizes, 1 <= n_k <= JACOBI_BATCH_MAX_N */
  const double* const* A;     /* host array [count] of device pointers: row-major n_k x n_k (stride n_k),
                                 read in place by every solve (keep unchanged until destroy) */
  const double* const* B;     /* host array [count] of device pointers: n_k values */
  double* const* X;           /* host array [count] of device pointers: n_k outputs */
  int32_t precision;          /* JACOBI_FP64: plain Jacobi with the previous-iterate relative-residual
                                 stop (strict <); JACOBI_FP32_IR / JACOBI_BF16_IR: FP64 refinement around
                                 narrow inner sweeps, stop at ||B - A X||_inf / ||B||_inf <= tol */
  int32_t rows_per_warp;      /* 1, 2, 4 or 8 rows a warp accumulates at once (0: 4) */
  int32_t ctas_per_sm;        /* cap on resident CTAs per SM (0: as many as fit); 3 or more selects the
                                 build limited to 64 registers per thread, so that 4 CTAs fit */
  int32_t max_outer;          /* IR: cap on residual evaluations per system (0: 30) */
  int32_t max_inner;          /* IR: cap on inner sweeps per outer step (0: 1000) */
  int32_t flags;              /* JACOBI_FLAG_SPLIT_RESIDUAL: split-float residuals (IR; see jacobi_desc) */
  double inner_rtol;          /* IR: inner stop, max|change| <= inner_rtol * max|delta| (0: 2^-14) */
  void* workspace;            /* device, >= jacobi_batch_workspace_size bytes, 256-byte aligned; NULL:
                                 the library allocates it */
  size_t workspace_bytes;
  void* stream;               /* cudaStream_t the solves are ordered on (NULL: legacy default) */
} jacobi_batch_desc;

/* Device bytes the batch needs: per system its narrow copy (IR) and four n-vectors, plus the system
 * table, the queue counter and the per-system records. */
JACOBI_API int jacobi_batch_workspace_size(const jacobi_batch_desc* d, size_t* bytes);

/* Validate, lay out the workspace, upload the system table (sorted by decreasing n).  Synchronises the
 * stream once.  *out is NULL on error. */
JACOBI_API int jacobi_batch_create(const jacobi_batch_desc* d, jacobi_batch** out);

/* Solve every system from X = 0, asynchronously on the batch's stream: one graph launch (queue reset
 * + the persistent kernel; captured on the first call for this (max_iter, tol) and replayed after).
 * max_iter caps sweeps per system (FP64) or inner sweeps per system (IR).  Each system's status lands
 * in its record (jacobi_batch_stats); a system with a zero or non-finite diagonal gets
 * JACOBI_ERR_ZERO_DIAGONAL / JACOBI_ERR_NONFINITE and its X is left as zeros. */
JACOBI_API int jacobi_batch_solve_async(jacobi_batch* b, int64_t max_iter, double tol);

/* Copy the per-system records of the last solve (host array [count], in the caller's order); waits
 * for the stream. */
JACOBI_API int jacobi_batch_stats(jacobi_batch* b, jacobi_stats* stats);

/* CTAs of the persistent batch kernel (0 for NULL). */
JACOBI_API int jacobi_batch_grid(jacobi_batch* b);

/* Release the batch (waits for its stream; NULL is a no-op). */
JACOBI_API void jacobi_batch_destroy(jacobi_batch* b);

/* One call for a whole batch, the batched form of jacobi_solve: create on the legacy default stream with the
 * launch shape the autotuner picks for thousands of systems of a few hundred unknowns (4 rows per warp, the
 * 64-register build at 4 CTAs per SM, inner tolerance 2^-10 for the IR precisions), solve every system from
 * X = 0, copy the per-system records into stats (host array
 * [count], may be NULL) and release.  A, B, X_out: host arrays [count] of device pointers as in
 * jacobi_batch_desc; precision JACOBI_FP64, JACOBI_FP32_IR or JACOBI_BF16_IR.  Returns the worst outcome
 * over the systems (an error status, else JACOBI_NOT_CONVERGED if any system hit its cap, else JACOBI_OK),
 * or the error of the create / solve itself. */
JACOBI_API int jacobi_batch_solve(int64_t count, const int64_t* n, const double* const* A, const double* const* B,
                                  double* const* X_out, double tol, int64_t max_iter, int32_t precision,
                                  jacobi_stats* stats);

/* ------------------------------------------------------------------------------------------------
 * Serving: continuous batching of independent solve requests.
 *
 * Each request is a system A X = B (n <= JACOBI_SERVE_MAX_N, 1 <= r <= JACOBI_SERVE_MAX_RHS right-hand
 * sides) solved by Section 2's Jacobi iteration as FP32 inner sweeps inside an FP64 refinement, to
 * ||B - A X||_inf / ||B||_inf <= tol per column.  Admitted requests keep all their state on the device
 * inside an arena of budget_bytes.  jacobi_server_step runs one round: admit waiting requests in arrival
 * order while the arena has room, advance every active request by one phase in one kernel launch, retire
 * the finished ones (their X is copied to the caller's X_out and their memory freed).  A request's
 * arithmetic does not depend on the other requests in the round.
 * ------------------------------------------------------------------------------------------------ */

#define JACOBI_SERVE_MAX_N 8192
#define JACOBI_SERVE_MAX_RHS 16

typedef struct jacobi_server jacobi_server;

typedef struct jacobi_server_desc {
  size_t budget_bytes;  /* device arena for admitted requests (allocated once at create) */
  double tol;           /* relative-residual target (0: 1e-10) */
  int64_t max_iter;     /* cap on inner sweeps per request (0: 5000) */
  int32_t max_inner;    /* cap on inner sweeps per refinement step (0: 1000) */
  int32_t max_outer;    /* cap on residual evaluations per request (0: 30) */
  double inner_rtol;    /* inner stop: max|change| <= inner_rtol * max|delta| (0: 2^-10) */
  int32_t max_active;   /* cap on concurrently active requests (0: only the budget limits) */
  int32_t flags;        /* JACOBI_FLAG_SPLIT_RESIDUAL: split-float residual rounds (see jacobi_desc);
                           JACOBI_FLAG_TC_RESIDUAL: residual rounds on the tensor cores (every request's A
                           split into digits at admission, 14 more bytes per entry of A in the arena; the
                           residual requests of a round run in one grouped launch before the round kernel) */
  void* stream;         /* cudaStream_t of every round (NULL: legacy default stream) */
} jacobi_server_desc;

JACOBI_API int jacobi_server_create(const jacobi_server_desc* d, jacobi_server** out);

/* Queue a request whose A (n x n row-major, stride n) and B (n x r column-major, stride n) are in device
 * or host memory; they are copied into the arena when the request is admitted, so they must stay valid
 * until then.  X_out (n x r column-major, device or pinned host) receives the solution when the request
 * finishes.  *id_out identifies the request in jacobi_server_poll.  JACOBI_ERR_OUT_OF_MEMORY if the
 * request could never fit the budget. */
JACOBI_API int jacobi_server_submit(jacobi_server* s, int64_t n, int64_t r, const double* A, const double* B,
                                    double* X_out, int64_t* id_out);

/* Queue a request generated on the device at admission from (seed, f): the generator of
 * jacobi_generate_request. */
JACOBI_API int jacobi_server_submit_generated(jacobi_server* s, int64_t n, int64_t r, double f, uint64_t seed,
                                              double* X_out, int64_t* id_out);

/* One round (see above); waits for it.  *active_out / *pending_out: requests on the device / waiting. */
JACOBI_API int jacobi_server_step(jacobi_server* s, int32_t* active_out, int32_t* pending_out);

/* Requests finished since the last poll (up to cap): their ids and records (status, sweeps = inner
 * sweeps, outer_steps = residual evaluations, rel_residual = final max over columns).  Their X_out is
 * complete when this returns. */
JACOBI_API int jacobi_server_poll(jacobi_server* s, int64_t* ids, jacobi_stats* stats, int32_t cap, int32_t* count);

/* Run rounds until request `id` finishes, then return its status and record (*stats may be NULL); its
 * X_out is complete.  The request is collected: later polls do not report it.  Other requests that
 * finish meanwhile stay for jacobi_server_poll.  JACOBI_ERR_INVALID_ARG for an unknown id or one
 * collected already. */
JACOBI_API int jacobi_server_wait(jacobi_server* s, int64_t id, jacobi_stats* stats);

/* Rounds run so far. */
JACOBI_API int jacobi_server_rounds(jacobi_server* s, int64_t* rounds);

/* Release the server and every queued or active request (waits for the stream). */
JACOBI_API void jacobi_server_destroy(jacobi_server* s);

/* Write a seeded dominant system on the device: A (n x n, row stride n) with off-diagonals
 * int32(w) * 2^-31 (w word i*n + j of Philox4x32-10 stream 0 under key `seed`), a_ii = f * sum_{j != i}
 * |a_ij| * (-1 if bit 0 of word i of stream 1 is set), and B[c*ldb + i] = int32(w) * 2^-31 (word c*n + i
 * of stream 5).  Asynchronous on `stream`. */
JACOBI_API int jacobi_generate_request(int64_t n, int64_t r, double f, uint64_t seed, double* A, double* B,
                                       int64_t ldb, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Measured arithmetic rates.  The paper has no counterpart: this is the measurement behind the roofline
 * that FP64 passes over A are held to (one FP64 FMA per 8-byte entry of A), and behind the FP32-unit
 * bound of the split-float residual.
 * ------------------------------------------------------------------------------------------------ */

/* Time independent FMA chains on every SM of the current device (16 chains x `iters` iterations per
 * thread, or 4 chains x 4 iters, at 4 and 8 blocks of 256 threads per SM; each chain either the
 * recurrence x = x m + c or the dot-product form acc = a b + acc), in FP64 and then in FP32 (64 times as
 * many iterations), each launch after an untimed one, with CUDA events on `stream` (a
 * cudaStream_t; NULL: legacy default stream).  Writes the best FMAs per second of each (host doubles).
 * Blocks until done.  JACOBI_ERR_INVALID_ARG for iters < 1 or a NULL output. */
JACOBI_API int jacobi_measure_fma_rates(int64_t iters, double* fp64_fma_per_s, double* fp32_fma_per_s, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Allocation-free FP64 solve.  The paper has no counterpart to this entry point: it exists for callers
 * that must not allocate device memory while they run, such as a plugin inside a host application that
 * owns the GPU's memory pool and forbids other allocations, or a latency-bound loop that cannot afford
 * cudaMalloc's implicit synchronisation and its possible failure.
 * ------------------------------------------------------------------------------------------------ */

/* Largest n jacobi_solve_fp64_noalloc accepts. */
#define JACOBI_NOALLOC_MAX_N 32768

/* The same FP64 Jacobi solve as jacobi_setup_ex + jacobi_solve_ex (max-norm test, strict < tol), with
 * no device allocation: the library's own scratch (about 1 MB: control block, iterate buffers, diagonal
 * reciprocals) is a fixed array in device memory that every device loading the library keeps until the
 * process exits.
 *   A      device, row-major n x n, A[i*lda + j]; 16-byte aligned, lda even; for odd n, lda > n and the
 *          element A[i*lda + n] of each row is read (its value is ignored).  Read in place.
 *   B      device, n values.  X0: device, n values, or NULL for zeros.  X_out: device, n values.
 *   stats  host, filled if not NULL.  stream: cudaStream_t (NULL: legacy default stream).
 * Returns the solve's jacobi_status; JACOBI_ERR_INVALID_ARG for n > JACOBI_NOALLOC_MAX_N, a misaligned
 * or non-device A / B / X_out, max_iter < 1, or tol not positive and finite.  JACOBI_ERR_ZERO_DIAGONAL /
 * JACOBI_ERR_NONFINITE as jacobi_setup_ex (first failing row).  Blocks until the solve is done: every
 * call synchronises the stream and reads the solve's status back to the host, so no call may be made
 * on a stream under capture.  The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; do not call this entry point after
 * cudaDeviceReset on that device (the reset unloads the array and the kept address goes stale).  Every call shares the one array and it keeps the last call's contents (each call
 * clears what must start at zero), so calls that overlap on the GPU - from two streams or two host
 * threads on one device - race: serialise them. */
JACOBI_API int jacobi_solve_fp64_noalloc(const double* A, int64_t lda, const double* B, int64_t n,
                                         const double* X0, int64_t max_iter, double tol, double* X_out,
                                         jacobi_stats* stats, void* stream);

/* ------------------------------------------------------------------------------------------------
 * Sparse A (compressed sparse rows).  The Section 2 iteration for a sparse A, the banded and
 * PDE-shaped matrices of the Jacobi codes for differential equations that the paper's related work
 * (Section 1) cites:
 *   x_i^(k) = ( beta_i - sum_{stored j != i} alpha_ij x_j^(k-1) ) / alpha_ii,
 * with the same stopping test, iteration count and return convention as the dense FP64 path (strict
 * `change < tol` after each sweep, the new iterate returned, X^(L) and JACOBI_NOT_CONVERGED at the cap).
 * FP64, one right-hand side.  Setup copies the matrix into a sliced-ELL layout of its off-diagonal part
 * (32-row slices, each as wide as its longest row) that the library owns; the caller's arrays may be
 * freed when setup returns.
 * ------------------------------------------------------------------------------------------------ */

typedef struct jacobi_csr jacobi_csr;

typedef struct jacobi_csr_desc {
  int64_t n;               /* unknowns (rows = columns), >= 1 */
  int64_t nnz;             /* stored entries, row_ptr[n] */
  const int64_t* row_ptr;  /* n + 1 offsets: row i is entries [row_ptr[i], row_ptr[i+1]); row_ptr[0] = 0 */
  const int32_t* col_idx;  /* nnz columns, strictly ascending within each row; each row stores its diagonal */
  const double* values;    /* nnz values */
  const double* B;         /* n values: the right-hand side */
  int32_t norm;            /* JACOBI_FP64: JACOBI_NORM_INF, JACOBI_NORM_2 or JACOBI_NORM_RESID (as jacobi_desc);
                            * mixed precision: JACOBI_NORM_INF (the relative residual is the test) */
  int32_t flags;           /* JACOBI_FLAG_SHORT_WAITS, JACOBI_FLAG_TEST_SKIP_ARRIVAL */
  void* stream;            /* cudaStream_t of every call on the handle (NULL: the legacy default stream) */
  int32_t precision;       /* JACOBI_FP64 (0: the plain iteration), JACOBI_FP32_IR or JACOBI_BF16_IR (below) */
  int32_t max_outer;       /* IR: outer steps after the first residual (0: 60) */
  int32_t max_inner;       /* IR: inner sweeps per outer step (0: 1000) */
  int32_t reserved;        /* 0 */
  double inner_rtol;       /* IR: inner stop at max|delta' - delta| <= inner_rtol max|delta'| (0: 2^-20 for FP32,
                            * 2^-8 for BF16) */
} jacobi_csr_desc;

/* Mixed precision (precision = JACOBI_FP32_IR or JACOBI_BF16_IR): the library also keeps T in FP32 or
 * BF16.  One persistent kernel alternates an FP64 residual, r' = C + T x - x = D^-1 (b - A x), with inner
 * Jacobi sweeps on the correction, delta <- r' + T_lo delta (FP32 accumulation), until
 * ||b - A x||_inf / ||b||_inf <= tol (not strict); x += delta in FP64.  The solve reports the relative
 * residual as final_delta and rel_residual, counts inner sweeps in `sweeps` and residual evaluations in
 * `outer_steps`.  JACOBI_FP8_IR is JACOBI_ERR_UNSUPPORTED here. */

/* Validate and copy the matrix (host or device pointers; setup blocks until the copy is built).
 * Errors: JACOBI_ERR_INVALID_ARG for a null pointer, n < 1, nnz < 1, a bad norm, or a malformed structure
 * (row_ptr[0] != 0 or row_ptr[n] != nnz, a row range that decreases, a column out of [0, n) or columns not
 * strictly ascending in a row); then, by the first failing row, JACOBI_ERR_ZERO_DIAGONAL (diagonal missing
 * or zero) or JACOBI_ERR_NONFINITE (non-finite diagonal); JACOBI_ERR_OUT_OF_MEMORY. */
JACOBI_API int jacobi_csr_setup(const jacobi_csr_desc* d, jacobi_csr** out);

/* Queue one solve on the handle's stream: one persistent kernel runs every sweep and the stopping test.
 * X0: n values (host or device) or NULL for zeros; X_out: n values (host or device; a host X_out makes
 * the call wait for the copy).  Read the outcome with jacobi_csr_last_stats. */
JACOBI_API int jacobi_csr_solve_async(jacobi_csr* h, const double* X0, int64_t max_iter, double tol,
                                      double* X_out);

/* Synchronous solve: returns the solve's jacobi_status and fills *stats (host) if not NULL. */
JACOBI_API int jacobi_csr_solve(jacobi_csr* h, const double* X0, int64_t max_iter, double tol, double* X_out,
                                jacobi_stats* stats);

/* Outcome of the last solve (waits for it). */
JACOBI_API int jacobi_csr_last_stats(jacobi_csr* h, jacobi_stats* stats);

/* Layout facts for byte accounting: slots stored (off-diagonal entries plus slice padding; DIA: diagonals
 * times n rounded up to whole slices), slices of 32 rows, and the grid of the sweep kernel.  Any output may
 * be NULL. */
JACOBI_API int jacobi_csr_info(jacobi_csr* h, int64_t* stored_slots, int64_t* slices, int32_t* grid);

/* Storage of T chosen by setup.  JACOBI_CSR_ELL: sliced ELL (slices of 32 rows, each as wide as its
 * longest row, values and int32 columns).  JACOBI_CSR_DIA: when every off-diagonal entry lies on one of at
 * most 16 diagonals j - i = const and the band stores at most 1.25 times the slots of sliced ELL (banded
 * and stencil matrices), T is kept diagonal by diagonal with no column array, absent entries as zeros,
 * and the sweep gathers x_{i + offset} contiguously.  The sums run over the same entries in the same
 * ascending column order either way (the zeros add nothing), so the iterates are the same.  *ndiag: the
 * number of diagonals (0 for ELL).  Either output may be NULL. */
#define JACOBI_CSR_ELL 0
#define JACOBI_CSR_DIA 1
JACOBI_API int jacobi_csr_format(jacobi_csr* h, int32_t* format, int32_t* ndiag);

/* End time of each phase of the last solve, in nanoseconds since the solve started, and its kind, as
 * jacobi_last_trace: JACOBI_PHASE_SWEEP64 sweeps, or (mixed precision) JACOBI_PHASE_RESID64 residuals and
 * JACOBI_PHASE_INNER sweeps; at most 512 are recorded, *count is the number of phases run. */
JACOBI_API int jacobi_csr_last_trace(jacobi_csr* h, int64_t* t_end_ns, int32_t* kinds, int32_t cap, int32_t* count);

JACOBI_API void jacobi_csr_destroy(jacobi_csr* h);

#ifdef __cplusplus
}
#endif

#endif /* JACOBI_H */
