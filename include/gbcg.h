/*
 * gbcg.h -- C ABI of the GB300 sparse conjugate-gradient library.
 *
 * The operation is the one in Section III of "Parallel Sparse Matrix Solver
 * on the GPU Applied to Simulation of Electrical Machines" (Rodrigues et al.):
 * solve A x = b for a known, square, symmetric positive-definite sparse A
 * (Section I) by the unpreconditioned conjugate-gradient iteration, with A
 * stored in CSR, in symmetric CSR (one triangle plus the diagonal, A = L + D +
 * U with U' = L) or in CSC, and the product y = A p computed by the library's
 * own kernels.
 *
 * Conventions for every entry point:
 *   - Return value: a gbcg_status (0 = GBCG_OK).  Nothing throws or aborts
 *     across this boundary; on failure gbcg_last_error() gives a message for
 *     the calling thread.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  All device work of a call is issued on it.
 *   - Vectors are dense, contiguous, length n, owned by the caller.  Unless a
 *     call says otherwise they are device pointers.
 *   - Indices are int32.  Matrices with more than 2^31 - 1 stored entries are
 *     rejected with GBCG_ERR_INVALID.
 *   - A gbcg_matrix_t is not thread-safe: one call at a time per handle.  Two
 *     handles may be used concurrently from different threads and streams.
 */
#ifndef GBCG_H
#define GBCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbcg_matrix_s* gbcg_matrix_t;

/* Storage formats accepted by gbcg_create (Section III, "CSR, and Symmetric
 * CSR and CSC formats"). */
enum gbcg_format {
  GBCG_CSR = 0,          /* full matrix by rows: ptr[n+1], idx = column, val */
  GBCG_SYM_CSR_UPPER = 1,/* upper triangle and diagonal by rows (j >= i): the
                            same numbers as the paper's L + D by rows read as
                            columns; each off-diagonal entry stands for both
                            (i, j) and (j, i) */
  GBCG_CSC = 2           /* full matrix by columns: ptr[n+1], idx = row, val */
};

enum gbcg_status {
  GBCG_OK = 0,
  GBCG_ERR_INVALID = 1,   /* bad argument or malformed matrix */
  GBCG_ERR_NOT_SPD = 2,   /* p'Ap <= 0 met during the iteration */
  GBCG_ERR_MAXIT = 3,     /* iteration bound reached before the tolerance */
  GBCG_ERR_NONFINITE = 4, /* NaN or Inf met in a reduction */
  GBCG_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out */
  GBCG_ERR_CUDA = 6,      /* a CUDA runtime call failed */
  GBCG_ERR_NOMEM = 7      /* device or host allocation failed */
};

enum gbcg_precision {
  GBCG_FP64 = 0,          /* CG in double precision throughout */
  GBCG_FP32_IR = 1,       /* single-precision inner CG (Section IV's
                             single-precision variant) inside double-precision
                             iterative refinement: each pass restarts the inner
                             CG on r / ||r|| */
  GBCG_FP32_RU = 2        /* single-precision CG iterations with double-precision
                             reliable updates: the correction is added to x and the
                             residual replaced by b - A x in double precision each
                             time the recurrence residual falls by inner_tol
                             (default 0.1), keeping the search direction (the
                             Krylov space is not restarted).  Every format and
                             layout; one persistent launch */
};

enum gbcg_memory { GBCG_HOST = 0, GBCG_DEVICE = 1 };

/* Arrangement of the CG recurrences (both give the Section III iterates in
 * exact arithmetic). */
enum gbcg_variant {
  GBCG_STANDARD = 0,      /* the Section III listing: three grid barriers per iteration */
  GBCG_PIPELINED = 1      /* single reduction (Chronopoulos-Gear recurrences, Ghysels-
                             Vanroose arrangement): one fused pass over the rows and one
                             grid barrier per iteration, for three more vector streams;
                             its recurrences drift faster, so it restarts more often.
                             Double precision (GBCG_FP64) and row-gather layouts only
                             (CSR, CSC, symmetric with the transpose plan); other
                             combinations return GBCG_ERR_INVALID */
};

/* Solver options.  Zero-initialised fields take the documented defaults. */
typedef struct {
  int32_t precision;          /* gbcg_precision; default GBCG_FP64 */
  int32_t max_outer;          /* refinement passes for GBCG_FP32_IR; default 30 */
  double inner_tol;           /* GBCG_FP32_IR: inner relative tolerance, default 1e-4;
                                 GBCG_FP32_RU: residual reduction between updates, default 0.1 */
  int32_t wait_timeout_ms;    /* bound on every device-side wait; default 1000 */
  int32_t max_restarts;       /* true-residual restarts for GBCG_FP64; default 3 */
  int32_t variant;            /* gbcg_variant; default GBCG_STANDARD */
  int32_t pad_;
} gbcg_opts;

/* Report of one solve. */
typedef struct {
  int32_t iterations;         /* CG iterations (inner ones for GBCG_FP32_IR) */
  int32_t outer;              /* restarts (FP64), refinement passes (IR) or reliable updates (RU) */
  int32_t status;             /* same as the return value of gbcg_solve */
  int32_t pad_;
  double rel_res_recursive;   /* ||r_k|| / ||b|| of the recurrence at exit */
  double rel_res_true;        /* ||b - A x|| / ||b|| recomputed in double */
  double ms;                  /* wall time of the call on the host, ms */
  double kernel_ms;           /* device time of the persistent CG launches,
                                 CUDA events on the caller's stream, ms */
  int32_t kernel_launches;    /* persistent CG launches of the call */
  int32_t launches;           /* kernels of this library launched by the call */
} gbcg_info;

/* Layout facts of a created matrix (for measurement and tests). */
typedef struct {
  int64_t n;                  /* rows */
  int64_t nnz_input;          /* entries passed to gbcg_create */
  int64_t nnz_full;           /* entries of the full symmetric operator */
  int64_t stored_slots;       /* SELL slots of the row-gather layout, padding included */
  int64_t plan_slots;         /* SELL slots of the symmetric transpose plan (0 if none) */
  int64_t long_rows;          /* rows handled warp-per-row */
  int64_t device_bytes;       /* device memory held by the handle */
  int64_t spmv_bytes_fp64;    /* algorithmic bytes of one double-precision product (value +
                                 index per entry, row pointers, x read once, y written once) */
  int64_t spmv_bytes_fp32;    /* the same for the single-precision product */
  int64_t ext_slots;          /* symmetric tiles: partial sums leaving the tiles */
  int32_t format;             /* gbcg_format */
  int32_t grid_ctas;          /* CTAs of the persistent CG launch */
  int32_t layout;             /* 0 row gather, 1 symmetric transpose plan, 2 symmetric tiles */
  int32_t tiles;              /* symmetric tiles: number of tiles */
  int32_t index_bytes;        /* bytes per column index in the product's stream: 2 when the
                                 row-gather layout stores 16-bit offsets from the row (every
                                 offset fits; natural-order finite-element matrices up to
                                 about 180^3 nodes), else 4 */
  int32_t pad_;
} gbcg_matrix_stats;

/*
 * gbcg_create -- build a matrix handle (Section III: the CG input is a
 * symmetric sparse matrix in full CSR, symmetric CSR or CSC).
 *
 *   A          out: the new handle (NULL on failure)
 *   format     gbcg_format
 *   n          rows = columns, n >= 0
 *   nnz        stored entries, = ptr[n] - index_base
 *   ptr, idx, val
 *              the arrays of `format`: ptr[n+1] non-decreasing, idx[nnz] in
 *              [index_base, n + index_base), val[nnz] finite doubles.  Within
 *              a row (column for CSC) indices are strictly increasing.  For
 *              GBCG_SYM_CSR_UPPER every idx of row i is >= i.  Symmetry of a
 *              full CSR/CSC input is the caller's promise (it is what CG
 *              needs); the products themselves are exact for any matrix.
 *              Debug mode: with the environment variable
 *              GBCG_CHECK_SYMMETRY=1 the call checks it (entry (i, j) equal
 *              to (j, i) bit for bit, O(nnz) host work) and returns
 *              GBCG_ERR_INVALID naming the first asymmetric entry.
 *   index_base 0 or 1 (the paper's kernel indexes from 1)
 *   memory     gbcg_memory: where ptr/idx/val live
 *   stream     used for the uploads
 *
 * The library deep-copies the arrays into its own device layout (a sliced
 * row-gather layout for the product, a single-precision copy of the values,
 * the solve workspace); the caller may free its arrays when the call returns.
 * Errors: GBCG_ERR_INVALID for malformed input (with the first offending
 * position in gbcg_last_error()), GBCG_ERR_NOMEM, GBCG_ERR_CUDA.
 */
int gbcg_create(gbcg_matrix_t* A, int32_t format, int64_t n, int64_t nnz, const int32_t* ptr,
                const int32_t* idx, const double* val, int32_t index_base, int32_t memory, void* stream);

/* gbcg_destroy -- free a handle and all device memory it holds (NULL is a no-op). */
int gbcg_destroy(gbcg_matrix_t A);

/*
 * gbcg_spmv -- y = A x in double precision (Section III: the A p product of
 * the CG listing), for every storage format.  x and y are device pointers to
 * n doubles, 16-byte aligned (GBCG_ERR_INVALID otherwise), and must not
 * overlap.  Deterministic: the same inputs give the
 * same bits on every call (no floating-point atomics).
 */
int gbcg_spmv(gbcg_matrix_t A, const double* x, double* y, void* stream);

/* gbcg_spmv_f32 -- y = A32 x with the single-precision copy of the values
 * and float vectors (the product of the single-precision variant, Section IV);
 * the same pointer rules as gbcg_spmv. */
int gbcg_spmv_f32(gbcg_matrix_t A, const float* x, float* y, void* stream);

/*
 * gbcg_solve -- conjugate gradient for A x = b (Section III listing).
 *
 *   b      n doubles, device or host memory
 *   x      n doubles, device or host memory (both b and x in the same
 *          space; device vectors 16-byte aligned, GBCG_ERR_INVALID
 *          otherwise); on input the initial guess x0, on output the last
 *          iterate
 *   tol    relative residual target: stop when ||b - A x||_2 <= tol ||b||_2,
 *          checked on the recurrence residual after each r update and then
 *          confirmed on the true residual in double precision
 *   maxit  bound on CG iterations (inner iterations for GBCG_FP32_IR); the
 *          paper's N; <= 0 means n
 *   opts   may be NULL (defaults)
 *   info   may be NULL; filled on every return that got past argument checks
 *
 * Host-memory b/x are staged through buffers allocated at create time; no
 * allocation happens in this call.  The call synchronises `stream` before it
 * returns (it reads the device status once per solve, once per refinement
 * pass for GBCG_FP32_IR).  On GBCG_ERR_MAXIT, _NOT_SPD or _NONFINITE, x holds
 * the last iterate.  On GBCG_ERR_TIMEOUT a device-side wait gave up after
 * opts->wait_timeout_ms and the GPU context remains usable.
 */
int gbcg_solve(gbcg_matrix_t A, const double* b, double* x, double tol, int32_t maxit,
               const gbcg_opts* opts, gbcg_info* info, void* stream);

/* Result of gbcg_solve_async, written to device memory by the solve's last
 * kernel (the fields of gbcg_info that the device knows). */
typedef struct {
  int32_t status;             /* gbcg_status: OK, MAXIT, NOT_SPD, NONFINITE or TIMEOUT */
  int32_t iterations;         /* CG iterations (single-precision ones for GBCG_FP32_RU) */
  int32_t outer;              /* true-residual restarts, or reliable updates (GBCG_FP32_RU) */
  int32_t pad_;
  double rel_res_recursive;   /* ||r_k|| / ||b|| of the recurrence at exit */
  double rel_res_true;        /* ||b - A x|| / ||b|| of the last confirmation or update */
} gbcg_device_info;

/*
 * gbcg_solve_async -- gbcg_solve enqueued on `stream` without synchronising:
 * the solve runs as one persistent launch (precisions GBCG_FP64, either
 * variant, and GBCG_FP32_RU; the refinement GBCG_FP32_IR steers its passes
 * from the host and is rejected with GBCG_ERR_INVALID), and a one-thread
 * kernel then writes the result to `dinfo`.  No host read, no event, no
 * allocation: the call can be captured into a CUDA graph and replayed, the
 * handle's workspace being reused by every replay (one solve of a handle in
 * flight at a time).
 *
 *   b, x   device pointers to n doubles, 16-byte aligned (not checked to be
 *          device memory: host pointers are the caller's error); x holds x0 on entry and the last iterate after
 *          the stream reaches the solve's end
 *   dinfo  device pointer to one gbcg_device_info, written at the end
 *   tol, maxit, opts  as for gbcg_solve
 *
 * Returns GBCG_OK once the work is enqueued, GBCG_ERR_INVALID for a bad
 * argument, GBCG_ERR_CUDA if a launch fails; the solve's own status arrives
 * in dinfo->status.
 */
int gbcg_solve_async(gbcg_matrix_t A, const double* b, double* x, double tol, int32_t maxit,
                     const gbcg_opts* opts, gbcg_device_info* dinfo, void* stream);

/*
 * gbcg_update_values -- replace the values of a handle, same pattern.  `val`
 * holds nnz doubles in the order of the arrays given to gbcg_create (memory:
 * gbcg_memory).  The first call builds and keeps a map from every device
 * value slot to its input entry (host work of the order of gbcg_create's
 * layout build, and 4 bytes per stored slot of device memory); later calls
 * are one gather kernel per value array, writing both precisions.  Used by
 * the differentiable solve, whose values change between calls.  Values are
 * not checked: non-finite values show up as GBCG_ERR_NONFINITE in a solve.
 */
int gbcg_update_values(gbcg_matrix_t A, const double* val, int32_t memory, void* stream);

/*
 * Gradients of a loss L(x) with respect to what the caller stores, for the
 * solution x of A x = b (A symmetric positive-definite).  With lambda the
 * solution of the adjoint system A lambda = dL/dx (same matrix, same
 * solver), dL/db = lambda and dL/dA_ij = -lambda_i x_j.  The configured
 * differentiable form of the Section III solve; no paper counterpart.
 *
 * gbcg_grad_values -- grad[k] = dL/d(stored value k) on the pattern
 * (format, n, nnz, ptr, idx, index_base as for gbcg_create; device arrays):
 * CSR entry k of row i, column j: -lambda_i x_j; CSC entry k of column j,
 * row i: -lambda_i x_j; symmetric upper entry of row i, column j > i (which
 * stands for A_ij and A_ji): -(lambda_i x_j + lambda_j x_i), diagonal:
 * -lambda_i x_i.  lambda, x, grad: device arrays (n, n, nnz).
 */
int gbcg_grad_values(int32_t format, int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                     int32_t index_base, const double* lambda, const double* x, double* grad, void* stream);

/*
 * gbcg_element_grad -- chain rule through a finite-element assembly
 * A = sum_e coef_e Kh_e: element e adds coef_e * w[e*m + k] to stored value
 * pos[e*m + k] (pos < 0: nothing), k < m; then
 * grad_coef[e] = sum_k w[e*m + k] * grad[pos[e*m + k]].  Device arrays;
 * ne elements, m <= 64 pairs each.  For symmetric upper storage list only
 * the vertex pairs a <= b (the stored gradient already holds both halves).
 */
int gbcg_element_grad(int64_t ne, int32_t m, const int32_t* pos, const double* w, const double* grad,
                      double* grad_coef, void* stream);

/*
 * gbcg_assemble -- the same assembly by stored position: val[p] =
 * sum over k in [tptr[p], tptr[p+1]) of tw[k] * coef[telem[k]], summed in
 * that order (no atomics; bitwise reproducible).  Device arrays.
 */
int gbcg_assemble(int64_t nnz, const int64_t* tptr, const int32_t* telem, const double* tw, const double* coef,
                  double* val, void* stream);

/*
 * Ablation baselines: the 2010 structure of the paper's GPU solver (Section
 * III), for measurement only; the solver never uses them.  Device arrays,
 * 0-based, full CSR (GBCG_CSR) or upper triangle and diagonal
 * (GBCG_SYM_CSR_UPPER); no validation beyond null and size checks.
 *
 * gbcg_ablation_spmv -- y = A x.  GBCG_CSR: the "trivial" kernel, one thread
 * per row reading the CSR arrays.  GBCG_SYM_CSR_UPPER: the SCSR + SCSC pair
 * as two launches one after the other: SCSR writes the direct half (D + U) x
 * by rows, SCSC reads the same arrays as columns and scatters the transpose
 * half with floating-point atomic additions (the last bits of y depend on
 * scheduling).
 *
 * gbcg_ablation_solve -- CG as the paper runs it: one launch per SpMV, dot
 * and axpy, each dot product copied to the host (two host round trips per
 * iteration), alpha, beta and the convergence test on the host.  Same
 * stopping rule on the recurrence residual as gbcg_solve, no confirmation;
 * info->rel_res_true is computed at the end.  Allocates its work vectors.
 */
int gbcg_ablation_spmv(int32_t format, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val,
                       const double* x, double* y, void* stream);
int gbcg_ablation_solve(int32_t format, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val,
                        const double* b, double* x, double tol, int32_t maxit, gbcg_info* info, void* stream);

/*
 * gbcg_measure_fp64_fma_rate -- measurement only: the device's FP64 FMA
 * throughput (FMAs per second, not flops), the second roof of the
 * double-precision symmetric product, which spends two FMAs per stored
 * off-diagonal entry (Section III: the direct and the transpose half).
 * Runs a kernel of independent FMA chains at full occupancy on every SM
 * four times on `stream` and reports the fastest of the last three.  Allocates
 * and frees one double of device memory; synchronises.
 */
int gbcg_measure_fp64_fma_rate(double* fma_per_s, void* stream);

/* gbcg_stats -- layout facts of a handle. */
int gbcg_stats(gbcg_matrix_t A, gbcg_matrix_stats* out);

/* gbcg_status_string -- static text for a gbcg_status value. */
const char* gbcg_status_string(int status);

/* gbcg_last_error -- message of the last failed call on this thread ("" if none). */
const char* gbcg_last_error(void);

/*
 * gbcg_selftest_wait_timeout -- check of the bounded device-side wait.  Runs
 * the grid barrier used by the persistent solver on `ctas` co-resident CTAs
 * (0 = the solver's own grid) with one CTA that never arrives, so every other
 * CTA must give up after `timeout_ms` and record GBCG_ERR_TIMEOUT.  Returns
 * GBCG_ERR_TIMEOUT when the wait ended as designed (the expected result),
 * GBCG_OK if the barrier wrongly completed.  No paper counterpart: it tests
 * the library's failure handling without faulting the GPU.
 */
int gbcg_selftest_wait_timeout(int32_t ctas, int32_t timeout_ms, void* stream);

/*
 * gbcg_solve_csr_static -- conjugate gradient for A x = b that allocates no
 * memory: no cudaMalloc, no cudaFree, no allocating library call.  The paper
 * has no counterpart; it exists for callers that cannot allocate device
 * memory -- code running inside a memory pool's or allocator's callback
 * (allocating there re-enters the allocator), latency-critical loops where an
 * allocation would stall or synchronise the device, and plug-ins whose host
 * application owns all device memory.
 *
 *   n, nnz, ptr, idx, val
 *          the full symmetric matrix in 0-based CSR, device pointers, used in
 *          place (sorted, in-range indices are the caller's promise: they are
 *          not checked here)
 *   b, x   device pointers to n doubles; x holds x0 on entry, the solution
 *          on return
 *   tol, maxit, info, stream  as for gbcg_solve (FP64, at most 3 restarts)
 *
 * The solver's scratch (three work vectors, partial sums, barrier and state)
 * lives in one fixed device array of GBCG_STATIC_SCRATCH_BYTES defined in the
 * library, so n must not exceed GBCG_STATIC_MAX_N; larger n is rejected with
 * GBCG_ERR_INVALID.  Every GPU that loads the library holds that array until
 * the process exits.  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress; the address is not cached, so a call
 * after cudaDeviceReset finds the array where the reloaded module put it).
 * The first call on a device also loads the library's device code there;
 * make that first call before any stream capture.  All calls share the array and the call clears what must start at
 * zero, so calls whose GPU work overlaps (several streams or host threads on
 * one device) race: issue one at a time per device.  The call synchronises
 * `stream` before it returns.
 */
#define GBCG_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
#define GBCG_STATIC_MAX_N 680000
int gbcg_solve_csr_static(int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx, const double* val,
                          const double* b, double* x, double tol, int32_t maxit, gbcg_info* info, void* stream);


/* ------------------------------------------------------------ batches ---
 * Many independent SPD systems of uneven size, each with up to eight
 * right-hand sides, solved by one persistent launch of thread-block clusters
 * replayed as a CUDA graph.  Per system and right-hand side the method is
 * the CG iteration of Section III, either in double precision or in the
 * single-precision form of Section IV inside double-precision iterative
 * refinement; the systems share nothing but the launch.
 *
 * Layout ("block-diagonal CSR"): instance i owns rows [row_off[i],
 * row_off[i+1]); ptr[n_tot+1] and idx/val are one 0-based CSR of the whole
 * block-diagonal matrix with global column numbers, and every column of a
 * row of instance i lies in instance i's row range.  Right-hand sides and
 * solutions are n_tot x nrhs row-major (the nrhs values of a row are
 * adjacent).
 */
typedef struct gbcg_batch_s* gbcg_batch_t;

/* Result of one system and right-hand side. */
typedef struct {
  int32_t iterations;     /* inner CG iterations */
  int32_t outer;          /* refinement passes (GBCG_FP64: first run + restarts;
                             GBCG_FP32_RU: reliable updates) */
  int32_t status;         /* gbcg_status */
  int32_t pad_;
  double rel_res_true;    /* ||b - A x|| / ||b|| in double precision at the last check */
} gbcg_batch_info;

/* Options of gbcg_batch_solve; zero fields take the defaults. */
typedef struct {
  int32_t precision;      /* gbcg_precision; default GBCG_FP64 (GBCG_FP32_RU: reliable updates,
                             one double-precision update of every right-hand side of an
                             instance whenever one of them has fallen by inner_tol) */
  int32_t max_outer;      /* passes: default 30 for GBCG_FP32_IR, 4 (one run and up to
                             three true-residual restarts) for GBCG_FP64 */
  double inner_tol;       /* GBCG_FP32_IR inner relative tolerance, default 1e-4;
                             GBCG_FP32_RU reduction between updates, default 0.1 */
  int32_t fixed_order;    /* 1: keep the schedule (by default every solve replans the
                             queue and the group sizes from the measured time per
                             instance, for the next solve) */
  int32_t max_group;      /* clusters one instance may span, 1..8; default 8 (1: none) */
  int32_t force_group;    /* > 0: every instance spans this many clusters (testing) */
  int32_t wait_timeout_ms;/* bound on each wait between the clusters of one instance;
                             default 1000; a wait that runs out ends the launch with
                             GBCG_ERR_TIMEOUT */
} gbcg_batch_opts;

/* Report of one gbcg_batch_solve.  busy_fraction counts an instance's time
 * once per cluster of its group. */
typedef struct {
  double ms;              /* host wall time of the call */
  double kernel_ms;       /* device time of the graph launch (CUDA events) */
  double span_ms;         /* first instance start to last instance end, global timer */
  double busy_fraction;   /* instance time summed / (span x clusters): queue balance */
  int64_t products;       /* inner matrix products summed over instances (eight
                             right-hand sides each) */
  int64_t iterations;     /* inner iterations summed over systems and right-hand sides */
  int32_t max_iterations; /* largest inner iteration count of one right-hand side */
  int32_t launches;       /* kernels launched: the one persistent kernel */
  int32_t graph;          /* 1: the launch was a CUDA graph replay */
  int32_t threads;        /* CTA size of the launch */
  int32_t cluster;        /* CTAs per cluster */
  int32_t clusters;       /* co-resident clusters (the grid) */
  int32_t groups;         /* instances that spanned more than one cluster */
  int32_t max_group;      /* largest number of clusters on one instance */
} gbcg_batch_report;

/* Launch configuration of a batch: chosen by the autotuner or set by hand. */
typedef struct {
  int32_t threads;           /* CTA size: 256 or 512 */
  int32_t cluster;           /* CTAs per cluster: 1, 2, 4, 8 or 16 */
  int32_t rows_per_warp[8];  /* per nnz-per-row bucket b (2^b <= nnz/row < 2^(b+1)):
                                rows a warp works on at once, 1, 2, 4, 8 or 16
                                (16 only for the single-precision inner solve) */
  int32_t clusters;          /* out: co-resident clusters of that configuration */
  int32_t from_cache;        /* out: 1 if taken from the process's tuning cache */
  int32_t candidates;        /* out: probe launches timed */
  int32_t pad_;
  double probe_ms;           /* out: time of the winning probe launch */
} gbcg_batch_tuning;

typedef struct {
  int64_t n;                 /* rows of all instances */
  int64_t nnz;               /* stored entries of all instances */
  int64_t device_bytes;      /* device memory held by the handle */
  int64_t iter_bytes_fp32;   /* algorithmic bytes of one single-precision inner
                                iteration of every instance (matrix once, eight
                                right-hand sides of vectors) */
  int64_t iter_bytes_fp64;   /* the same in double precision */
  int32_t count;             /* instances */
  int32_t nrhs;              /* right-hand sides */
  int32_t threads[2];        /* [0] double, [1] single-precision inner solve */
  int32_t cluster[2];
  int32_t rows_per_warp[2][8];
} gbcg_batch_stats_t;

/*
 * gbcg_batch_create -- build a batch handle.
 *
 *   count      instances, >= 1
 *   row_off    host array of count + 1 row offsets, row_off[0] = 0, non-decreasing
 *   ptr, idx, val
 *              the block-diagonal CSR described above (memory: gbcg_memory);
 *              within a row columns strictly increase; values finite.  Each
 *              instance must be symmetric positive-definite (the caller's promise)
 *   nrhs       right-hand sides per instance, 1..8 (the kernels always carry
 *              eight; fewer leave lanes idle)
 *   tune       1: run the autotuner for the single-precision inner solve now
 *              (or take its cached result for an identical batch shape)
 *
 * Deep-copies the matrix (double and single-precision values), allocates the
 * solve workspace (five vectors of n_tot x 8 values) and the pinned host
 * blocks the graph reads and writes.  Errors: GBCG_ERR_INVALID with the first
 * offending position, GBCG_ERR_NOMEM, GBCG_ERR_CUDA.
 */
int gbcg_batch_create(gbcg_batch_t* B, int32_t count, const int64_t* row_off, const int32_t* ptr, const int32_t* idx,
                      const double* val, int32_t nrhs, int32_t memory, int32_t tune, void* stream);

/* gbcg_batch_destroy -- free a batch handle (NULL is a no-op). */
int gbcg_batch_destroy(gbcg_batch_t B);

/*
 * gbcg_batch_autotune -- choose the CTA size, the cluster size and, per
 * nnz-per-row bucket, the rows per warp of the inner product for `precision`
 * by timing probe launches (every instance runs 16 inner iterations of one
 * refinement pass; each candidate's per-instance times come from the device's
 * global timer).  The result is cached per process by device and batch shape.
 * `rep` may be NULL.  Allocates two temporary n_tot x nrhs vectors.
 */
int gbcg_batch_autotune(gbcg_batch_t B, int32_t precision, gbcg_batch_tuning* rep, void* stream);

/* gbcg_batch_set_tuning -- set the launch configuration of `precision` by hand. */
int gbcg_batch_set_tuning(gbcg_batch_t B, int32_t precision, const gbcg_batch_tuning* t);

/*
 * gbcg_batch_solve -- solve every instance for every right-hand side.
 *
 *   b, x     n_tot x nrhs doubles, both device or both host memory (device
 *            vectors 16-byte aligned, GBCG_ERR_INVALID otherwise); x holds
 *            x0 on entry and the solutions on return
 *   tol      relative residual target per system and right-hand side, checked
 *            on the true residual in double precision
 *   maxit    bound on inner iterations per system and right-hand side; <= 0
 *            means the instance's row count
 *   opts     may be NULL (double precision)
 *   infos    host array of count x nrhs results (instance-major), may be NULL
 *   rep      may be NULL
 *
 * The first call per precision (and the first after a tuning change)
 * captures the solve graph: upload of the argument block, queue reset, the
 * persistent launch and the result downloads; later calls replay it.  No
 * device allocation.  Returns GBCG_OK when every system converged, else the
 * status of the first failing one in instance order; synchronises `stream`.
 */
int gbcg_batch_solve(gbcg_batch_t B, const double* b, double* x, double tol, int32_t maxit,
                     const gbcg_batch_opts* opts, gbcg_batch_info* infos, gbcg_batch_report* rep, void* stream);

/*
 * gbcg_batch_selftest_group_timeout -- check of the bounded wait between the
 * clusters of one instance.  Runs the batch kernel with the last instance of
 * the queue made a group of two clusters whose second part is left out of
 * the queue, so its first part must give up after `timeout_ms` and end the
 * launch.  Returns GBCG_ERR_TIMEOUT when the wait ended as designed (the
 * expected result), GBCG_OK if it wrongly completed.  Needs two co-resident
 * clusters.  No paper counterpart: it tests failure handling without
 * faulting the GPU.
 */
int gbcg_batch_selftest_group_timeout(gbcg_batch_t B, int32_t timeout_ms, void* stream);

/* gbcg_batch_instance_times -- of the last solve, per instance: global-timer
 * start and end (2 x count, ns), inner products and double-precision residual
 * products.  Any output may be NULL. */
int gbcg_batch_instance_times(gbcg_batch_t B, int64_t* t_ns, int32_t* products, int32_t* outer_products);

/* gbcg_batch_stats -- shape, memory and launch configuration of a batch. */
int gbcg_batch_stats(gbcg_batch_t B, gbcg_batch_stats_t* out);

#ifdef __cplusplus
}
#endif
#endif /* GBCG_H */
