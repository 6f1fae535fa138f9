/*
 * oracle.c -- plain, slow, obviously correct CPU implementation of what the
 * GPU solver computes.  TEST INFRASTRUCTURE ONLY: it is loaded by the tests,
 * by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * library.  It shares no code with the CUDA path.
 *
 * Everything is IEEE double precision (single precision only where the paper's
 * single-precision solver is restated), written as the textbook definitions:
 * no blocking, no fusion, no reordering.  Build with -ffp-contract=off so a
 * multiply and an add are two roundings on every host.
 *
 * Sections of "Parallel Sparse Matrix Solver on the GPU Applied to Simulation
 * of Electrical Machines" (Rodrigues, Guyomarc'h, Le Menach, Dekeyser):
 *   - Section III, the CG listing: alpha = r'r / p'Ap; x += alpha p; break on
 *     convergence; r -= alpha Ap; beta = r_k'r_k / r_{k-1}'r_{k-1};
 *     p = r + beta p; for 1 <= k <= N.
 *   - Section III, after the listing: A = L + D + U with U' = L, so A can be
 *     stored as the triangle L + D; the SCSR kernel applies L + D by rows and
 *     the SCSC kernel applies U by reading the same arrays as columns.
 *   - Section III: the "trivial" kernel forms y[row] += A[k] * x[col[k]] over
 *     the row's stored entries (full CSR).
 *   - Section IV: a double-precision CPU CG is the reference; a
 *     single-precision GPU CG is the other variant.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   1. "init variables": x0 given (default 0), r0 = b - A x0, p0 = r0.
 *   2. "convergence": ||r_k||_2 / ||b||_2 <= tol, tested on the updated
 *      residual right after the r update (one step later than the listing's
 *      position, which sits between the x and r updates and so could only
 *      test the previous residual); a solve is declared converged only once
 *      the true residual ||b - A x||_2 / ||b||_2 <= tol; otherwise the
 *      recurrence restarts from r = b - A x, p = r (at most 3 restarts).
 *   3. N (the iteration bound) is the caller's maxit; b = 0 gives x = 0.
 *   4. Symmetric storage is the upper triangle D + U stored by rows, which
 *      holds the same numbers as the paper's L + D stored by rows (read as
 *      columns); entry (i, j), j > i, acts for both (i, j) and (j, i).
 *   5. Breakdown: p'Ap not finite -> NONFINITE; p'Ap <= 0 -> NOT_SPD.
 *   6. Single-precision variant: the same recurrence in float (values,
 *      vectors and dots), used as the inner solver of an iterative-refinement
 *      loop whose residual b - A x, correction x += ||r|| d and norms are in
 *      double precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_INVALID = 1, ORC_NOT_SPD = 2, ORC_MAXIT = 3, ORC_NONFINITE = 4 };
enum { ORC_CSR = 0, ORC_SYM_UPPER = 1, ORC_CSC = 2 };

typedef struct {
  int32_t iterations;     /* CG iterations (inner iterations for refinement) */
  int32_t restarts;       /* residual replacements (outer passes for refinement) */
  int32_t status;
  int32_t pad_;
  double rel_res_recursive;
  double rel_res_true;
} orc_info;

/* ------------------------------------------------ sparse products -------- */
/* Full CSR (the "trivial" kernel of Section III): y_i = sum_k val[k] x[idx[k]]. */
void orc_spmv_csr(int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* x,
                  double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) s += val[k] * x[idx[k]];
    y[i] = s;
  }
}

/* Symmetric storage (Section III, A = L + D + U, U' = L): rows hold D + U.
 * Entry (i, j) adds a_ij x_j to y_i and, when j > i, a_ij x_i to y_j. */
void orc_spmv_sym_upper(int64_t n, const int32_t* ptr, const int32_t* idx, const double* val,
                        const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      int64_t j = idx[k];
      y[i] += val[k] * x[j];
      if (j > i) y[j] += val[k] * x[i];
    }
  }
}

/* Column storage (the SCSC view of Section III): column j holds the entries
 * a_ij, i = rowidx[k]; y = sum_j a_:j x_j, columns in increasing order. */
void orc_spmv_csc(int64_t n, const int32_t* colptr, const int32_t* rowidx, const double* val,
                  const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = colptr[j]; k < colptr[j + 1]; ++k) y[rowidx[k]] += val[k] * x[j];
}

void orc_spmv(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* x,
              double* y) {
  if (fmt == ORC_SYM_UPPER)
    orc_spmv_sym_upper(n, ptr, idx, val, x, y);
  else if (fmt == ORC_CSC)
    orc_spmv_csc(n, ptr, idx, val, x, y);
  else
    orc_spmv_csr(n, ptr, idx, val, x, y);
}

/* Same products in single precision (values and vectors float). */
void orc_spmv_f32(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const float* val, const float* x,
                  float* y) {
  if (fmt == ORC_CSR) {
    for (int64_t i = 0; i < n; ++i) {
      float s = 0.0f;
      for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) s += val[k] * x[idx[k]];
      y[i] = s;
    }
    return;
  }
  for (int64_t i = 0; i < n; ++i) y[i] = 0.0f;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      int64_t j = idx[k];
      if (fmt == ORC_CSC) {
        y[j] += val[k] * x[i];
      } else {
        y[i] += val[k] * x[j];
        if (j > i) y[j] += val[k] * x[i];
      }
    }
}

/* |A| |x| row by row: the scale of the componentwise rounding bound of a
 * product (used by the tests as the denominator of the SpMV tolerance). */
void orc_abs_spmv(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* x,
                  double* y) {
  for (int64_t i = 0; i < n; ++i) y[i] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      int64_t j = idx[k];
      double a = fabs(val[k]);
      if (fmt == ORC_CSC) {
        y[j] += a * fabs(x[i]);
      } else {
        y[i] += a * fabs(x[j]);
        if (fmt == ORC_SYM_UPPER && j > i) y[j] += a * fabs(x[i]);
      }
    }
}

/* ------------------------------------------------ vector kernels --------- */
double orc_dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Dot product accumulated in long double: a checker for the GPU reductions. */
double orc_dot_long(int64_t n, const double* a, const double* b) {
  long double s = 0.0L;
  for (int64_t i = 0; i < n; ++i) s += (long double)a[i] * (long double)b[i];
  return (double)s;
}

/* Single-precision dot product.  Section III computes the scalar products
 * with CuBLAS, a GPU library whose reduction adds partial sums in a tree, not
 * left to right; the same order is taken here: halves summed recursively
 * (pairwise summation), so the float rounding error grows like log2(n) eps
 * instead of the n eps of a running sum. */
static float dot_f(int64_t n, const float* a, const float* b) {
  if (n <= 8) {
    float s = 0.0f;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
  }
  const int64_t h = n / 2;
  return dot_f(h, a, b) + dot_f(n - h, a + h, b + h);
}

float orc_dot_f32(int64_t n, const float* a, const float* b) { return dot_f(n, a, b); }

/* ------------------------------------------------ multi-threaded build --- */
/* The same file compiled with -fopenmp gives a second, separate library (the
 * oracle timed on every host core, and the way its large reference solves
 * are computed).  That build must give the single-threaded build's bits:
 *   - element-wise vector loops run their elements on several threads (each
 *     element is computed exactly as before);
 *   - the double-precision dot product stays one left-to-right sum;
 *   - the single-precision pairwise dot computes the subtrees of its top
 *     levels on several threads and adds them in the tree's own order;
 *   - the symmetric and column-storage products run output by output: y_j
 *     adds the terms that the row-order loop of orc_spmv_sym_upper (or the
 *     column-order loop of orc_spmv_csc) adds to y_j, in the same order --
 *     transpose terms a_ij x_i by increasing source i, then (symmetric) the
 *     entries of row j in storage order -- through an index of those terms
 *     built once per solve.
 * Without -fopenmp every pragma below is ignored and the products are the
 * plain loops above. */
int32_t orc_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int32_t t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads((int)t);
#else
  (void)t;
#endif
}

/* Operand of the CG loops: the matrix in its storage format, its float
 * values when the loop needs them, and (multi-threaded build, symmetric or
 * column storage) the index of the terms each output receives from other
 * rows: for output j, tk[tptr[j] .. tptr[j+1]) are the storage positions k
 * of the entries aimed at j, by increasing source row (column for CSC), and
 * ts[] those sources. */
typedef struct {
  int fmt;
  int64_t n;
  const int32_t* ptr;
  const int32_t* idx;
  const double* val;
  const float* val32;
  int64_t* tptr;
  int64_t* tk;
  int32_t* ts;
} orc_op;

static void op_init(orc_op* A, int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val,
                    const float* val32) {
  A->fmt = fmt;
  A->n = n;
  A->ptr = ptr;
  A->idx = idx;
  A->val = val;
  A->val32 = val32;
  A->tptr = NULL;
  A->tk = NULL;
  A->ts = NULL;
#ifdef _OPENMP
  if (fmt == ORC_CSR || n <= 0) return;
  /* counting sort of the terms by output, sources visited in increasing order */
  int64_t* tptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
      if (fmt == ORC_CSC || idx[k] > i) ++tptr[idx[k] + 1];
  for (int64_t j = 0; j < n; ++j) tptr[j + 1] += tptr[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(fill, tptr, sizeof(int64_t) * (size_t)n);
  int64_t* tk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tptr[n] ? tptr[n] : 1));
  int32_t* ts = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tptr[n] ? tptr[n] : 1));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
      if (fmt == ORC_CSC || idx[k] > i) {
        const int64_t at = fill[idx[k]]++;
        tk[at] = k;
        ts[at] = (int32_t)i;
      }
  free(fill);
  A->tptr = tptr;
  A->tk = tk;
  A->ts = ts;
#endif
}

static void op_free(orc_op* A) {
  free(A->tptr);
  free(A->tk);
  free(A->ts);
}

/* y = A x in double precision (orc_spmv's arithmetic, see above). */
static void op_spmv(const orc_op* A, const double* x, double* y) {
#ifdef _OPENMP
  const int64_t n = A->n;
  if (A->fmt == ORC_CSR) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = A->ptr[i]; k < A->ptr[i + 1]; ++k) s += A->val[A->idx ? k : k] * x[A->idx[k]];
      y[i] = s;
    }
    return;
  }
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t t = A->tptr[j]; t < A->tptr[j + 1]; ++t) s += A->val[A->tk[t]] * x[A->ts[t]];
    if (A->fmt == ORC_SYM_UPPER)
      for (int64_t k = A->ptr[j]; k < A->ptr[j + 1]; ++k) s += A->val[k] * x[A->idx[k]];
    y[j] = s;
  }
#else
  orc_spmv(A->fmt, A->n, A->ptr, A->idx, A->val, x, y);
#endif
}

/* y = A32 x in single precision (orc_spmv_f32's arithmetic). */
static void op_spmv_f32(const orc_op* A, const float* x, float* y) {
#ifdef _OPENMP
  const int64_t n = A->n;
  if (A->fmt == ORC_CSR) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      float s = 0.0f;
      for (int64_t k = A->ptr[i]; k < A->ptr[i + 1]; ++k) s += A->val32[k] * x[A->idx[k]];
      y[i] = s;
    }
    return;
  }
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    float s = 0.0f;
    for (int64_t t = A->tptr[j]; t < A->tptr[j + 1]; ++t) s += A->val32[A->tk[t]] * x[A->ts[t]];
    if (A->fmt == ORC_SYM_UPPER)
      for (int64_t k = A->ptr[j]; k < A->ptr[j + 1]; ++k) s += A->val32[k] * x[A->idx[k]];
    y[j] = s;
  }
#else
  orc_spmv_f32(A->fmt, A->n, A->ptr, A->idx, A->val32, x, y);
#endif
}

/* dot_f with the subtrees of its top levels summed on several threads and
 * combined in the tree's order (the same bits as dot_f). */
static float dotf(int64_t n, const float* a, const float* b) {
#ifdef _OPENMP
  enum { DEPTH = 6, LEAVES = 1 << DEPTH };
  if (n >= ((int64_t)1 << 16)) {
    int64_t off[LEAVES], len[LEAVES];
    off[0] = 0;
    len[0] = n;
    for (int d = 0, cnt = 1; d < DEPTH; ++d, cnt *= 2)
      for (int u = cnt - 1; u >= 0; --u) {  /* node u splits into 2u, 2u + 1 as dot_f halves it */
        const int64_t o = off[u], m = len[u], h = m / 2;
        off[2 * u] = o;
        len[2 * u] = h;
        off[2 * u + 1] = o + h;
        len[2 * u + 1] = m - h;
      }
    float part[LEAVES];
#pragma omp parallel for schedule(static)
    for (int u = 0; u < LEAVES; ++u) part[u] = dot_f(len[u], a + off[u], b + off[u]);
    for (int cnt = LEAVES / 2; cnt >= 1; cnt /= 2)
      for (int u = 0; u < cnt; ++u) part[u] = part[2 * u] + part[2 * u + 1];
    return part[0];
  }
#endif
  return dot_f(n, a, b);
}

/* ------------------------------------------------ conjugate gradient ----- */
/* History buffers (may be NULL): for k = 0..hist_cap-1 the search direction
 * p_k and the iterate x_{k+1}, n values each; alpha/beta per iteration. */
typedef struct {
  int32_t cap;
  int32_t count;
  double* p;
  double* x;
  double* alpha;
  double* beta;
} orc_history;

int orc_cg(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* b,
           double* x, double tol, int32_t maxit, orc_info* info, orc_history* hist) {
  memset(info, 0, sizeof(*info));
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) {
    info->status = ORC_INVALID;
    return ORC_INVALID;
  }
  double* r = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  if (hist) hist->count = 0;
  orc_op A;
  op_init(&A, fmt, n, ptr, idx, val, NULL);
  int status = ORC_OK;
  int32_t k = 0, restarts = 0;
  double nb = sqrt(orc_dot(n, b, b));
  double rr = 0.0;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  /* reading 1: r0 = b - A x0, p0 = r0 */
  op_spmv(&A, x, q);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) p[i] = r[i];
  rr = orc_dot(n, r, r);
  for (;;) {
    while (k < maxit && !(sqrt(rr) / nb <= tol)) {
      op_spmv(&A, p, q);                             /* A p */
      double pq = orc_dot(n, p, q);                  /* p' A p */
      if (!isfinite(pq)) { status = ORC_NONFINITE; goto done; }
      if (!(pq > 0.0)) { status = ORC_NOT_SPD; goto done; }
      double alpha = rr / pq;                        /* alpha = r'r / p'Ap */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];   /* x += alpha p */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];   /* r -= alpha A p */
      double rr_new = orc_dot(n, r, r);
      ++k;
      double beta = rr_new / rr;                     /* beta = r_k'r_k / r_{k-1}'r_{k-1} */
      if (hist && hist->count < hist->cap) {
        int32_t h = hist->count++;
        if (hist->p) memcpy(hist->p + (size_t)h * n, p, sizeof(double) * n);
        if (hist->x) memcpy(hist->x + (size_t)h * n, x, sizeof(double) * n);
        if (hist->alpha) hist->alpha[h] = alpha;
        if (hist->beta) hist->beta[h] = beta;
      }
      rr = rr_new;
      if (!isfinite(rr)) { status = ORC_NONFINITE; goto done; }
      if (sqrt(rr) / nb <= tol) break;               /* reading 2: test after the r update */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];  /* p = r + beta p */
    }
    /* reading 2: confirm with the true residual; restart from it otherwise */
    op_spmv(&A, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double rt = orc_dot(n, r, r);
    info->rel_res_true = sqrt(rt) / nb;
    if (info->rel_res_true <= tol) break;
    if (k >= maxit || restarts >= 3) { status = ORC_MAXIT; break; }
    ++restarts;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i];
    rr = rt;
  }
done:
  info->iterations = k;
  info->restarts = restarts;
  info->status = status;
  info->rel_res_recursive = nb > 0.0 ? sqrt(rr) / nb : 0.0;
  if (status != ORC_OK && status != ORC_MAXIT) info->rel_res_true = NAN;
  if (nb == 0.0) info->rel_res_true = 0.0;
  op_free(&A);
  free(r);
  free(p);
  free(q);
  return status;
}

/* Single-reduction ("pipelined") CG.  The Chronopoulos-Gear form of the
 * Section III iteration, rearranged (Ghysels and Vanroose) so that both inner
 * products of an iteration, r'r and w'r with w = A r, are formed together
 * and the product q = A w does not wait for them.  With s = A p and z = A s
 * kept by recurrence:
 *   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
 *   (first step: beta = 0, alpha = gamma / delta); the denominator is p'Ap;
 *   z = q + beta z, s = w + beta s, p = r + beta p,
 *   x += alpha p, r -= alpha s, w -= alpha z.
 * In exact arithmetic x_k equals the Section III iterate.  Stopping rule,
 * true-residual confirmation and restarts (from r = b - A x, w = A r, p = r)
 * as in orc_cg.  Its recurrences for r and w drift from b - A x and A r
 * faster than the Section III ones, so it restarts more often; and its p'Ap,
 * formed by the recurrence delta - beta gamma / alpha_old, cancels near the
 * attainable residual, so a non-positive value there also ends the run into
 * the confirmation.  Only on the first step of a run (p'Ap = r'Ar) does it
 * show that A is not positive definite.  The history
 * records x after each iteration. */
int orc_cg_pipelined(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* b,
                     double* x, double tol, int32_t maxit, orc_info* info, orc_history* hist) {
  memset(info, 0, sizeof(*info));
  if (n < 0 || maxit < 0 || !(tol >= 0.0)) {
    info->status = ORC_INVALID;
    return ORC_INVALID;
  }
  const size_t nn = (size_t)(n ? n : 1);
  double* r = (double*)malloc(sizeof(double) * nn);
  double* w = (double*)malloc(sizeof(double) * nn);
  double* p = (double*)malloc(sizeof(double) * nn);
  double* s = (double*)malloc(sizeof(double) * nn);
  double* z = (double*)malloc(sizeof(double) * nn);
  double* q = (double*)malloc(sizeof(double) * nn);
  if (hist) hist->count = 0;
  int status = ORC_OK;
  int32_t k = 0, restarts = 0;
  double nb = sqrt(orc_dot(n, b, b));
  double gamma = 0.0;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  for (;;) {
    orc_spmv(fmt, n, ptr, idx, val, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];      /* r = b - A x */
    orc_spmv(fmt, n, ptr, idx, val, r, w);                   /* w = A r */
    double gamma_old = 0.0, alpha_old = 0.0;
    int first = 1;
    for (;;) {
      gamma = orc_dot(n, r, r);
      const double delta = orc_dot(n, w, r);
      if (!isfinite(gamma) || !isfinite(delta)) { status = ORC_NONFINITE; goto done; }
      if (sqrt(gamma) / nb <= tol || k >= maxit) break;
      orc_spmv(fmt, n, ptr, idx, val, w, q);                 /* q = A w */
      const double beta = first ? 0.0 : gamma / gamma_old;
      const double den = first ? delta : delta - beta * gamma / alpha_old;   /* p'Ap */
      if (!isfinite(den)) { status = ORC_NONFINITE; goto done; }
      if (!(den > 0.0)) {
        /* on a first step den = r'Ar: A is not positive definite; later, the
         * recurrence for p'Ap has lost its accuracy (near the attainable
         * residual): confirm and restart from the true residual */
        if (first) { status = ORC_NOT_SPD; goto done; }
        break;
      }
      const double alpha = gamma / den;
      for (int64_t i = 0; i < n; ++i) {
        z[i] = (first ? 0.0 : beta * z[i]) + q[i];
        s[i] = (first ? 0.0 : beta * s[i]) + w[i];
        p[i] = (first ? 0.0 : beta * p[i]) + r[i];
      }
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * s[i];
        w[i] -= alpha * z[i];
      }
      ++k;
      if (hist && hist->count < hist->cap) {
        int32_t h = hist->count++;
        if (hist->p) memcpy(hist->p + (size_t)h * n, p, sizeof(double) * n);
        if (hist->x) memcpy(hist->x + (size_t)h * n, x, sizeof(double) * n);
        if (hist->alpha) hist->alpha[h] = alpha;
        if (hist->beta) hist->beta[h] = beta;
      }
      gamma_old = gamma;
      alpha_old = alpha;
      first = 0;
    }
    orc_spmv(fmt, n, ptr, idx, val, x, q);
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    const double rt = orc_dot(n, q, q);
    info->rel_res_true = sqrt(rt) / nb;
    if (info->rel_res_true <= tol) break;
    if (k >= maxit || restarts >= 3) { status = ORC_MAXIT; break; }
    ++restarts;
  }
done:
  info->iterations = k;
  info->restarts = restarts;
  info->status = status;
  info->rel_res_recursive = nb > 0.0 ? sqrt(gamma) / nb : 0.0;
  if (status != ORC_OK && status != ORC_MAXIT) info->rel_res_true = NAN;
  if (nb == 0.0) info->rel_res_true = 0.0;
  free(r);
  free(w);
  free(p);
  free(s);
  free(z);
  free(q);
  return status;
}

/* Single-precision CG (Section IV's single-precision variant): solves
 * A32 d = rhs from d = 0 until ||r|| <= tol ||rhs|| or maxit; float
 * throughout.  Returns iterations used; *breakdown set on p'Ap <= 0. */
int32_t orc_cg_f32(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const float* val, const float* rhs,
                   float* d, float tol, int32_t maxit, int32_t* breakdown) {
  float* r = (float*)malloc(sizeof(float) * (size_t)(n ? n : 1));
  float* p = (float*)malloc(sizeof(float) * (size_t)(n ? n : 1));
  float* q = (float*)malloc(sizeof(float) * (size_t)(n ? n : 1));
  *breakdown = 0;
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0f;
    r[i] = rhs[i];
    p[i] = rhs[i];
  }
  float nr0 = sqrtf(dot_f(n, rhs, rhs));
  float rr = nr0 * nr0;
  int32_t k = 0;
  while (k < maxit && nr0 > 0.0f && !(sqrtf(rr) <= tol * nr0)) {
    orc_spmv_f32(fmt, n, ptr, idx, val, p, q);
    float pq = dot_f(n, p, q);
    if (!(pq > 0.0f) || !isfinite(pq)) { *breakdown = 1; break; }
    float alpha = rr / pq;
    for (int64_t i = 0; i < n; ++i) d[i] += alpha * p[i];
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    float rr_new = dot_f(n, r, r);
    ++k;
    if (sqrtf(rr_new) <= tol * nr0) break;
    float beta = rr_new / rr;
    rr = rr_new;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
  }
  free(r);
  free(p);
  free(q);
  return k;
}

/* Mixed precision by iterative refinement: outer residual, norms and the
 * correction in double precision; inner solve A32 d = r / ||r|| in float.
 * maxit bounds the total inner iterations, max_outer the refinement passes. */
int orc_cg_ir(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* b,
              double* x, double tol, int32_t maxit, double inner_tol, int32_t max_outer, orc_info* info) {
  memset(info, 0, sizeof(*info));
  int64_t nnz = n > 0 ? ptr[n] : 0;
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(nnz ? nnz : 1));
  float* rs = (float*)malloc(sizeof(float) * (size_t)(n ? n : 1));
  float* d = (float*)malloc(sizeof(float) * (size_t)(n ? n : 1));
  double* r = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)val[k];
  int status = ORC_MAXIT;
  int32_t used = 0, outer = 0;
  double nb = sqrt(orc_dot(n, b, b));
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    status = ORC_OK;
    goto done;
  }
  for (;;) {
    orc_spmv(fmt, n, ptr, idx, val, x, r);                      /* A x in double */
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];         /* r = b - A x */
    double nr = sqrt(orc_dot(n, r, r));
    info->rel_res_true = nr / nb;
    if (!isfinite(nr)) { status = ORC_NONFINITE; break; }
    if (nr / nb <= tol) { status = ORC_OK; break; }
    if (outer >= max_outer || used >= maxit) { status = ORC_MAXIT; break; }
    for (int64_t i = 0; i < n; ++i) rs[i] = (float)(r[i] / nr);
    int32_t bd = 0;
    int32_t it = orc_cg_f32(fmt, n, ptr, idx, v32, rs, d, (float)inner_tol, maxit - used, &bd);
    used += it;
    ++outer;
    if (bd && it == 0) { status = ORC_NOT_SPD; break; }
    for (int64_t i = 0; i < n; ++i) x[i] += nr * (double)d[i];  /* x += ||r|| d */
  }
done:
  info->iterations = used;
  info->restarts = outer;
  info->status = status;
  info->rel_res_recursive = info->rel_res_true;
  free(v32);
  free(rs);
  free(d);
  free(r);
  return status;
}

/* ------------------------------------------------ differentiation -------- */
/* Gradient of a loss L(x) through x = A^-1 b (the configured differentiable
 * form of the Section III solve).  With lambda = A^-T dL/dx (the adjoint
 * solve; A is symmetric, so A lambda = dL/dx) the derivative with respect to
 * matrix entry A_ij is -lambda_i x_j.  For each STORED value:
 *   CSR:  value k of row i, column j = idx[k]        -> -lambda_i x_j
 *   CSC:  value k of column j, row i = idx[k]        -> -lambda_i x_j
 *   symmetric upper: value k of row i, column j >= i stands for A_ij and A_ji:
 *         j > i -> -(lambda_i x_j + lambda_j x_i),   j = i -> -lambda_i x_i. */
void orc_grad_values(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* lambda,
                     const double* x, double* g) {
  for (int64_t r = 0; r < n; ++r)
    for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) {
      const int64_t c = idx[k];
      if (fmt == ORC_CSC) {                      /* r is the column, c the row */
        g[k] = -(lambda[c] * x[r]);
      } else if (fmt == ORC_SYM_UPPER && c != r) {
        g[k] = -(lambda[r] * x[c] + lambda[c] * x[r]);
      } else {
        g[k] = -(lambda[r] * x[c]);
      }
    }
}

/* Chain rule through the assembly A = sum_e coef_e Kh_e: with the stored
 * positions pos[e*m + k] (-1: none) and weights w[e*m + k] of element e,
 * dL/dcoef_e = sum_k w[e*m+k] * g[pos[e*m+k]]. */
void orc_element_grad(int64_t ne, int32_t m, const int32_t* pos, const double* w, const double* g, double* gc) {
  for (int64_t e = 0; e < ne; ++e) {
    double s = 0.0;
    for (int32_t k = 0; k < m; ++k) {
      const int32_t p = pos[e * m + k];
      if (p >= 0) s += w[e * m + k] * g[p];
    }
    gc[e] = s;
  }
}

/* The assembly itself, by stored position: val[p] = sum over the
 * contributions (elem, weight) at tptr[p]..tptr[p+1] of weight * coef_elem. */
void orc_assemble(int64_t nnz, const int64_t* tptr, const int32_t* telem, const double* tw, const double* coef,
                  double* val) {
  for (int64_t p = 0; p < nnz; ++p) {
    double s = 0.0;
    for (int64_t k = tptr[p]; k < tptr[p + 1]; ++k) s += tw[k] * coef[telem[k]];
    val[p] = s;
  }
}

/* Mixed precision with reliable updates.  Single-precision CG iterations on
 * A32 (the single-precision variant of Section IV, float dots, alpha and
 * beta) build a correction d; each time the recurrence residual has fallen
 * by the factor delta since the last update, and when it reaches tol, the
 * correction is added to the double-precision solution (x += d, d = 0) and the
 * single-precision residual is replaced by the double-precision b - A x.  The
 * search direction p is kept, so the Krylov space is not restarted (the
 * refinement of orc_cg_ir restarts it every pass).  Converged when an
 * update's true residual is <= tol ||b||.  restarts counts the updates. */
int orc_cg_ru(int fmt, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* b,
              double* x, double tol, int32_t maxit, double delta, orc_info* info) {
  memset(info, 0, sizeof(*info));
  int64_t nnz = n > 0 ? (fmt == ORC_CSC ? ptr[n] : ptr[n]) : 0;
  const size_t nn = (size_t)(n ? n : 1);
  float* v32 = (float*)malloc(sizeof(float) * (size_t)(nnz ? nnz : 1));
  float* r = (float*)malloc(sizeof(float) * nn);
  float* p = (float*)malloc(sizeof(float) * nn);
  float* q = (float*)malloc(sizeof(float) * nn);
  float* d = (float*)malloc(sizeof(float) * nn);
  double* r64 = (double*)malloc(sizeof(double) * nn);
  for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)val[k];
  orc_op A;
  op_init(&A, fmt, n, ptr, idx, val, v32);
  int status = ORC_MAXIT;
  int32_t k = 0, updates = 0;
  const double nb = sqrt(orc_dot(n, b, b));
  double rel = 0.0;
  float rr = 0.0f, rmax = 0.0f;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    status = ORC_OK;
    goto done;
  }
  /* the double-precision residual, replacing the single-precision one */
  op_spmv(&A, x, r64);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r64[i] = b[i] - r64[i];
  rel = sqrt(orc_dot(n, r64, r64)) / nb;
  if (!isfinite(rel)) { status = ORC_NONFINITE; goto done; }
  if (rel <= tol) { status = ORC_OK; goto done; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    r[i] = (float)r64[i];
    p[i] = r[i];
    d[i] = 0.0f;
  }
  rr = dotf(n, r, r);
  rmax = sqrtf(rr);
  while (k < maxit) {
    op_spmv_f32(&A, p, q);                                          /* A32 p */
    const float pq = dotf(n, p, q);
    if (!isfinite(pq)) { status = ORC_NONFINITE; break; }
    if (!(pq > 0.0f)) { status = ORC_NOT_SPD; break; }
    const float alpha = rr / pq;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) d[i] += alpha * p[i];           /* correction */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    float rr_new = dotf(n, r, r);
    ++k;
    if (sqrtf(rr_new) < (float)delta * rmax || sqrtf(rr_new) <= (float)(tol * nb) || k >= maxit) {
      /* reliable update: x += d in double, r = b - A x in double */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        x[i] += (double)d[i];
        d[i] = 0.0f;
      }
      op_spmv(&A, x, r64);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) r64[i] = b[i] - r64[i];
      rel = sqrt(orc_dot(n, r64, r64)) / nb;
      ++updates;
      if (!isfinite(rel)) { status = ORC_NONFINITE; break; }
      if (rel <= tol) { status = ORC_OK; break; }
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) r[i] = (float)r64[i];
      rr_new = dotf(n, r, r);
      rmax = sqrtf(rr_new);
    }
    const float beta = rr_new / rr;
    rr = rr_new;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
  }
done:
  if (status == ORC_NOT_SPD || status == ORC_NONFINITE || status == ORC_MAXIT) {
    /* leave the last correction in x */
    for (int64_t i = 0; i < n && k > 0; ++i) x[i] += (double)d[i];
  }
  info->iterations = k;
  info->restarts = updates;
  info->status = status;
  info->rel_res_true = rel;
  info->rel_res_recursive = rel;
  op_free(&A);
  free(v32);
  free(r);
  free(p);
  free(q);
  free(d);
  free(r64);
  return status;
}
