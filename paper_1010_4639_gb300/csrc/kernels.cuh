// kernels.cuh -- device code of the GB300 conjugate-gradient library (sm_103a).
//
// Sparse product (Section III, "A p product on line 2"): the sliced row-gather
// layout of layout.h, one warp per slice of 32 rows and one lane per row, as
// in the paper's thread-per-row kernel but with the row data interleaved so
// that each warp load is one contiguous segment.  The symmetric format adds
// the transpose half U' x as a second gather through the transpose plan,
// reading U's values in place (the paper used a separate scatter kernel with
// atomics; here every output element is summed by one lane in a fixed
// order, so results are bitwise reproducible).
//
// CG iteration (Section III listing): one persistent cooperative launch per
// solve.  Each CTA owns a contiguous range of slices (and so of rows); per
// iteration it runs
//   A: q = A p on its rows, partial p'q            -> grid barrier
//   B: alpha = r'r / p'q; x += alpha p; r -= alpha q; partial r'r -> barrier
//   C: beta = r_k'r_k / r_{k-1}'r_{k-1}; p = r + beta p           -> barrier
// The partial sums of all CTAs are added by every CTA in the same fixed
// order, so every CTA takes the same decisions.  Every grid-barrier wait is
// bounded by a global-timer limit; on expiry the CTA records GBCG_ERR_TIMEOUT
// and returns, so a lost CTA cannot hang the device.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbcg {

constexpr int kCgThreads = 512;
constexpr uint16_t kPlanPad = 0xFFFF;

enum DevStatus { kOk = 0, kNotSpd = 2, kMaxit = 3, kNonfinite = 4, kTimeout = 5 };

template <typename V>
struct OpDev {
  int64_t n = 0, nslices = 0, nlong = 0;
  const int64_t* __restrict__ sl_ptr = nullptr;
  const int32_t* __restrict__ col = nullptr;
  const V* __restrict__ val = nullptr;
  const uint32_t* __restrict__ long_mask = nullptr;
  const int32_t* __restrict__ long_row = nullptr;
  const int64_t* __restrict__ long_ptr = nullptr;
  const int32_t* __restrict__ long_col = nullptr;
  const V* __restrict__ long_val = nullptr;
  // symmetric layout only
  const V* __restrict__ diag = nullptr;
  const int64_t* __restrict__ pl_ptr = nullptr;
  const int32_t* __restrict__ pl_i = nullptr;
  const uint16_t* __restrict__ pl_k = nullptr;
};

struct GridBar {
  unsigned long long count;  // arrivals since launch (monotone)
  int32_t status;            // first failure recorded by any CTA
  int32_t where;             // barrier index of that failure
};

struct CgState {
  double rr;        // r'r of the recurrence at exit
  double nb;        // ||b||
  double rel_true;  // true relative residual of the confirm step (outer solve)
  int32_t k;        // iterations done
  int32_t restarts; // true-residual restarts
  int32_t status;   // DevStatus
  int32_t pad_;
};

template <typename V>
struct CgArgs {
  OpDev<V> A;
  V* x;
  V* r;
  V* p;
  V* q;
  const V* b;
  double* part;               // 2 * gridDim.x partial sums
  GridBar* bar;
  CgState* st;
  const int32_t* cta_slice;   // gridDim.x + 1 slice offsets
  const int32_t* cta_long;    // gridDim.x + 1 long-row offsets
  double tol;
  int32_t maxit;
  int32_t max_restarts;
  long long timeout_ns;
};

// ------------------------------------------------------------ helpers ---
__device__ __forceinline__ long long gtime() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int32_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Matrix streams are read once per product: cache-streaming loads.
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }

// Vector gathers: read-only path in one-shot kernels (NC = true); plain
// coherent loads in the persistent solver, whose vectors change between
// grid barriers.
template <bool NC, typename T>
__device__ __forceinline__ T ld_vec(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }

// Row product of the lane's row in slice s (layout.h).  Symmetric rows sum
// in increasing column order: transpose half (columns < row), diagonal,
// upper half.
template <typename V, bool SYM, bool NC, int UNROLL = 8>
__device__ __forceinline__ V sell_row(const OpDev<V>& A, int64_t s, int lane, const V* x) {
  const int64_t row = s * 32 + lane;
  V acc = V(0);
  if constexpr (SYM) {
    const int64_t p1 = A.pl_ptr[s + 1];
#pragma unroll 4
    for (int64_t q = A.pl_ptr[s] + lane; q < p1; q += 32) {
      const uint16_t k = ld_stream(A.pl_k + q);
      if (k != kPlanPad) {
        const int32_t i = ld_stream(A.pl_i + q);
        const int64_t pos = __ldg(A.sl_ptr + (i >> 5)) + 32 * (int64_t)k + (i & 31);
        acc = fma_(__ldg(A.val + pos), ld_vec<NC>(x + i), acc);
      }
    }
    if (row < A.n) acc = fma_(ld_stream(A.diag + row), ld_vec<NC>(x + row), acc);
  }
  const int64_t b1 = A.sl_ptr[s + 1];
#pragma unroll UNROLL
  for (int64_t q = A.sl_ptr[s] + lane; q < b1; q += 32)
    acc = fma_(ld_stream(A.val + q), ld_vec<NC>(x + ld_stream(A.col + q)), acc);
  return acc;
}

// Warp-per-row product of long row li; the fixed xor tree's lane-0 value is
// the result.
template <typename V, bool NC>
__device__ __forceinline__ V long_row(const OpDev<V>& A, int64_t li, int lane, const V* x) {
  V acc = V(0);
  const int64_t e = A.long_ptr[li + 1];
  for (int64_t q = A.long_ptr[li] + lane; q < e; q += 32)
    acc = fma_(ld_stream(A.long_val + q), ld_vec<NC>(x + ld_stream(A.long_col + q)), acc);
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Visits every row of slices [s0, s1) and long rows [l0, l1) of the CTA:
// f(row, (A x)_row) runs on the lane that computed the row.
template <typename V, bool SYM, bool NC, class F>
__device__ __forceinline__ void spmv_rows(const OpDev<V>& A, int64_t s0, int64_t s1, int64_t l0, int64_t l1,
                                          const V* x, F&& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t s = s0 + warp; s < s1; s += nw) {
    const V v = sell_row<V, SYM, NC, 4>(A, s, lane, x);
    const int64_t row = s * 32 + lane;
    if (row < A.n && !((A.long_mask[s] >> lane) & 1u)) f(row, v);
  }
  for (int64_t li = l0 + warp; li < l1; li += nw) {
    const V v = long_row<V, NC>(A, li, lane, x);
    if (lane == 0) f((int64_t)A.long_row[li], v);
  }
}

// Deterministic CTA sum (fixed trees); the result is valid on thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Sum of part[0..G) in a fixed order, broadcast to every thread of the CTA.
__device__ __forceinline__ double grid_sum(const double* part, int G, double* red) {
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i < G; i += 32) t += part[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// Bounded grid barrier.  Returns false (uniformly within the CTA) when the
// wait ran out or another CTA already failed.
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned long long& target, long long timeout_ns,
                                             int* sflag, int where) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(&gb->count, 1ull);
    const long long t0 = gtime();
    unsigned spins = 0;
    for (;;) {
      if (ld_acquire(&gb->count) >= target) break;
      if (ld_relaxed(&gb->status) != 0) { ok = 0; break; }
      if ((++spins & 63u) == 0 && gtime() - t0 > timeout_ns) {
        if (atomicCAS(&gb->status, 0, (int)kTimeout) == 0) gb->where = where;
        ok = 0;
        break;
      }
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// -------------------------------------------------- one-shot kernels ---
template <typename V, bool SYM>
__global__ void __launch_bounds__(256) k_spmv(OpDev<V> A, const V* __restrict__ x, V* __restrict__ y) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w < A.nslices) {
    const V v = sell_row<V, SYM, true>(A, w, lane, x);
    const int64_t row = w * 32 + lane;
    if (row < A.n && !((A.long_mask[w] >> lane) & 1u)) y[row] = v;
  } else if (w - A.nslices < A.nlong) {
    const int64_t li = w - A.nslices;
    const V v = long_row<V, true>(A, li, lane, x);
    if (lane == 0) y[A.long_row[li]] = v;
  }
}

// r = b - A x in double precision, with per-CTA partial sums of r'r.
template <bool SYM>
__global__ void __launch_bounds__(256) k_residual(OpDev<double> A, const double* __restrict__ b,
                                                  const double* __restrict__ x, double* __restrict__ r,
                                                  double* __restrict__ part) {
  __shared__ double red[33];
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  if (w < A.nslices) {
    const double v = sell_row<double, SYM, true>(A, w, lane, x);
    const int64_t row = w * 32 + lane;
    if (row < A.n && !((A.long_mask[w] >> lane) & 1u)) {
      const double t = b[row] - v;
      r[row] = t;
      acc = t * t;
    }
  } else if (w - A.nslices < A.nlong) {
    const int64_t li = w - A.nslices;
    const double v = long_row<double, true>(A, li, lane, x);
    if (lane == 0) {
      const int64_t row = A.long_row[li];
      const double t = b[row] - v;
      r[row] = t;
      acc = t * t;
    }
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_dot_part(const double* __restrict__ a, const double* __restrict__ b,
                                                  int64_t n, double* __restrict__ part) {
  __shared__ double red[33];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[i], b[i], acc);
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[0] = sum of part[0..m) in a fixed order (one CTA of 256 threads).
__global__ void __launch_bounds__(256) k_sum_part(const double* __restrict__ part, int m, double* out) {
  __shared__ double red[33];
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) acc += part[i];
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) out[0] = s;
}

// rhs32 = float(r * scale)
__global__ void k_scale_to_f32(const double* __restrict__ r, double scale, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(r[i] * scale);
}

// x += a * double(d)
__global__ void k_axpy_f32(double a, const float* __restrict__ d, int64_t n, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, (double)d[i], x[i]);
}

// ------------------------------------------------- persistent solver ---
// OUTER = false: inner single-precision solve from x = 0 (rhs in b), no
// true-residual confirmation.  OUTER = true: the full solve of Section III
// from the caller's x0 with the confirm/restart step.
template <typename V, bool SYM, bool OUTER>
__global__ void __launch_bounds__(kCgThreads, 1) k_cg(CgArgs<V> a) {
  __shared__ double red[33];
  __shared__ int sflag;
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t s0 = a.cta_slice[c], s1 = a.cta_slice[c + 1];
  const int64_t l0 = a.cta_long[c], l1 = a.cta_long[c + 1];
  const int64_t r0 = s0 * 32;
  const int64_t r1 = s1 * 32 < a.A.n ? s1 * 32 : a.A.n;
  const OpDev<V>& A = a.A;
  V* __restrict__ x = a.x;
  V* __restrict__ r = a.r;
  V* __restrict__ p = a.p;
  V* __restrict__ q = a.q;
  const V* __restrict__ b = a.b;
  double* part0 = a.part;
  double* part1 = a.part + G;
  unsigned long long target = 0;
  int nbar = 0;
  int status = kOk;
  int k = 0, restarts = 0;
  double rr = 0.0, nb = 0.0, rel_true = 0.0;

  // init: r = b - A x0, p = r, r'r and b'b
  {
    V pr = V(0), pb = V(0);
    if constexpr (OUTER) {
      spmv_rows<V, SYM, false>(A, s0, s1, l0, l1, x, [&](int64_t row, V v) {
        const V bi = b[row];
        const V t = bi - v;
        r[row] = t;
        p[row] = t;
        pr = fma_(t, t, pr);
        pb = fma_(bi, bi, pb);
      });
    } else {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const V bi = b[i];
        x[i] = V(0);
        r[i] = bi;
        p[i] = bi;
        pr = fma_(bi, bi, pr);
      }
      for (int64_t li = l0; li < l1; ++li) (void)li;  // long rows lie inside [r0, r1)
      pb = pr;
    }
    const double s_rr = block_sum((double)pr, red);
    if (threadIdx.x == 0) part0[c] = s_rr;
    const double s_bb = block_sum((double)pb, red);
    if (threadIdx.x == 0) part1[c] = s_bb;
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    rr = grid_sum(part0, G, red);
    nb = sqrt(grid_sum(part1, G, red));
  }
  if (nb == 0.0) {  // b = 0: x = 0
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[i] = V(0);
    rr = 0.0;
    goto finish;
  }
  for (;;) {
    while (k < a.maxit && !(sqrt(rr) / nb <= a.tol)) {
      // A: q = A p, p'q
      V ppq = V(0);
      spmv_rows<V, SYM, false>(A, s0, s1, l0, l1, p, [&](int64_t row, V v) {
        q[row] = v;
        ppq = fma_(p[row], v, ppq);
      });
      {
        const double s = block_sum((double)ppq, red);
        if (threadIdx.x == 0) part0[c] = s;
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
      const double pq = grid_sum(part0, G, red);
      if (!isfinite(pq)) { status = kNonfinite; goto finish; }
      if (!(pq > 0.0)) { status = kNotSpd; goto finish; }
      const double alpha = rr / pq;
      // B: x += alpha p, r -= alpha q, r'r
      {
        const V al = (V)alpha;
        V prr = V(0);
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
          const V pi = p[i];
          x[i] = fma_(al, pi, x[i]);
          const V ri = fma_(-al, q[i], r[i]);
          r[i] = ri;
          prr = fma_(ri, ri, prr);
        }
        const double s = block_sum((double)prr, red);
        if (threadIdx.x == 0) part1[c] = s;
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
      const double rr_new = grid_sum(part1, G, red);
      ++k;
      if (!isfinite(rr_new)) { status = kNonfinite; rr = rr_new; goto finish; }
      const double beta = rr_new / rr;
      rr = rr_new;
      if (sqrt(rr) / nb <= a.tol) break;
      // C: p = r + beta p
      {
        const V be = (V)beta;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) p[i] = fma_(be, p[i], r[i]);
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    }
    if constexpr (!OUTER) {
      if (!(sqrt(rr) / nb <= a.tol)) status = kMaxit;
      break;
    } else {
      // confirm on the true residual; restart the recurrence from it otherwise
      V ptt = V(0);
      spmv_rows<V, SYM, false>(A, s0, s1, l0, l1, x, [&](int64_t row, V v) {
        const V t = b[row] - v;
        r[row] = t;
        ptt = fma_(t, t, ptt);
      });
      {
        const double s = block_sum((double)ptt, red);
        if (threadIdx.x == 0) part0[c] = s;
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
      const double tt = grid_sum(part0, G, red);
      rel_true = sqrt(tt) / nb;
      if (!isfinite(tt)) { status = kNonfinite; break; }
      if (rel_true <= a.tol) break;
      if (k >= a.maxit || restarts >= a.max_restarts) { status = kMaxit; break; }
      ++restarts;
      rr = tt;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) p[i] = r[i];
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    }
  }
finish:
  if (c == 0 && threadIdx.x == 0) {
    a.st->rr = rr;
    a.st->nb = nb;
    a.st->rel_true = rel_true;
    a.st->k = k;
    a.st->restarts = restarts;
    a.st->status = status;
  }
}

// Self-test of the bounded wait: CTA 0 never arrives.
__global__ void k_wait_selftest(GridBar* gb, long long timeout_ns) {
  __shared__ int sflag;
  if (blockIdx.x == 0) return;
  unsigned long long target = 0;
  grid_barrier(gb, target, timeout_ns, &sflag, 0);
}

}  // namespace gbcg
