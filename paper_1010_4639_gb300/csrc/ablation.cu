// ablation.cu -- the 2010 structure of the paper's GPU solver, rebuilt as
// measurement baselines.  The solver never calls these.
//
// Section III runs CG with the SpMV as a custom kernel and the scalar
// products and axpy updates as CuBLAS calls, each a separate launch; every
// scalar product returns its value to the host, which forms alpha and beta
// and decides convergence.  Its SpMV kernels are
//   - the "trivial" CSR kernel: one thread per row, reading the CSR arrays
//     directly;
//   - the symmetric pair SCSR + SCSC, two launches one after the other (one
//     kernel at a time per device on the paper's GPUs): SCSR reads the
//     stored triangle by rows and writes the direct half, one thread per
//     row; SCSC reads the same arrays as columns and scatters the transpose
//     half with floating-point atomic additions (so the result's last bits
//     depend on the scheduling).
// Here the same structure runs on GB300 with the library's own simple
// kernels standing in for CuBLAS.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/gbcg.h"

namespace gbcg {
void set_last_error(const std::string& m);
}

namespace {

int fail(int code, const std::string& msg) {
  gbcg::set_last_error(msg);
  return code;
}

#define ACUDA(...)                                                                                   \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? GBCG_ERR_NOMEM : GBCG_ERR_CUDA,                  \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

constexpr int kThreads = 256;

int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 1 << 20)); }

// y_i = sum_k val[k] x[idx[k]] over row i: one thread per row.
__global__ void k_spmv_trivial(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                               const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) s = fma(val[k], x[idx[k]], s);
  y[i] = s;
}

// Symmetric storage (upper triangle and diagonal by rows), first launch
// (SCSR): y_i = sum over row i's stored entries (D + U) of a_ij x_j.
__global__ void k_spmv_scsr(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                            const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) s = fma(val[k], x[idx[k]], s);
  y[i] = s;
}

// Second launch (SCSC): the same arrays read as columns of L = U'; column i
// scatters a_ij x_i into y_j for its entries j > i, with atomic additions.
__global__ void k_spmv_scsc(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                            const double* __restrict__ val, const double* __restrict__ x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = x[i];
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
    const int32_t j = idx[k];
    if (j != i) atomicAdd(&y[j], val[k] * xi);
  }
}

// Scalar product in two launches, the result copied to the host.
__global__ void k_dot_blocks(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* part) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(~0u, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(~0u, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void k_sum_blocks(int m, const double* __restrict__ part, double* out) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(~0u, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(~0u, s, o);
    if (threadIdx.x == 0) out[0] = s;
  }
}

// y += a x
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}

// y = x + a y
__global__ void k_xpay(int64_t n, const double* __restrict__ x, double a, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, y[i], x[i]);
}

__global__ void k_sub(int64_t n, const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = b[i] - ax[i];
}

int spmv(int32_t format, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val, const double* x,
         double* y, cudaStream_t s, int& launches) {
  if (format == GBCG_SYM_CSR_UPPER) {
    k_spmv_scsr<<<blocks_for(n), kThreads, 0, s>>>(n, ptr, idx, val, x, y);
    k_spmv_scsc<<<blocks_for(n), kThreads, 0, s>>>(n, ptr, idx, val, x, y);
    launches += 2;
  } else {
    k_spmv_trivial<<<blocks_for(n), kThreads, 0, s>>>(n, ptr, idx, val, x, y);
    ++launches;
  }
  ACUDA(cudaGetLastError());
  return 0;
}

struct Work {
  double *r = nullptr, *p = nullptr, *q = nullptr, *part = nullptr, *out = nullptr, *host = nullptr;
  ~Work() {
    cudaFree(r);
    cudaFree(p);
    cudaFree(q);
    cudaFree(part);
    cudaFree(out);
    cudaFreeHost(host);
  }
};

int dot(int64_t n, const double* a, const double* b, Work& w, cudaStream_t s, int& launches, double& v) {
  const int m = std::min(blocks_for(n), 1024);
  k_dot_blocks<<<m, kThreads, 0, s>>>(n, a, b, w.part);
  k_sum_blocks<<<1, kThreads, 0, s>>>(m, w.part, w.out);
  ACUDA(cudaGetLastError());
  launches += 2;
  ACUDA(cudaMemcpyAsync(w.host, w.out, sizeof(double), cudaMemcpyDeviceToHost, s));
  ACUDA(cudaStreamSynchronize(s));
  v = *w.host;
  return 0;
}

// FP64 FMA throughput probe: every thread runs kFmaChains independent FMA
// chains of kFmaSteps steps (enough independent work to fill the FP64 pipe
// at full occupancy); the sum is tested against a value it never takes, so
// the chains stay live without a store per thread.
constexpr int kFmaChains = 8, kFmaSteps = 4096;
__global__ void __launch_bounds__(kThreads) k_fp64_fma(double seed, double* out) {
  double a[kFmaChains];
  const double m = 1.0 - 1e-13 * (double)(threadIdx.x & 7), c = 1e-9 * (double)(blockIdx.x & 15);
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = seed + k;
  for (int i = 0; i < kFmaSteps; ++i)
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], m, c);
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) t += a[k];
  if (t == -1.0) out[0] = t;
}

int check_format(int32_t format) {
  if (format != GBCG_CSR && format != GBCG_SYM_CSR_UPPER)
    return fail(GBCG_ERR_INVALID, "ablation kernels take GBCG_CSR or GBCG_SYM_CSR_UPPER");
  return 0;
}

}  // namespace

extern "C" {

int gbcg_ablation_spmv(int32_t format, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val,
                       const double* x, double* y, void* stream) {
  gbcg::set_last_error("");
  if (int rc = check_format(format)) return rc;
  if (n < 0) return fail(GBCG_ERR_INVALID, "n must be >= 0");
  if (n == 0) return GBCG_OK;
  if (!ptr || !idx || !val || !x || !y) return fail(GBCG_ERR_INVALID, "null argument");
  int launches = 0;
  return spmv(format, n, ptr, idx, val, x, y, (cudaStream_t)stream, launches);
}

int gbcg_ablation_solve(int32_t format, int64_t n, const int32_t* ptr, const int32_t* idx, const double* val,
                        const double* b, double* x, double tol, int32_t maxit, gbcg_info* info, void* stream) {
  gbcg::set_last_error("");
  gbcg_info local;
  if (!info) info = &local;
  memset(info, 0, sizeof(*info));
  if (int rc = check_format(format)) return rc;
  if (n < 0 || !(tol >= 0.0)) return fail(GBCG_ERR_INVALID, "bad n or tol");
  if (n == 0) return GBCG_OK;
  if (!ptr || !idx || !val || !b || !x) return fail(GBCG_ERR_INVALID, "null argument");
  if (maxit <= 0) maxit = (int32_t)std::min<int64_t>(n, 0x7fffffff);
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  ACUDA(cudaMalloc(&w.r, sizeof(double) * n));
  ACUDA(cudaMalloc(&w.p, sizeof(double) * n));
  ACUDA(cudaMalloc(&w.q, sizeof(double) * n));
  ACUDA(cudaMalloc(&w.part, sizeof(double) * 1024));
  ACUDA(cudaMalloc(&w.out, sizeof(double)));
  ACUDA(cudaMallocHost(&w.host, sizeof(double)));
  int launches = 0, k = 0, status = GBCG_ERR_MAXIT, rc = 0;
  const int nb_ = blocks_for(n);
  double bb = 0.0, rr = 0.0;
  if ((rc = dot(n, b, b, w, s, launches, bb))) return rc;
  const double nb = std::sqrt(bb);
  if (nb == 0.0) {
    ACUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    ACUDA(cudaStreamSynchronize(s));
    info->status = GBCG_OK;
    return GBCG_OK;
  }
  // r = b - A x, p = r
  if ((rc = spmv(format, n, ptr, idx, val, x, w.q, s, launches))) return rc;
  k_sub<<<nb_, kThreads, 0, s>>>(n, b, w.q, w.r);
  ACUDA(cudaMemcpyAsync(w.p, w.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launches += 1;
  if ((rc = dot(n, w.r, w.r, w, s, launches, rr))) return rc;
  while (true) {
    if (std::sqrt(rr) / nb <= tol) {
      status = GBCG_OK;
      break;
    }
    if (k >= maxit) break;
    if ((rc = spmv(format, n, ptr, idx, val, w.p, w.q, s, launches))) return rc;   // q = A p
    double pq = 0.0;
    if ((rc = dot(n, w.p, w.q, w, s, launches, pq))) return rc;                      // p'q to the host
    if (!std::isfinite(pq)) {
      status = GBCG_ERR_NONFINITE;
      break;
    }
    if (!(pq > 0.0)) {
      status = GBCG_ERR_NOT_SPD;
      break;
    }
    const double alpha = rr / pq;
    k_axpy<<<nb_, kThreads, 0, s>>>(n, alpha, w.p, x);      // x += alpha p
    k_axpy<<<nb_, kThreads, 0, s>>>(n, -alpha, w.q, w.r);   // r -= alpha q
    launches += 2;
    double rr_new = 0.0;
    if ((rc = dot(n, w.r, w.r, w, s, launches, rr_new))) return rc;                  // r'r to the host
    ++k;
    const double beta = rr_new / rr;
    rr = rr_new;
    if (std::sqrt(rr) / nb <= tol) {
      status = GBCG_OK;
      break;
    }
    k_xpay<<<nb_, kThreads, 0, s>>>(n, w.r, beta, w.p);     // p = r + beta p
    launches += 1;
    ACUDA(cudaGetLastError());
  }
  // the true residual, for the report
  if ((rc = spmv(format, n, ptr, idx, val, x, w.q, s, launches))) return rc;
  k_sub<<<nb_, kThreads, 0, s>>>(n, b, w.q, w.r);
  launches += 1;
  double tt = 0.0;
  if ((rc = dot(n, w.r, w.r, w, s, launches, tt))) return rc;
  info->iterations = k;
  info->status = status;
  info->rel_res_recursive = std::sqrt(rr) / nb;
  info->rel_res_true = std::sqrt(tt) / nb;
  info->launches = launches;
  info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

int gbcg_measure_fp64_fma_rate(double* fma_per_s, void* stream) {
  if (!fma_per_s) return fail(GBCG_ERR_INVALID, "null output");
  *fma_per_s = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  ACUDA(cudaGetDevice(&dev));
  ACUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * (2048 / kThreads);  // full occupancy on every SM
  double* out = nullptr;
  ACUDA(cudaMalloc(&out, sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      k_fp64_fma<<<blocks, kThreads, 0, s>>>(1.0 + rep, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  ACUDA(e);
  const double fmas = (double)blocks * kThreads * kFmaSteps * kFmaChains;
  *fma_per_s = best > 0.f ? fmas / (best * 1e-3) : 0.0;
  return GBCG_OK;
}

}  // extern "C"
