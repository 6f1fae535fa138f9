// grad.cu -- the differentiable form of the solve.
//
// For a loss L(x) of the solution of A x = b, the adjoint solve
// A lambda = dL/dx (A symmetric: the same operator and the same solver)
// gives dL/db = lambda and dL/dA_ij = -lambda_i x_j.  The kernels here turn
// that into gradients of what the caller stores:
//   - k_grad_values: the sampled outer product on the stored pattern (one
//     value per stored entry; for symmetric storage an off-diagonal value
//     stands for A_ij and A_ji and gets both terms);
//   - k_element_grad: the chain rule through a finite-element assembly
//     A = sum_e coef_e Kh_e, given as stored positions and weights per element;
//   - k_assemble: that assembly, per stored position, summing its
//     contributions in a fixed order (no atomics, bitwise reproducible).
// All three are streaming kernels bound by HBM.
#include <cuda_runtime.h>

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

constexpr int kLanesPerRow = 8;

// One group of 8 lanes per row (CSR / symmetric) or column (CSC) of the
// stored pattern; entries of the row are taken 8 at a time, so a group's
// stores are contiguous.
template <int FMT>
__global__ void __launch_bounds__(256) k_grad_values(int64_t n, const int32_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ idx, int32_t base,
                                                     const double* __restrict__ lam, const double* __restrict__ x,
                                                     double* __restrict__ g) {
  const int sub = threadIdx.x % kLanesPerRow;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kLanesPerRow);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / kLanesPerRow) + threadIdx.x / kLanesPerRow; r < n;
       r += groups) {
    const double lr = lam[r], xr = x[r];
    const int64_t k1 = (int64_t)ptr[r + 1] - base;
    for (int64_t k = (int64_t)ptr[r] - base + sub; k < k1; k += kLanesPerRow) {
      const int64_t c = (int64_t)idx[k] - base;
      double v;
      if (FMT == GBCG_CSC)
        v = -(lam[c] * xr);  // column r, row c
      else if (FMT == GBCG_SYM_CSR_UPPER && c != r)
        v = -(lr * x[c] + lam[c] * xr);
      else
        v = -(lr * x[c]);
      g[k] = v;
    }
  }
}

__global__ void __launch_bounds__(256) k_element_grad(int64_t ne, int m, const int32_t* __restrict__ pos,
                                                      const double* __restrict__ w, const double* __restrict__ g,
                                                      double* __restrict__ gc) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) {
      const int32_t p = pos[e * m + k];
      if (p >= 0) s = fma(w[e * m + k], g[p], s);
    }
    gc[e] = s;
  }
}

__global__ void __launch_bounds__(256) k_assemble(int64_t nnz, const int64_t* __restrict__ tptr,
                                                  const int32_t* __restrict__ telem, const double* __restrict__ tw,
                                                  const double* __restrict__ coef, double* __restrict__ val) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t k = tptr[p]; k < tptr[p + 1]; ++k) s = fma(tw[k], coef[telem[k]], s);
    val[p] = s;
  }
}

int grid_for(int64_t items, int per_block) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)sms * 8;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

int launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GBCG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return GBCG_OK;
}

}  // namespace

extern "C" {

int gbcg_grad_values(int32_t format, int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                     int32_t index_base, const double* lambda, const double* x, double* grad, void* stream) {
  gbcg::set_last_error("");
  if (format != GBCG_CSR && format != GBCG_SYM_CSR_UPPER && format != GBCG_CSC)
    return fail(GBCG_ERR_INVALID, "unknown format");
  if (n < 0 || nnz < 0) return fail(GBCG_ERR_INVALID, "n and nnz must be non-negative");
  if (index_base != 0 && index_base != 1) return fail(GBCG_ERR_INVALID, "index_base must be 0 or 1");
  if (n == 0) return GBCG_OK;
  if (!ptr || !lambda || !x || (nnz > 0 && (!idx || !grad))) return fail(GBCG_ERR_INVALID, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = grid_for(n, 256 / kLanesPerRow);
  if (format == GBCG_CSR)
    k_grad_values<GBCG_CSR><<<blocks, 256, 0, s>>>(n, ptr, idx, index_base, lambda, x, grad);
  else if (format == GBCG_CSC)
    k_grad_values<GBCG_CSC><<<blocks, 256, 0, s>>>(n, ptr, idx, index_base, lambda, x, grad);
  else
    k_grad_values<GBCG_SYM_CSR_UPPER><<<blocks, 256, 0, s>>>(n, ptr, idx, index_base, lambda, x, grad);
  return launched("k_grad_values");
}

int gbcg_element_grad(int64_t ne, int32_t m, const int32_t* pos, const double* w, const double* grad,
                      double* grad_coef, void* stream) {
  gbcg::set_last_error("");
  if (ne < 0 || m < 0 || m > 64) return fail(GBCG_ERR_INVALID, "ne must be >= 0 and m in [0, 64]");
  if (ne == 0) return GBCG_OK;
  if (!grad_coef || (m > 0 && (!pos || !w || !grad))) return fail(GBCG_ERR_INVALID, "null argument");
  k_element_grad<<<grid_for(ne, 256), 256, 0, (cudaStream_t)stream>>>(ne, m, pos, w, grad, grad_coef);
  return launched("k_element_grad");
}

int gbcg_assemble(int64_t nnz, const int64_t* tptr, const int32_t* telem, const double* tw, const double* coef,
                  double* val, void* stream) {
  gbcg::set_last_error("");
  if (nnz < 0) return fail(GBCG_ERR_INVALID, "nnz must be >= 0");
  if (nnz == 0) return GBCG_OK;
  if (!tptr || !val || !telem || !tw || !coef) return fail(GBCG_ERR_INVALID, "null argument");
  k_assemble<<<grid_for(nnz, 256), 256, 0, (cudaStream_t)stream>>>(nnz, tptr, telem, tw, coef, val);
  return launched("k_assemble");
}

}  // extern "C"
