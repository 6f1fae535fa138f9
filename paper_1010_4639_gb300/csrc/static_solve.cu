// static_solve.cu -- gbcg_solve_csr_static: conjugate gradient on the
// caller's device CSR arrays without any device allocation.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool's or allocator's own callback (allocating there re-enters the
// allocator and can deadlock), latency-critical loops where cudaMalloc and
// cudaFree would stall or synchronise the device, and plug-ins whose host
// application owns every byte of device memory.  For them this entry point
// keeps all its scratch -- three work vectors, per-CTA partial sums, the grid
// barrier and the solver state -- in one fixed device array defined below.
// Every GPU that loads the library holds that array until the process exits.
// All calls share it, so calls whose work overlaps on the GPU (different
// streams, or different host threads on one device) race and must not be
// issued; one call at a time per device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/gbcg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxCtas = 4096;
constexpr size_t kHeader = 256;                               // barrier + state
constexpr size_t kPartials = 2 * kMaxCtas * sizeof(double);   // two partial-sum arrays
constexpr size_t kVecAlign = 256;

// The scratch: file scope, fixed size, 256-byte aligned.  In host code this
// name is only a stand-in for the device array; its device address comes from
// cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_static_scratch[GBCG_STATIC_SCRATCH_BYTES];

__host__ __device__ constexpr size_t vec_bytes(int64_t n) { return (((size_t)n * sizeof(double)) + kVecAlign - 1) / kVecAlign * kVecAlign; }
static_assert(kHeader + kPartials + 3 * vec_bytes(GBCG_STATIC_MAX_N) <= GBCG_STATIC_SCRATCH_BYTES,
              "GBCG_STATIC_MAX_N does not fit the static scratch");

struct Bar {
  unsigned long long count;
  int status;
  int pad;
};
struct State {
  double rr, nb, rel_true;
  int k, restarts, status, pad;
};
static_assert(sizeof(Bar) + sizeof(State) <= kHeader, "header");

enum { kOk = 0, kNotSpd = 2, kMaxit = 3, kNonfinite = 4, kTimeout = 5 };

__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// CTA sum in a fixed order; valid on thread 0.
__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Sum of part[0..G) in a fixed order, on every thread.
__device__ double all_sum(const double* part, int G, double* red) {
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i < G; i += 32) t += part[i];
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// Grid barrier with a global-timer bound; false on timeout or earlier failure.
__device__ bool barrier(Bar* b, unsigned long long& target, long long limit_ns, int* flag) {
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(&b->count, 1ull);
    const long long t0 = now_ns();
    for (unsigned spins = 0;; ++spins) {
      if (*(volatile unsigned long long*)&b->count >= target) break;
      if (*(volatile int*)&b->status != 0) { ok = 0; break; }
      if ((spins & 63u) == 63u && now_ns() - t0 > limit_ns) {
        atomicCAS(&b->status, 0, (int)kTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// y_i = sum_k val[k] x[idx[k]] for the CTA's rows, one thread per row (the
// row-by-row product of Section III).
__device__ __forceinline__ double row_dot(const int32_t* ptr, const int32_t* idx, const double* val, const double* x,
                                          int64_t i) {
  double s = 0.0;
  for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) s = fma(val[k], x[idx[k]], s);
  return s;
}

// The whole solve of Section III's listing in one cooperative launch, on the
// caller's CSR arrays, with r, p, q, partial sums, barrier and state in the
// static scratch.
__global__ void __launch_bounds__(kThreads) k_cg_static(int64_t n, const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ idx,
                                                        const double* __restrict__ val, const double* __restrict__ b,
                                                        double* __restrict__ x, unsigned char* scratch, double tol,
                                                        int maxit, long long limit_ns) {
  __shared__ double red[33];
  __shared__ int flag;
  Bar* bar = reinterpret_cast<Bar*>(scratch);
  State* st = reinterpret_cast<State*>(scratch + sizeof(Bar));
  double* part0 = reinterpret_cast<double*>(scratch + kHeader);
  double* part1 = part0 + kMaxCtas;
  double* r = reinterpret_cast<double*>(scratch + kHeader + kPartials);
  double* p = reinterpret_cast<double*>(scratch + kHeader + kPartials + vec_bytes(n));
  double* q = reinterpret_cast<double*>(scratch + kHeader + kPartials + 2 * vec_bytes(n));
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t r0 = n * c / G, r1 = n * (c + 1) / G;
  unsigned long long target = 0;
  int status = kOk, k = 0, restarts = 0;
  double rr, nb, rel_true = 0.0;
  {
    double pr = 0.0, pb = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double t = b[i] - row_dot(ptr, idx, val, x, i);
      r[i] = t;
      p[i] = t;
      pr = fma(t, t, pr);
      pb = fma(b[i], b[i], pb);
    }
    const double a0 = cta_sum(pr, red);
    if (threadIdx.x == 0) part0[c] = a0;
    const double a1 = cta_sum(pb, red);
    if (threadIdx.x == 0) part1[c] = a1;
    if (!barrier(bar, target, limit_ns, &flag)) return;
    rr = all_sum(part0, G, red);
    nb = sqrt(all_sum(part1, G, red));
    // the first iteration writes part0 again: no CTA may do so while another
    // is still adding up the sums above
    if (!barrier(bar, target, limit_ns, &flag)) return;
  }
  if (nb == 0.0) {
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[i] = 0.0;
    rr = 0.0;
    goto done;
  }
  for (;;) {
    while (k < maxit && !(sqrt(rr) / nb <= tol)) {
      double ppq = 0.0;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double v = row_dot(ptr, idx, val, p, i);
        q[i] = v;
        ppq = fma(p[i], v, ppq);
      }
      const double a0 = cta_sum(ppq, red);
      if (threadIdx.x == 0) part0[c] = a0;
      if (!barrier(bar, target, limit_ns, &flag)) return;
      const double pq = all_sum(part0, G, red);
      if (!isfinite(pq)) { status = kNonfinite; goto done; }
      if (!(pq > 0.0)) { status = kNotSpd; goto done; }
      const double alpha = rr / pq;
      double prr = 0.0;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        prr = fma(ri, ri, prr);
      }
      const double a1 = cta_sum(prr, red);
      if (threadIdx.x == 0) part1[c] = a1;
      if (!barrier(bar, target, limit_ns, &flag)) return;
      const double rr_new = all_sum(part1, G, red);
      ++k;
      if (!isfinite(rr_new)) { status = kNonfinite; rr = rr_new; goto done; }
      const double beta = rr_new / rr;
      rr = rr_new;
      if (sqrt(rr) / nb <= tol) break;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) p[i] = fma(beta, p[i], r[i]);
      if (!barrier(bar, target, limit_ns, &flag)) return;
    }
    // confirm on the true residual; restart from it otherwise (at most 3 times)
    double ptt = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double t = b[i] - row_dot(ptr, idx, val, x, i);
      r[i] = t;
      ptt = fma(t, t, ptt);
    }
    const double a0 = cta_sum(ptt, red);
    if (threadIdx.x == 0) part0[c] = a0;
    if (!barrier(bar, target, limit_ns, &flag)) return;
    const double tt = all_sum(part0, G, red);
    rel_true = sqrt(tt) / nb;
    if (!isfinite(tt)) { status = kNonfinite; break; }
    if (rel_true <= tol) break;
    if (k >= maxit || restarts >= 3) { status = kMaxit; break; }
    ++restarts;
    rr = tt;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) p[i] = r[i];
    if (!barrier(bar, target, limit_ns, &flag)) return;
  }
done:
  if (c == 0 && threadIdx.x == 0) {
    st->rr = rr;
    st->nb = nb;
    st->rel_true = rel_true;
    st->k = k;
    st->restarts = restarts;
    st->status = status;
  }
}

}  // namespace

namespace gbcg {
void set_last_error(const std::string& m);  // gbcg.cu: the message gbcg_last_error() returns
}

namespace {
int fail(int code, const std::string& m) {
  gbcg::set_last_error(m);
  return code;
}
}  // namespace

extern "C" int gbcg_solve_csr_static(int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                                     const double* val, const double* b, double* x, double tol, int32_t maxit,
                                     gbcg_info* info, void* stream) {
  gbcg_info local;
  if (!info) info = &local;
  memset(info, 0, sizeof(*info));
  gbcg::set_last_error("");
  const auto t0 = std::chrono::steady_clock::now();
  if (n < 0 || nnz < 0) return fail(GBCG_ERR_INVALID, "n and nnz must be non-negative");
  if (n > GBCG_STATIC_MAX_N)
    return fail(GBCG_ERR_INVALID, "n = " + std::to_string(n) + " exceeds GBCG_STATIC_MAX_N = " +
                                      std::to_string((long long)GBCG_STATIC_MAX_N) + " of the static scratch");
  if (nnz > 0x7fffffffLL) return fail(GBCG_ERR_INVALID, "nnz exceeds 2^31 - 1");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(GBCG_ERR_INVALID, "tol must be finite and >= 0");
  if (n == 0) return GBCG_OK;
  if (!ptr || !b || !x || (nnz > 0 && (!idx || !val))) return fail(GBCG_ERR_INVALID, "null array");
  if (maxit <= 0) maxit = (int32_t)n;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(GBCG_ERR_CUDA, "cudaGetDevice failed");
  // The array's device address on the current device, looked up on every
  // call (no allocation once the library's module is loaded on the device;
  // the first call on a device loads it).  Not cached: after cudaDeviceReset
  // or a new primary context the module is loaded again and the array may
  // sit elsewhere.
  unsigned char* scratch = nullptr;
  {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(GBCG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    scratch = (unsigned char*)p;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_static, kThreads, 0) != cudaSuccess || per_sm < 1)
    return fail(GBCG_ERR_CUDA, "cannot size the cooperative grid");
  int grid = (int)std::min<int64_t>({(int64_t)per_sm * sms, (int64_t)kMaxCtas, (n + kThreads - 1) / kThreads});
  if (grid < 1) grid = 1;
  // the barrier and state words must start at zero on every call
  if (cudaMemsetAsync(scratch, 0, kHeader, s) != cudaSuccess) return fail(GBCG_ERR_CUDA, "cudaMemsetAsync failed");
  long long limit = 1000000000LL;
  void* args[] = {&n, &ptr, &idx, &val, &b, &x, &scratch, &tol, &maxit, &limit};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_cg_static, dim3(grid), dim3(kThreads), args, 0, s);
  if (e != cudaSuccess) return fail(GBCG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  unsigned char head[kHeader];
  e = cudaMemcpyAsync(head, scratch, kHeader, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(GBCG_ERR_CUDA, cudaGetErrorString(e));
  Bar hb;
  State hs;
  memcpy(&hb, head, sizeof hb);
  memcpy(&hs, head + sizeof(Bar), sizeof hs);
  int status = hb.status != 0 ? GBCG_ERR_TIMEOUT
               : hs.status == kOk ? GBCG_OK
               : hs.status == kNotSpd ? GBCG_ERR_NOT_SPD
               : hs.status == kMaxit ? GBCG_ERR_MAXIT
                                     : GBCG_ERR_NONFINITE;
  info->iterations = hs.k;
  info->outer = hs.restarts;
  info->status = status;
  info->rel_res_recursive = hs.nb > 0 ? std::sqrt(hs.rr) / hs.nb : 0.0;
  info->rel_res_true = hs.nb > 0 ? hs.rel_true : 0.0;
  info->kernel_launches = 1;
  info->launches = 1;
  info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (status != GBCG_OK) gbcg::set_last_error(std::string("gbcg_solve_csr_static: ") + gbcg_status_string(status));
  return status;
}
