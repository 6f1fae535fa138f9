// batch.cu -- many independent SPD systems of uneven size, each with up to
// eight right-hand sides, solved by one persistent launch under a CUDA graph.
//
// The method per system and right-hand side is the conjugate-gradient
// iteration of Section III, in the single-precision form of Section IV inside
// double-precision iterative refinement (or in double precision throughout).
// The batch layout is a block-diagonal CSR: instance i owns rows
// [row_off[i], row_off[i+1]) and only columns in that range.  Right-hand
// sides are interleaved per row (eight values of one row are contiguous), so
// each stored entry gathers one 32-byte (float) or 64-byte (double) group and
// the matrix is read once for all of them.
//
// Execution: a persistent kernel of thread-block clusters.  Each cluster
// takes the next instance from a work queue (instances ordered longest
// first), splits its rows over the cluster's CTAs and runs the whole solve of
// that instance with cluster barriers; per-right-hand-side sums go through
// distributed shared memory in a fixed order, so an instance's result does
// not depend on which cluster solved it or when.  No CTA ever waits on a CTA
// outside its cluster, and the hardware co-schedules a cluster, so there is
// no software spin-wait anywhere in this launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/gbcg.h"

namespace gbcg {
void set_last_error(const std::string& m);
}

namespace {

constexpr int kRhs = 8;          // right-hand sides held per row
constexpr int kBuckets = 8;      // nnz-per-row buckets [2^b, 2^(b+1))
constexpr int kMaxWarps = 16;
constexpr int kMaxGroup = 8;     // clusters one instance may span

enum { kOk = 0, kNotSpd = 2, kMaxit = 3, kNonfinite = 4, kTimeout = 5 };

int fail(int code, const std::string& msg) {
  gbcg::set_last_error(msg);
  return code;
}

#define BCUDA(...)                                                                                   \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess)                                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? GBCG_ERR_NOMEM : GBCG_ERR_CUDA,                  \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

// ------------------------------------------------------------ device side
template <typename V>
struct V16;
template <>
struct V16<float> {
  using T = float4;
  static constexpr int W = 4;
};
template <>
struct V16<double> {
  using T = double2;
  static constexpr int W = 2;
};

// Everything a launch reads, kept in device memory so that a captured graph
// serves every solve (the host rewrites this block before each launch).
struct BArgs {
  const int64_t* inst_row;  // count + 1 row offsets
  const int32_t* ptr;       // n_tot + 1
  const int32_t* idx;       // global column of every entry
  const double* val64;
  const float* val32;
  const int32_t* slot_inst; // queue slot -> instance
  const int32_t* slot_part; // queue slot -> part of a multi-cluster group (0 .. G-1)
  const int8_t* grp;        // clusters per instance (G)
  const int8_t* rpw;        // rows per warp of the inner product, per instance
  unsigned* gbar;           // per instance: group barrier arrivals
  double* gpart;            // per instance: [2][kMaxGroup][16] cluster partial sums
  int* err;                 // launch-wide failure (a group wait ran out)
  const double* B;          // n_tot x nrhs, caller layout
  double* X;                // n_tot x nrhs, caller layout
  double* R64;              // n_tot x 8: outer residual
  void* R;                  // n_tot x 8 inner vectors (float or double)
  void* P;
  void* Q;
  void* D;
  int* queue;
  gbcg_batch_info* out;     // count x nrhs
  int32_t* inst_iters;      // count: products with the inner matrix
  int32_t* inst_outer;      // count: double-precision residual products
  long long* t_inst;        // 2 x count: start and end, global timer ns
  double tol, inner_tol;     // inner_tol: refinement tolerance, or the reliable-update factor
  long long timeout_ns;
  int count, nslots, nrhs, maxit, max_outer, force_rpw;
  int reliable;              // 1: single-precision iterations with double-precision reliable updates
};

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_ctas() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// All threads of all CTAs of the cluster; release/acquire at cluster scope
// orders the global and shared memory accesses on either side.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned dsmem_addr(const void* local, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ double ld_dsmem_f64(const double* local, unsigned rank) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(dsmem_addr(local, rank)) : "memory");
  return v;
}
__device__ __forceinline__ int ld_dsmem_s32(const int* local, unsigned rank) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(dsmem_addr(local, rank)) : "memory");
  return v;
}

struct Red {
  double warp[kMaxWarps][2 * kRhs];
  double cta[2][2 * kRhs];
  double sum[2 * kRhs];
};

// Per-instance scalars of the eight right-hand sides; lane k of warp 0 owns
// right-hand side k, every other thread only reads.
struct St {
  double rr[kRhs], nr0[kRhs], nb[kRhs], nr[kRhs], alpha[kRhs], beta[kRhs], rel[kRhs], itol[kRhs], rmax[kRhs];
  int used[kRhs], outer[kRhs], status[kRhs], kin[kRhs], bd[kRhs];
  unsigned fin, oact, iact, zero;
  int maxit, products, outers;
};

// Cluster-wide sums of NS x 8 values.  v[s][j] is this thread's partial of
// sum (s, c*VW + j), c = lane % (8/VW) the thread's group of right-hand
// sides.  Fixed order everywhere: lanes by xor tree, warps in index order,
// CTAs in rank order.  The result for sum t = s*8 + k is returned on thread
// t (t < NS*8); every CTA of the cluster computes identical values.
template <int VW, int NS>
__device__ __forceinline__ double cluster_reduce(double (&v)[NS][VW], Red& red, int& par, unsigned C) {
  constexpr int CH = kRhs / VW;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      double t = v[s][j];
#pragma unroll
      for (int o = CH; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[s][j] = t;
    }
  if (lane < CH) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int j = 0; j < VW; ++j) red.warp[w][s * kRhs + lane * VW + j] = v[s][j];
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (threadIdx.x < NS * kRhs) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red.warp[i][threadIdx.x];
    red.cta[par][threadIdx.x] = t;
  }
  cluster_sync();
  double s = 0.0;
  if (threadIdx.x < NS * kRhs)
    for (unsigned c = 0; c < C; ++c) s += ld_dsmem_f64(&red.cta[par][threadIdx.x], c);
  par ^= 1;
  return s;
}

template <typename VT, typename V>
__device__ __forceinline__ VT vfma(V a, VT x, VT y);
template <>
__device__ __forceinline__ float4 vfma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
template <>
__device__ __forceinline__ double2 vfma(double a, double2 x, double2 y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float4 vshfl_xor(float4 v, int o) {
  return make_float4(__shfl_xor_sync(~0u, v.x, o), __shfl_xor_sync(~0u, v.y, o), __shfl_xor_sync(~0u, v.z, o),
                     __shfl_xor_sync(~0u, v.w, o));
}
__device__ __forceinline__ double2 vshfl_xor(double2 v, int o) {
  return make_double2(__shfl_xor_sync(~0u, v.x, o), __shfl_xor_sync(~0u, v.y, o));
}
__device__ __forceinline__ float4 vadd(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Q = A P over rows [r0, r1) for all eight right-hand sides, LPR lanes per
// row: lane (row, s, c) sums entries s, s+S, ... of the row for the
// right-hand-side group c (S = LPR / CH slices), then the slices are added by
// an xor tree.  emit(row, c, sum) runs on the slice-0 lane of every group.
template <typename V, int LPR, class Emit>
__device__ __forceinline__ void product(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const V* __restrict__ val, const V* __restrict__ x, int64_t r0, int64_t r1,
                                        Emit&& emit) {
  using VT = typename V16<V>::T;
  constexpr int VW = V16<V>::W, CH = kRhs / VW, S = LPR / CH, RPW = 32 / LPR;
  static_assert(S >= 1, "at least one slice per group");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane % LPR, c = sub % CH, sl = sub / CH;
  for (int64_t base = r0 + (int64_t)warp * RPW; base < r1; base += (int64_t)nw * RPW) {
    const int64_t row = base + lane / LPR;
    VT acc{};
    if (row < r1) {
      const int k1 = ptr[row + 1];
#pragma unroll 4
      for (int k = ptr[row] + sl; k < k1; k += S) {
        const VT xv = *reinterpret_cast<const VT*>(x + (int64_t)idx[k] * kRhs + c * VW);
        acc = vfma(val[k], xv, acc);
      }
    }
#pragma unroll
    for (int o = CH; o < LPR; o <<= 1) acc = vadd(acc, vshfl_xor(acc, o));
    if (row < r1 && sl == 0) emit(row, c, acc);
  }
}

template <typename V, class Emit>
__device__ __forceinline__ void product_rpw(int rpw, const int32_t* ptr, const int32_t* idx, const V* val,
                                            const V* x, int64_t r0, int64_t r1, Emit&& emit) {
  switch (rpw) {
    case 1: product<V, 32>(ptr, idx, val, x, r0, r1, emit); break;
    case 2: product<V, 16>(ptr, idx, val, x, r0, r1, emit); break;
    case 4: product<V, 8>(ptr, idx, val, x, r0, r1, emit); break;
    default:
      if constexpr (sizeof(V) == 4) {
        if (rpw == 16) {
          product<V, 2>(ptr, idx, val, x, r0, r1, emit);
          break;
        }
      }
      product<V, 4>(ptr, idx, val, x, r0, r1, emit);
  }
}

// Outer residual R64 = B - A64 X (caller layout of B and X, nrhs columns),
// eight lanes per row in pairs of right-hand sides; partial sums of r'r and
// b'b per right-hand side.
__device__ __forceinline__ void outer_residual(const BArgs& a, int64_t r0, int64_t r1, double (&v)[2][2]) {
  constexpr int LPR = 8, CH = 4, S = 2, RPW = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane % LPR, c = sub % CH, sl = sub / CH;
  const int nrhs = a.nrhs;
  const int k0 = 2 * c, k1 = 2 * c + 1;
  for (int64_t base = r0 + (int64_t)warp * RPW; base < r1; base += (int64_t)nw * RPW) {
    const int64_t row = base + lane / LPR;
    double s0 = 0.0, s1 = 0.0;
    if (row < r1) {
      const int e1 = a.ptr[row + 1];
      for (int k = a.ptr[row] + sl; k < e1; k += S) {
        const double av = a.val64[k];
        const int64_t j = (int64_t)a.idx[k] * nrhs;
        if (k0 < nrhs) s0 = fma(av, a.X[j + k0], s0);
        if (k1 < nrhs) s1 = fma(av, a.X[j + k1], s1);
      }
    }
    s0 += __shfl_xor_sync(~0u, s0, CH);
    s1 += __shfl_xor_sync(~0u, s1, CH);
    if (row < r1 && sl == 0) {
      const double b0 = k0 < nrhs ? a.B[row * nrhs + k0] : 0.0;
      const double b1 = k1 < nrhs ? a.B[row * nrhs + k1] : 0.0;
      const double t0 = b0 - s0, t1 = b1 - s1;
      a.R64[row * kRhs + k0] = t0;
      a.R64[row * kRhs + k1] = t1;
      v[0][0] = fma(t0, t0, v[0][0]);
      v[0][1] = fma(t1, t1, v[0][1]);
      v[1][0] = fma(b0, b0, v[1][0]);
      v[1][1] = fma(b1, b1, v[1][1]);
    }
  }
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The clusters working on one instance: G clusters of C CTAs, this cluster
// being part p.  With G = 1 every synchronisation is a cluster barrier;
// with G > 1 cluster rank 0 of each part meets the others on a global
// counter (bounded wait).
struct Group {
  int G, p;
  unsigned C, cr;
  unsigned* bar;
  double* part;     // [2][kMaxGroup][16]
  unsigned target;  // arrivals awaited by the next wait (cluster rank 0, thread 0 only)
  int gpar;         // slot of the next group sum; changed by thread 0 between barriers
};

// Barrier of the whole group; false (uniformly within the cluster) when the
// wait ran out or another group failed.  Writes before it, by any CTA of the
// group, are visible after it.
__device__ __forceinline__ bool group_sync(const BArgs& a, Group& g, int* s_flag) {
  cluster_sync();
  if (g.G == 1) return true;
  if (g.cr == 0 && threadIdx.x == 0) {
    g.target += (unsigned)g.G;
    int ok = 1;
    __threadfence();
    atomicAdd(g.bar, 1u);
    const long long t0 = now_ns();
    for (unsigned spins = 0;; ++spins) {
      if (ld_acquire_u32(g.bar) >= g.target) break;
      if (ld_relaxed_s32(a.err) != 0) {
        ok = 0;
        break;
      }
      if ((spins & 63u) == 63u && now_ns() - t0 > a.timeout_ns) {
        atomicCAS(a.err, 0, (int)kTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  cluster_sync();
  const int ok = ld_dsmem_s32(s_flag, 0);
  if (!ok) {
    cluster_sync();  // no CTA leaves while another still reads its shared memory
    return false;
  }
  if (threadIdx.x == 0) __threadfence();  // acquire for this SM before reading the other clusters' data
  __syncthreads();
  return true;
}

// Sums over the whole group (see cluster_reduce): the cluster's sums, then
// for G > 1 the parts' sums in part order, read from global memory.
template <int VW, int NS>
__device__ __forceinline__ double group_reduce(const BArgs& a, double (&v)[NS][VW], Red& red, int& par, Group& g,
                                               int* s_flag, bool& ok) {
  double s = cluster_reduce<VW, NS>(v, red, par, g.C);
  if (g.G == 1) return s;
  double* slot = g.part + g.gpar * (kMaxGroup * 2 * kRhs);
  if (g.cr == 0 && threadIdx.x < NS * kRhs) slot[g.p * 2 * kRhs + threadIdx.x] = s;
  ok = group_sync(a, g, s_flag);  // every thread has read g.gpar before it returns
  if (threadIdx.x == 0) g.gpar ^= 1;  // read again only after the caller's next __syncthreads
  s = 0.0;
  if (threadIdx.x < NS * kRhs)
    for (int q = 0; q < g.G; ++q) s += __ldcg(slot + q * 2 * kRhs + threadIdx.x);
  return s;
}

// One instance, all right-hand sides, on this cluster's share of its rows.
// Returns false when a group wait failed (the instance is abandoned).
template <typename V, int NT>
__device__ bool solve_instance(const BArgs& a, int inst, Group& g, Red& red, St& st, int& par, int* s_flag) {
  using VT = typename V16<V>::T;
  constexpr int VW = V16<V>::W, CH = kRhs / VW;
  const int t = threadIdx.x;
  const int ch = t % CH;  // this thread's group of right-hand sides in the vector passes
  V* __restrict__ R = reinterpret_cast<V*>(a.R);
  V* __restrict__ P = reinterpret_cast<V*>(a.P);
  V* __restrict__ Q = reinterpret_cast<V*>(a.Q);
  V* __restrict__ D = reinterpret_cast<V*>(a.D);
  const V* __restrict__ AV = sizeof(V) == 4 ? reinterpret_cast<const V*>(a.val32) : reinterpret_cast<const V*>(a.val64);
  const int64_t row0 = a.inst_row[inst];
  const int64_t nI = a.inst_row[inst + 1] - row0;
  const int64_t GC = (int64_t)g.G * g.C, gc = (int64_t)g.p * g.C + g.cr;
  const int64_t per = (nI + GC - 1) / GC;
  const int64_t r0 = row0 + min64(nI, per * gc);
  const int64_t r1 = row0 + min64(nI, per * (gc + 1));
  const int rp = a.force_rpw > 0 ? a.force_rpw : (int)a.rpw[inst];
  const int64_t e0 = r0 * CH, e1 = r1 * CH;  // 16-byte groups of the CTA's rows
  bool ok = true;
  if (t < 32) {
    if (t < kRhs) {
      st.used[t] = 0;
      st.outer[t] = 0;
      st.status[t] = kMaxit;
      st.rel[t] = 0.0;
      st.nb[t] = 0.0;
    }
    const unsigned pad = __ballot_sync(~0u, t < kRhs && t >= a.nrhs);
    if (t == 0) {
      st.fin = pad;
      st.zero = 0;
      st.maxit = a.maxit > 0 ? a.maxit : (int)min64(nI, 0x7fffffff);
      st.products = 0;
      st.outers = 0;
    }
  }
  __syncthreads();
  for (bool first = true;; first = false) {
    // outer step: R64 = B - A64 X and the norms, in double precision
    {
      double v[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      outer_residual(a, r0, r1, v);
      const double s = group_reduce<2, 2>(a, v, red, par, g, s_flag, ok);
      if (!ok) return false;
      if (t >= kRhs && t < 2 * kRhs) red.sum[t] = s;
      __syncthreads();
      if (t < 32) {
        bool act = false, zero = false, done = false;
        if (t < kRhs && !((st.fin >> t) & 1u)) {
          if (first) st.nb[t] = sqrt(red.sum[kRhs + t]);
          const double nb = st.nb[t];
          if (nb == 0.0) {
            zero = true;
            done = true;
            st.status[t] = kOk;
            st.rel[t] = 0.0;
          } else {
            const double nr = sqrt(s);
            const double rel = nr / nb;
            st.rel[t] = rel;
            if (!isfinite(rel)) {
              st.status[t] = kNonfinite;
              done = true;
            } else if (rel <= a.tol) {
              st.status[t] = kOk;
              done = true;
            } else if (st.outer[t] >= a.max_outer || st.used[t] >= st.maxit) {
              st.status[t] = kMaxit;
              done = true;
            } else {
              act = true;
              st.nr[t] = nr;
              // inner target relative to the pass's own starting residual:
              // fixed for the refinement; for double precision the one that
              // brings ||b - A x|| to tol ||b||, so that later passes are the
              // true-residual restarts of the Section III solve
              st.itol[t] = sizeof(V) == 4 ? a.inner_tol : a.tol * nb / nr;
            }
          }
        }
        const unsigned am = __ballot_sync(~0u, act), zm = __ballot_sync(~0u, zero), dm = __ballot_sync(~0u, done);
        if (t == 0) {
          st.oact = am;
          st.zero = zm;
          st.fin |= dm;
          st.outers += 1;
        }
      }
      __syncthreads();
    }
    if (st.zero) {  // b = 0: x = 0
      const unsigned zm = st.zero;
      for (int64_t row = r0 + t; row < r1; row += NT)
        for (int k = 0; k < a.nrhs; ++k)
          if ((zm >> k) & 1u) a.X[row * a.nrhs + k] = 0.0;
    }
    const unsigned oact = st.oact;
    if (oact == 0) break;
    // inner setup: R = P = r / ||r|| in V, D = 0, r'r
    {
      V pr[VW];
      double nrv[VW];
      bool on[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) {
        pr[j] = V(0);
        on[j] = (oact >> (ch * VW + j)) & 1u;
        nrv[j] = on[j] ? st.nr[ch * VW + j] : 1.0;
      }
      for (int64_t e = e0 + t; e < e1; e += NT) {
        VT rv;
        V* re = reinterpret_cast<V*>(&rv);
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          re[j] = on[j] ? (V)(a.R64[e * VW + j] / nrv[j]) : V(0);
          pr[j] = re[j] * re[j] + pr[j];
        }
        reinterpret_cast<VT*>(R)[e] = rv;
        reinterpret_cast<VT*>(P)[e] = rv;
        reinterpret_cast<VT*>(D)[e] = VT{};
      }
      double v[1][VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) v[0][j] = (double)pr[j];
      const double s = group_reduce<VW, 1>(a, v, red, par, g, s_flag, ok);  // also publishes P
      if (!ok) return false;
      if (t < 32) {
        bool go = false;
        if (t < kRhs && ((oact >> t) & 1u)) {
          st.rr[t] = s;
          st.nr0[t] = sqrt(s);
          st.kin[t] = 0;
          st.bd[t] = 0;
          go = st.nr0[t] > 0.0 && !(sqrt(s) <= st.itol[t] * st.nr0[t]) && st.used[t] < st.maxit;
        }
        const unsigned m = __ballot_sync(~0u, go);
        if (t == 0) st.iact = m;
      }
      __syncthreads();
    }
    // inner CG, one right-hand side per bit of st.iact
    while (st.iact) {
      // q = A p, p'q
      {
        double v[1][VW];
        V pq[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) pq[j] = V(0);
        product_rpw<V>(rp, a.ptr, a.idx, AV, P, r0, r1, [&](int64_t row, int c, VT acc) {
          const int64_t e = row * CH + c;
          reinterpret_cast<VT*>(Q)[e] = acc;
          const VT pv = reinterpret_cast<const VT*>(P)[e];
          const V* pe = reinterpret_cast<const V*>(&pv);
          const V* qe = reinterpret_cast<const V*>(&acc);
#pragma unroll
          for (int j = 0; j < VW; ++j) pq[j] = pe[j] * qe[j] + pq[j];
        });
#pragma unroll
        for (int j = 0; j < VW; ++j) v[0][j] = (double)pq[j];
        const double s = group_reduce<VW, 1>(a, v, red, par, g, s_flag, ok);
        if (!ok) return false;
        if (t < kRhs) {
          double al = 0.0;
          if ((st.iact >> t) & 1u) {
            if (!isfinite(s) || !(s > 0.0))
              st.bd[t] = 1;
            else
              al = st.rr[t] / s;
          }
          st.alpha[t] = al;
        }
        __syncthreads();
      }
      // x_inner += alpha p, r -= alpha q, r'r   (alpha = 0 leaves a stopped column unchanged)
      {
        V al[VW], pr[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          al[j] = (V)st.alpha[ch * VW + j];
          pr[j] = V(0);
        }
        for (int64_t e = e0 + t; e < e1; e += NT) {
          const VT pv = reinterpret_cast<const VT*>(P)[e];
          const VT qv = reinterpret_cast<const VT*>(Q)[e];
          VT dv = reinterpret_cast<const VT*>(D)[e];
          VT rv = reinterpret_cast<const VT*>(R)[e];
          const V* pe = reinterpret_cast<const V*>(&pv);
          const V* qe = reinterpret_cast<const V*>(&qv);
          V* de = reinterpret_cast<V*>(&dv);
          V* re = reinterpret_cast<V*>(&rv);
#pragma unroll
          for (int j = 0; j < VW; ++j) {
            de[j] = al[j] * pe[j] + de[j];
            re[j] = -al[j] * qe[j] + re[j];
            pr[j] = re[j] * re[j] + pr[j];
          }
          reinterpret_cast<VT*>(D)[e] = dv;
          reinterpret_cast<VT*>(R)[e] = rv;
        }
        double v[1][VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) v[0][j] = (double)pr[j];
        const double s = group_reduce<VW, 1>(a, v, red, par, g, s_flag, ok);
        if (!ok) return false;
        if (t < 32) {
          bool go = false;
          if (t < kRhs && ((st.iact >> t) & 1u)) {
            if (st.bd[t]) {
              st.beta[t] = 0.0;
            } else {
              st.kin[t] += 1;
              st.used[t] += 1;
              if (sqrt(s) <= st.itol[t] * st.nr0[t]) {
                st.beta[t] = 0.0;
              } else {
                st.beta[t] = s / st.rr[t];
                st.rr[t] = s;
                go = st.used[t] < st.maxit;
              }
            }
          } else if (t < kRhs) {
            st.beta[t] = 0.0;
          }
          const unsigned m = __ballot_sync(~0u, go);
          if (t == 0) {
            st.iact = m;
            st.products += 1;
          }
        }
        __syncthreads();
      }
      if (!st.iact) break;
      // p = r + beta p
      {
        V be[VW];
#pragma unroll
        for (int j = 0; j < VW; ++j) be[j] = (V)st.beta[ch * VW + j];
        for (int64_t e = e0 + t; e < e1; e += NT) {
          const VT rv = reinterpret_cast<const VT*>(R)[e];
          VT pv = reinterpret_cast<const VT*>(P)[e];
          const V* re = reinterpret_cast<const V*>(&rv);
          V* pe = reinterpret_cast<V*>(&pv);
#pragma unroll
          for (int j = 0; j < VW; ++j) pe[j] = be[j] * pe[j] + re[j];
          reinterpret_cast<VT*>(P)[e] = pv;
        }
        if (!group_sync(a, g, s_flag)) return false;  // the new p of every CTA is visible to the next product
      }
    }
    // x += ||r|| x_inner in double precision; a breakdown before any
    // inner iteration ends that right-hand side
    {
      double nrv[VW];
      bool on[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) {
        const int k = ch * VW + j;
        on[j] = ((oact >> k) & 1u) && k < a.nrhs;
        nrv[j] = on[j] ? st.nr[k] : 0.0;
      }
      for (int64_t e = e0 + t; e < e1; e += NT) {
        const VT dv = reinterpret_cast<const VT*>(D)[e];
        const V* de = reinterpret_cast<const V*>(&dv);
        const int64_t row = e / CH;
#pragma unroll
        for (int j = 0; j < VW; ++j)
          if (on[j]) {
            double* xp = a.X + row * a.nrhs + ch * VW + j;
            *xp = fma(nrv[j], (double)de[j], *xp);
          }
      }
      if (t < 32) {
        bool stop = false;
        if (t < kRhs && ((oact >> t) & 1u)) {
          st.outer[t] += 1;
          // p'Ap <= 0: in double precision the Section III iteration stops
          // there; the refinement stops only when no inner step was taken
          if (st.bd[t] && (sizeof(V) == 8 || st.kin[t] == 0)) {
            st.status[t] = kNotSpd;
            stop = true;
          }
        }
        const unsigned m = __ballot_sync(~0u, stop);
        if (t == 0) st.fin |= m;
      }
      if (!group_sync(a, g, s_flag)) return false;  // x of every CTA is visible to the next residual product
    }
  }
  return true;
}

// Reliable updates for one instance (single-precision iterations, double-
// precision updates), all right-hand sides: the single-precision CG of the
// refinement's inner solve, but the correction d goes into x in double and
// the residual is replaced by b - A x in double whenever an active
// right-hand side's recurrence residual has fallen by inner_tol since its
// last update (or reached tol, or the iteration bound); the search
// directions are kept.  An update serves every right-hand side at once (an
// update is valid at any time).  outer counts the updates.
template <int NT>
__device__ bool solve_instance_ru(const BArgs& a, int inst, Group& g, Red& red, St& st, int& par, int* s_flag) {
  using VT = float4;
  constexpr int VW = 4, CH = 2;
  const int t = threadIdx.x;
  const int ch = t % CH;
  float* __restrict__ R = reinterpret_cast<float*>(a.R);
  float* __restrict__ P = reinterpret_cast<float*>(a.P);
  float* __restrict__ Q = reinterpret_cast<float*>(a.Q);
  float* __restrict__ D = reinterpret_cast<float*>(a.D);
  const int64_t row0 = a.inst_row[inst];
  const int64_t nI = a.inst_row[inst + 1] - row0;
  const int64_t GC = (int64_t)g.G * g.C, gc = (int64_t)g.p * g.C + g.cr;
  const int64_t per = (nI + GC - 1) / GC;
  const int64_t r0 = row0 + min64(nI, per * gc);
  const int64_t r1 = row0 + min64(nI, per * (gc + 1));
  const int rp = a.force_rpw > 0 ? a.force_rpw : (int)a.rpw[inst];
  const int64_t e0 = r0 * CH, e1 = r1 * CH;
  bool ok = true;
  if (t < 32) {
    if (t < kRhs) {
      st.used[t] = 0;
      st.outer[t] = 0;
      st.status[t] = kMaxit;
      st.rel[t] = 0.0;
      st.nb[t] = 0.0;
      st.bd[t] = 0;
    }
    const unsigned pad = __ballot_sync(~0u, t < kRhs && t >= a.nrhs);
    if (t == 0) {
      st.fin = pad;
      st.zero = 0;
      st.maxit = a.maxit > 0 ? a.maxit : (int)min64(nI, 0x7fffffff);
      st.products = 0;
      st.outers = 0;
    }
  }
  for (int64_t e = e0 + t; e < e1; e += NT) reinterpret_cast<VT*>(D)[e] = VT{};
  __syncthreads();
  // x += d (double), d = 0, R64 = B - A64 x; then decisions, R = float(R64), r'r
  auto update = [&](bool first) -> bool {
    {
      bool on[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) on[j] = ch * VW + j < a.nrhs;
      for (int64_t e = e0 + t; e < e1; e += NT) {
        VT dv = reinterpret_cast<const VT*>(D)[e];
        const float* de = reinterpret_cast<const float*>(&dv);
        const int64_t row = e / CH;
#pragma unroll
        for (int j = 0; j < VW; ++j)
          if (on[j] && de[j] != 0.f) a.X[row * a.nrhs + ch * VW + j] += (double)de[j];
        reinterpret_cast<VT*>(D)[e] = VT{};
      }
    }
    if (!group_sync(a, g, s_flag)) return false;  // x of every CTA before the product
    double v[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    outer_residual(a, r0, r1, v);
    const double s = group_reduce<2, 2>(a, v, red, par, g, s_flag, ok);
    if (!ok) return false;
    if (t >= kRhs && t < 2 * kRhs) red.sum[t] = s;
    __syncthreads();
    if (t < 32) {
      bool zero = false, done = false;
      if (t < kRhs && !((st.fin >> t) & 1u)) {
        if (first) st.nb[t] = sqrt(red.sum[kRhs + t]);
        const double nb = st.nb[t];
        if (nb == 0.0) {
          zero = true;
          done = true;
          st.status[t] = kOk;
          st.rel[t] = 0.0;
        } else {
          const double rel = sqrt(s) / nb;
          st.rel[t] = rel;
          if (!first) st.outer[t] += 1;
          if (!isfinite(rel)) {
            st.status[t] = kNonfinite;
            done = true;
          } else if (rel <= a.tol) {
            st.status[t] = kOk;
            done = true;
          } else if (st.used[t] >= st.maxit) {
            st.status[t] = kMaxit;
            done = true;
          }
        }
      }
      const unsigned zm = __ballot_sync(~0u, zero), dm = __ballot_sync(~0u, done);
      if (t == 0) {
        st.zero = zm;
        st.fin |= dm;
        st.outers += 1;
      }
    }
    __syncthreads();
    if (st.zero) {
      const unsigned zm = st.zero;
      for (int64_t row = r0 + t; row < r1; row += NT)
        for (int k = 0; k < a.nrhs; ++k)
          if ((zm >> k) & 1u) a.X[row * a.nrhs + k] = 0.0;
    }
    // R = float(R64) for the right-hand sides still running, r'r
    {
      const unsigned live = ~st.fin;
      bool on[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) on[j] = (live >> (ch * VW + j)) & 1u;
      float pr[VW] = {0.f, 0.f, 0.f, 0.f};
      for (int64_t e = e0 + t; e < e1; e += NT) {
        VT rv;
        float* re = reinterpret_cast<float*>(&rv);
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          re[j] = on[j] ? (float)a.R64[e * VW + j] : 0.f;
          pr[j] = fmaf(re[j], re[j], pr[j]);
        }
        reinterpret_cast<VT*>(R)[e] = rv;
      }
      double w[1][VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) w[0][j] = (double)pr[j];
      const double s2 = group_reduce<VW, 1>(a, w, red, par, g, s_flag, ok);
      if (!ok) return false;
      if (t < kRhs) {
        st.nr[t] = s2;  // r'r of the replaced residual
        st.rmax[t] = sqrt(s2);
      }
      __syncthreads();
    }
    return true;
  };
  if (!update(true)) return false;
  if (t < kRhs) st.rr[t] = st.nr[t];
  // p = r
  for (int64_t e = e0 + t; e < e1; e += NT) reinterpret_cast<VT*>(P)[e] = reinterpret_cast<const VT*>(R)[e];
  if (!group_sync(a, g, s_flag)) return false;
  while (~st.fin & 0xFFu) {
    // q = A32 p, p'q
    {
      float pq[VW] = {0.f, 0.f, 0.f, 0.f};
      product_rpw<float>(rp, a.ptr, a.idx, a.val32, P, r0, r1, [&](int64_t row, int c, VT acc) {
        const int64_t e = row * CH + c;
        reinterpret_cast<VT*>(Q)[e] = acc;
        const VT pv = reinterpret_cast<const VT*>(P)[e];
        const float* pe = reinterpret_cast<const float*>(&pv);
        const float* qe = reinterpret_cast<const float*>(&acc);
#pragma unroll
        for (int j = 0; j < VW; ++j) pq[j] = fmaf(pe[j], qe[j], pq[j]);
      });
      double v[1][VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) v[0][j] = (double)pq[j];
      const double s = group_reduce<VW, 1>(a, v, red, par, g, s_flag, ok);
      if (!ok) return false;
      if (t < 32) {
        bool stop = false;
        if (t < kRhs) {
          double al = 0.0;
          if (!((st.fin >> t) & 1u)) {
            if (!isfinite(s)) {
              st.status[t] = kNonfinite;
              stop = true;
            } else if (!(s > 0.0)) {
              st.status[t] = kNotSpd;
              stop = true;
            } else {
              al = st.rr[t] / s;
            }
          }
          st.alpha[t] = al;
        }
        const unsigned m = __ballot_sync(~0u, stop);
        if (t == 0) st.fin |= m;
      }
      __syncthreads();
    }
    // d += alpha p, r -= alpha q, r'r
    {
      float al[VW], pr[VW] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < VW; ++j) al[j] = (float)st.alpha[ch * VW + j];
      for (int64_t e = e0 + t; e < e1; e += NT) {
        const VT pv = reinterpret_cast<const VT*>(P)[e];
        const VT qv = reinterpret_cast<const VT*>(Q)[e];
        VT dv = reinterpret_cast<const VT*>(D)[e];
        VT rv = reinterpret_cast<const VT*>(R)[e];
        const float* pe = reinterpret_cast<const float*>(&pv);
        const float* qe = reinterpret_cast<const float*>(&qv);
        float* de = reinterpret_cast<float*>(&dv);
        float* re = reinterpret_cast<float*>(&rv);
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          de[j] = fmaf(al[j], pe[j], de[j]);
          re[j] = fmaf(-al[j], qe[j], re[j]);
          pr[j] = fmaf(re[j], re[j], pr[j]);
        }
        reinterpret_cast<VT*>(D)[e] = dv;
        reinterpret_cast<VT*>(R)[e] = rv;
      }
      double v[1][VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) v[0][j] = (double)pr[j];
      const double s = group_reduce<VW, 1>(a, v, red, par, g, s_flag, ok);
      if (!ok) return false;
      if (t < 32) {
        bool need = false;
        if (t < kRhs && !((st.fin >> t) & 1u) && st.alpha[t] != 0.0) {
          st.used[t] += 1;
          st.nr[t] = s;
          const double nr = sqrt(s);
          need = nr < a.inner_tol * st.rmax[t] || nr <= a.tol * st.nb[t] || st.used[t] >= st.maxit;
        } else if (t < kRhs) {
          st.nr[t] = st.rr[t];
        }
        const unsigned m = __ballot_sync(~0u, need);
        if (t == 0) {
          st.iact = m;
          st.products += 1;
        }
      }
      __syncthreads();
    }
    if (st.iact || !(~st.fin & 0xFFu)) {
      // a reliable update: x += d, r = b - A x in double (also flushes the
      // correction of right-hand sides that just stopped)
      if (!update(false)) return false;
      if (!(~st.fin & 0xFFu)) break;
    }
    // p = r + beta p
    {
      if (t < kRhs) {
        const bool live = !((st.fin >> t) & 1u);
        st.beta[t] = live ? st.nr[t] / st.rr[t] : 0.0;
        if (live) st.rr[t] = st.nr[t];
      }
      __syncthreads();
      float be[VW];
#pragma unroll
      for (int j = 0; j < VW; ++j) be[j] = (float)st.beta[ch * VW + j];
      for (int64_t e = e0 + t; e < e1; e += NT) {
        const VT rv = reinterpret_cast<const VT*>(R)[e];
        VT pv = reinterpret_cast<const VT*>(P)[e];
        const float* re = reinterpret_cast<const float*>(&rv);
        float* pe = reinterpret_cast<float*>(&pv);
#pragma unroll
        for (int j = 0; j < VW; ++j) pe[j] = fmaf(be[j], pe[j], re[j]);
        reinterpret_cast<VT*>(P)[e] = pv;
      }
      if (!group_sync(a, g, s_flag)) return false;
    }
  }
  return true;
}

// The persistent batched solver.  V is the precision of the inner CG (float:
// Section IV's single-precision iteration inside double-precision
// refinement; double: double precision throughout, where each refinement
// pass is a restart of the Section III iteration from the current x).  Each
// cluster takes queue slots in order; a slot is (instance, part) and an
// instance of G parts is solved by the G clusters that take its G slots.
template <typename V, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_bcg(const BArgs* __restrict__ args) {
  __shared__ BArgs a;
  __shared__ Red red;
  __shared__ St st;
  __shared__ int s_next, s_flag;
  __shared__ Group g;
  if (threadIdx.x == 0) {
    a = *args;
    g.C = cluster_ctas();
    g.cr = cluster_rank();
  }
  __syncthreads();
  const int t = threadIdx.x;
  int par = 0;
  cluster_sync();  // every CTA of the cluster is running before any shared-memory access across CTAs
  for (;;) {
    if (g.cr == 0 && t == 0) s_next = ld_relaxed_s32(a.err) != 0 ? a.nslots : atomicAdd(a.queue, 1);
    cluster_sync();
    const int qpos = ld_dsmem_s32(&s_next, 0);
    cluster_sync();
    if (qpos >= a.nslots) break;
    const int inst = a.slot_inst[qpos];
    if (t == 0) {
      g.p = a.slot_part[qpos];
      g.G = a.grp[inst];
      g.bar = a.gbar + inst;
      g.part = a.gpart + (int64_t)inst * (2 * kMaxGroup * 2 * kRhs);
      g.target = 0;
      g.gpar = 0;
    }
    __syncthreads();
    const bool lead = g.p == 0 && g.cr == 0;
    if (lead && t == 0) a.t_inst[2 * inst] = now_ns();
    bool ok;
    if constexpr (sizeof(V) == 4)
      ok = a.reliable ? solve_instance_ru<NT>(a, inst, g, red, st, par, &s_flag)
                      : solve_instance<V, NT>(a, inst, g, red, st, par, &s_flag);
    else
      ok = solve_instance<V, NT>(a, inst, g, red, st, par, &s_flag);
    if (!ok) {
      if (lead && t < a.nrhs) {
        gbcg_batch_info o = {st.used[t], st.outer[t], (int)kTimeout, 0, st.rel[t]};
        a.out[(int64_t)inst * a.nrhs + t] = o;
      }
      break;
    }
    if (lead && t < a.nrhs) {
      gbcg_batch_info o;
      o.iterations = st.used[t];
      o.outer = st.outer[t];
      o.status = st.status[t];
      o.pad_ = 0;
      o.rel_res_true = st.rel[t];
      a.out[(int64_t)inst * a.nrhs + t] = o;
    }
    if (lead && t == 0) {
      a.inst_iters[inst] = st.products;
      a.inst_outer[inst] = st.outers;
      a.t_inst[2 * inst + 1] = now_ns();
    }
    __syncthreads();  // st is rewritten by the next instance
  }
}

template <typename V, int NT>
void* kernel_of() {
  return (void*)k_bcg<V, NT>;
}

// ------------------------------------------------------------- host side
struct Tuning {
  int threads = 512, cluster = 8;
  int rpw[kBuckets] = {4, 4, 4, 2, 2, 1, 1, 1};
};

void* kernel_for(bool f32, int threads) {
  if (f32) return threads == 256 ? kernel_of<float, 256>() : kernel_of<float, 512>();
  return threads == 256 ? kernel_of<double, 256>() : kernel_of<double, 512>();
}

int max_clusters(void* k, int threads, int cluster, int* out) {
  *out = 0;
  if (cluster > 8) BCUDA(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaOccupancyMaxActiveClusters(out, k, &cfg);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *out = 0;
  }
  return 0;
}

int launch(void* k, int threads, int cluster, int clusters, const BArgs* dargs, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* params[] = {(void*)&dargs};
  BCUDA(cudaLaunchKernelExC(&cfg, k, params));
  return 0;
}

std::mutex g_tune_mu;
std::map<std::string, Tuning>& tune_cache() {
  static std::map<std::string, Tuning> m;
  return m;
}

}  // namespace

struct gbcg_batch_s {
  int count = 0, nrhs = 0, dev = 0;
  int64_t n_tot = 0, nnz_tot = 0, bytes = 0;
  std::vector<int64_t> row_off, nnz_of;
  std::vector<int> bucket;
  int64_t* d_inst_row = nullptr;
  int32_t *d_ptr = nullptr, *d_idx = nullptr, *d_slot_inst = nullptr, *d_slot_part = nullptr;
  int8_t* d_grp = nullptr;
  unsigned* d_gbar = nullptr;
  double* d_gpart = nullptr;
  int* d_err = nullptr;
  int* h_err = nullptr;  // pinned
  double* d_val64 = nullptr;
  float* d_val32 = nullptr;
  int8_t* d_rpw = nullptr;
  double* d_R64 = nullptr;
  void *d_R = nullptr, *d_P = nullptr, *d_Q = nullptr, *d_D = nullptr;
  double *d_Bst = nullptr, *d_Xst = nullptr;  // staging for host-memory b and x
  int* d_queue = nullptr;
  gbcg_batch_info* d_out = nullptr;
  int32_t *d_iters = nullptr, *d_outer = nullptr;
  long long* d_t = nullptr;
  BArgs* d_args = nullptr;
  BArgs* h_args = nullptr;          // pinned
  gbcg_batch_info* h_out = nullptr; // pinned
  int32_t *h_iters = nullptr, *h_outer = nullptr;
  long long* h_t = nullptr;
  std::vector<double> weight;      // per instance: expected cluster time (a priori, then measured)
  std::vector<int8_t> rpw_loaded;  // per-instance rows per warp now in d_rpw
  std::vector<int8_t> grp_loaded;  // schedule now on the device
  std::vector<int32_t> sinst_loaded, spart_loaded;
  Tuning tune[2];        // [0] double inner, [1] float inner
  bool tuned[2] = {false, false};
  int clusters[2] = {0, 0};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaStream_t cap = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool reorder = true;
};

namespace {

template <typename T>
int balloc(gbcg_batch_s* B, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return fail(GBCG_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  B->bytes += (int64_t)(count * sizeof(T));
  return 0;
}

void free_batch(gbcg_batch_s* B) {
  if (!B) return;
  for (int i = 0; i < 2; ++i) {
    if (B->exec[i]) cudaGraphExecDestroy(B->exec[i]);
    if (B->graph[i]) cudaGraphDestroy(B->graph[i]);
  }
  void* dev[] = {B->d_inst_row, B->d_ptr,  B->d_idx,  B->d_slot_inst, B->d_slot_part, B->d_grp,  B->d_gbar,
                 B->d_gpart,    B->d_err,  B->d_val64, B->d_val32,  B->d_rpw,       B->d_R64,  B->d_R,
                 B->d_P,        B->d_Q,    B->d_D,     B->d_Bst,    B->d_Xst,       B->d_queue, B->d_out,
                 B->d_iters,    B->d_outer, B->d_t,    B->d_args};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {B->h_args, B->h_out, B->h_iters, B->h_outer, B->h_t, B->h_err};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  delete B;
}

// The kernels read and write vectors with 16-byte loads and bulk copies.
bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int bucket_of(int64_t n, int64_t nnz) {
  if (n <= 0) return 0;
  const double avg = (double)nnz / (double)n;
  int b = 0;
  while (b + 1 < kBuckets && avg >= (double)(1 << (b + 1))) ++b;
  return b;
}

std::string tune_key(const gbcg_batch_s* B, bool f32) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, B->dev) != cudaSuccess) {
    (void)cudaGetLastError();
    memset(&pr, 0, sizeof(pr));
  }
  int hist[kBuckets] = {0};
  for (int b : B->bucket) hist[b]++;
  std::string k = std::string(pr.name) + "|sm" + std::to_string(pr.multiProcessorCount) + (f32 ? "|f32" : "|f64");
  auto lg = [](double v) { return (int)std::floor(std::log2(std::max(1.0, v))); };
  k += "|n" + std::to_string(lg((double)B->n_tot)) + "|z" + std::to_string(lg((double)B->nnz_tot)) + "|c" +
       std::to_string(lg((double)B->count)) + "|r" + std::to_string(B->nrhs);
  for (int b = 0; b < kBuckets; ++b) k += "|" + std::to_string(lg((double)hist[b]));
  return k;
}

int rpw_limit(bool f32) { return f32 ? 16 : 8; }

// Writes the per-instance rows-per-warp of tuning T to the device.
int apply_rpw(gbcg_batch_s* B, const Tuning& T, bool f32, cudaStream_t s) {
  std::vector<int8_t> h(B->count);
  for (int i = 0; i < B->count; ++i) h[i] = (int8_t)std::min(T.rpw[B->bucket[i]], rpw_limit(f32));
  if (h == B->rpw_loaded) return 0;
  B->rpw_loaded = h;
  BCUDA(cudaMemcpyAsync(B->d_rpw, h.data(), h.size(), cudaMemcpyHostToDevice, s));
  BCUDA(cudaStreamSynchronize(s));
  return 0;
}

// Queue of (instance, part) slots.  Instances whose expected cluster time
// exceeds the average load per cluster span G clusters (a power of two, at
// most max_group, the groups together holding at most half the clusters),
// so that no single instance outlasts the rest of the batch.  Groups come
// first in the queue, then single-cluster instances, each longest first.
void make_schedule(const gbcg_batch_s* B, int clusters, int max_group, int force_group, std::vector<int8_t>& grp,
                   std::vector<int32_t>& sinst, std::vector<int32_t>& spart) {
  const int n = B->count;
  const std::vector<double>& w = B->weight;
  grp.assign(n, 1);
  const int gmax = std::max(1, std::min(std::min(max_group, kMaxGroup), clusters));
  std::vector<int32_t> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) { return w[p] > w[q]; });
  if (force_group > 0) {
    const int G = std::min(force_group, gmax);
    for (int i = 0; i < n; ++i) grp[i] = (int8_t)G;
  } else if (gmax > 1 && clusters > 1) {
    const double W = std::accumulate(w.begin(), w.end(), 0.0) / clusters;
    int budget = clusters / 2;
    for (int i : ord) {
      if (!(w[i] > W)) break;
      int G = 1;
      while (G < gmax && w[i] / G > W) G *= 2;
      if (G > 1 && G <= budget) {
        grp[i] = (int8_t)G;
        budget -= G;
      }
    }
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) {
    const bool gp = grp[p] > 1, gq = grp[q] > 1;
    if (gp != gq) return gp;
    return w[p] / grp[p] > w[q] / grp[q];
  });
  sinst.clear();
  spart.clear();
  for (int i : ord)
    for (int part = 0; part < grp[i]; ++part) {
      sinst.push_back(i);
      spart.push_back(part);
    }
}

int upload_schedule(gbcg_batch_s* B, const std::vector<int8_t>& grp, const std::vector<int32_t>& sinst,
                    const std::vector<int32_t>& spart, cudaStream_t s) {
  if (grp == B->grp_loaded && sinst == B->sinst_loaded && spart == B->spart_loaded) return 0;
  BCUDA(cudaMemcpyAsync(B->d_grp, grp.data(), grp.size(), cudaMemcpyHostToDevice, s));
  BCUDA(cudaMemcpyAsync(B->d_slot_inst, sinst.data(), sizeof(int32_t) * sinst.size(), cudaMemcpyHostToDevice, s));
  BCUDA(cudaMemcpyAsync(B->d_slot_part, spart.data(), sizeof(int32_t) * spart.size(), cudaMemcpyHostToDevice, s));
  BCUDA(cudaStreamSynchronize(s));
  B->grp_loaded = grp;
  B->sinst_loaded = sinst;
  B->spart_loaded = spart;
  return 0;
}

// The single-cluster schedule (every G = 1), longest first.
int single_schedule(gbcg_batch_s* B, cudaStream_t s) {
  std::vector<int8_t> grp;
  std::vector<int32_t> si, sp;
  make_schedule(B, 1, 1, 0, grp, si, sp);
  return upload_schedule(B, grp, si, sp, s);
}

BArgs base_args(gbcg_batch_s* B) {
  BArgs a = {};
  a.inst_row = B->d_inst_row;
  a.ptr = B->d_ptr;
  a.idx = B->d_idx;
  a.val64 = B->d_val64;
  a.val32 = B->d_val32;
  a.slot_inst = B->d_slot_inst;
  a.slot_part = B->d_slot_part;
  a.grp = B->d_grp;
  a.gbar = B->d_gbar;
  a.gpart = B->d_gpart;
  a.err = B->d_err;
  a.nslots = (int)B->sinst_loaded.size();
  a.timeout_ns = 1000000000LL;
  a.rpw = B->d_rpw;
  a.R64 = B->d_R64;
  a.R = B->d_R;
  a.P = B->d_P;
  a.Q = B->d_Q;
  a.D = B->d_D;
  a.queue = B->d_queue;
  a.out = B->d_out;
  a.inst_iters = B->d_iters;
  a.inst_outer = B->d_outer;
  a.t_inst = B->d_t;
  a.count = B->count;
  a.nrhs = B->nrhs;
  return a;
}

// One probe launch (not captured): every instance runs `iters` inner
// iterations of one refinement pass with rows-per-warp `rpw` (0: the
// per-instance table).  Returns the launch time and fills h_t.
int probe(gbcg_batch_s* B, bool f32, int threads, int cluster, int clusters, int rpw, int iters, const double* Bp,
          double* Xp, cudaStream_t s, float* ms) {
  if (int rc = single_schedule(B, s)) return rc;
  BArgs a = base_args(B);
  a.B = Bp;
  a.X = Xp;
  a.tol = 0.0;
  a.inner_tol = 0.0;
  a.maxit = iters;
  a.max_outer = 1;
  a.force_rpw = rpw;
  *B->h_args = a;
  BCUDA(cudaMemcpyAsync(B->d_args, B->h_args, sizeof(BArgs), cudaMemcpyHostToDevice, s));
  BCUDA(cudaMemsetAsync(Xp, 0, sizeof(double) * (size_t)std::max<int64_t>(1, B->n_tot) * B->nrhs, s));
  BCUDA(cudaMemsetAsync(B->d_queue, 0, sizeof(int), s));
  BCUDA(cudaMemsetAsync(B->d_err, 0, sizeof(int), s));
  BCUDA(cudaMemsetAsync(B->d_gbar, 0, sizeof(unsigned) * B->count, s));
  BCUDA(cudaEventRecord(B->ev0, s));
  if (int rc = launch(kernel_for(f32, threads), threads, cluster, clusters, B->d_args, s)) return rc;
  BCUDA(cudaEventRecord(B->ev1, s));
  BCUDA(cudaMemcpyAsync(B->h_t, B->d_t, sizeof(long long) * 2 * B->count, cudaMemcpyDeviceToHost, s));
  BCUDA(cudaStreamSynchronize(s));
  BCUDA(cudaEventElapsedTime(ms, B->ev0, B->ev1));
  return 0;
}

int autotune(gbcg_batch_s* B, bool f32, gbcg_batch_tuning* rep, cudaStream_t s) {
  const std::string key = tune_key(B, f32);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      B->tune[f32] = it->second;
      B->tuned[f32] = true;
      if (rep) rep->from_cache = 1;
      return 0;
    }
  }
  // probe right-hand sides: ones (every system has a nonzero b)
  double *Bp = nullptr, *Xp = nullptr;
  const size_t nv = (size_t)std::max<int64_t>(1, B->n_tot) * B->nrhs;
  BCUDA(cudaMalloc(&Bp, sizeof(double) * nv));
  BCUDA(cudaMalloc(&Xp, sizeof(double) * nv));
  {
    std::vector<double> ones(nv, 1.0);
    cudaError_t e = cudaMemcpy(Bp, ones.data(), sizeof(double) * nv, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(Bp);
      cudaFree(Xp);
      return fail(GBCG_ERR_CUDA, std::string("autotune upload: ") + cudaGetErrorString(e));
    }
  }
  const int iters = 16;
  const int rpws_f32[] = {1, 2, 4, 8, 16}, rpws_f64[] = {1, 2, 4, 8};
  const int* rpws = f32 ? rpws_f32 : rpws_f64;
  const int nr = f32 ? 5 : 4;
  Tuning best;
  float best_ms = 1e30f;
  int cand = 0, rc = 0;
  for (int threads : {256, 512}) {
    for (int cluster : {1, 2, 4, 8, 16}) {
      int nc = 0;
      if ((rc = max_clusters(kernel_for(f32, threads), threads, cluster, &nc))) break;
      if (nc <= 0) continue;
      // per bucket: time of each rows-per-warp choice summed over the bucket's instances
      std::vector<std::vector<double>> tb(kBuckets, std::vector<double>(nr, 0.0));
      for (int j = 0; j < nr && !rc; ++j) {
        float ms = 0.f;
        if ((rc = probe(B, f32, threads, cluster, nc, rpws[j], iters, Bp, Xp, s, &ms))) break;
        ++cand;
        for (int i = 0; i < B->count; ++i) tb[B->bucket[i]][j] += (double)(B->h_t[2 * i + 1] - B->h_t[2 * i]);
      }
      if (rc) break;
      Tuning T;
      T.threads = threads;
      T.cluster = cluster;
      for (int b = 0; b < kBuckets; ++b) {
        int bj = 0;
        for (int j = 1; j < nr; ++j)
          if (tb[b][j] < tb[b][bj]) bj = j;
        T.rpw[b] = rpws[bj];
      }
      if ((rc = apply_rpw(B, T, f32, s))) break;
      float ms = 0.f;
      if ((rc = probe(B, f32, threads, cluster, nc, 0, iters, Bp, Xp, s, &ms))) break;
      ++cand;
      if (ms < best_ms) {
        best_ms = ms;
        best = T;
      }
    }
    if (rc) break;
  }
  cudaFree(Bp);
  cudaFree(Xp);
  if (rc) return rc;
  if (best_ms >= 1e30f) return fail(GBCG_ERR_CUDA, "autotune: no launchable cluster configuration");
  B->tune[f32] = best;
  B->tuned[f32] = true;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_cache()[key] = best;
  }
  if (rep) {
    rep->from_cache = 0;
    rep->probe_ms = best_ms;
    rep->candidates = cand;
  }
  return 0;
}

// Captures the solve graph of precision f32 with the current tuning: the
// argument block upload, the queue reset, the persistent launch and the
// result downloads.
int capture(gbcg_batch_s* B, bool f32) {
  const Tuning& T = B->tune[f32];
  if (B->exec[f32]) {
    cudaGraphExecDestroy(B->exec[f32]);
    B->exec[f32] = nullptr;
  }
  if (B->graph[f32]) {
    cudaGraphDestroy(B->graph[f32]);
    B->graph[f32] = nullptr;
  }
  int nc = 0;
  if (int rc = max_clusters(kernel_for(f32, T.threads), T.threads, T.cluster, &nc)) return rc;
  if (nc <= 0) return fail(GBCG_ERR_CUDA, "cluster configuration cannot be launched on this device");
  B->clusters[f32] = nc;
  cudaStream_t s = B->cap;
  BCUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int rc = 0;
  auto step = [&](cudaError_t e, const char* what) {
    if (!rc && e != cudaSuccess) rc = fail(GBCG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  step(cudaMemcpyAsync(B->d_args, B->h_args, sizeof(BArgs), cudaMemcpyHostToDevice, s), "capture args");
  step(cudaMemsetAsync(B->d_queue, 0, sizeof(int), s), "capture queue reset");
  step(cudaMemsetAsync(B->d_err, 0, sizeof(int), s), "capture error reset");
  step(cudaMemsetAsync(B->d_out, 0, sizeof(gbcg_batch_info) * (size_t)B->count * B->nrhs, s), "capture info reset");
  step(cudaMemsetAsync(B->d_gbar, 0, sizeof(unsigned) * B->count, s), "capture group barrier reset");
  if (!rc) rc = launch(kernel_for(f32, T.threads), T.threads, T.cluster, nc, B->d_args, s);
  step(cudaMemcpyAsync(B->h_out, B->d_out, sizeof(gbcg_batch_info) * (size_t)B->count * B->nrhs,
                       cudaMemcpyDeviceToHost, s),
       "capture info");
  step(cudaMemcpyAsync(B->h_iters, B->d_iters, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost, s), "capture iters");
  step(cudaMemcpyAsync(B->h_outer, B->d_outer, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost, s), "capture outer");
  step(cudaMemcpyAsync(B->h_t, B->d_t, sizeof(long long) * 2 * B->count, cudaMemcpyDeviceToHost, s), "capture times");
  step(cudaMemcpyAsync(B->h_err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "capture error flag");
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  BCUDA(e);
  B->graph[f32] = g;
  BCUDA(cudaGraphInstantiate(&B->exec[f32], g, 0));
  return 0;
}

int validate(int32_t count, const int64_t* row_off, const int32_t* ptr, const int32_t* idx, const double* val,
             std::string& err) {
  if (row_off[0] != 0) {
    err = "row_off[0] must be 0";
    return GBCG_ERR_INVALID;
  }
  for (int i = 0; i < count; ++i)
    if (row_off[i + 1] < row_off[i]) {
      err = "row_off decreases at instance " + std::to_string(i);
      return GBCG_ERR_INVALID;
    }
  const int64_t n = row_off[count];
  if (ptr[0] != 0) {
    err = "ptr[0] must be 0";
    return GBCG_ERR_INVALID;
  }
  for (int i = 0; i < count; ++i) {
    for (int64_t r = row_off[i]; r < row_off[i + 1]; ++r) {
      if (ptr[r + 1] < ptr[r]) {
        err = "ptr decreases at row " + std::to_string(r);
        return GBCG_ERR_INVALID;
      }
      for (int64_t k = ptr[r]; k < ptr[r + 1]; ++k) {
        const int64_t j = idx[k];
        if (j < row_off[i] || j >= row_off[i + 1]) {
          err = "entry " + std::to_string(k) + " of row " + std::to_string(r) + " has column " + std::to_string(j) +
                " outside instance " + std::to_string(i);
          return GBCG_ERR_INVALID;
        }
        if (k > ptr[r] && j <= idx[k - 1]) {
          err = "columns not strictly increasing in row " + std::to_string(r);
          return GBCG_ERR_INVALID;
        }
        if (!std::isfinite(val[k])) {
          err = "non-finite value at entry " + std::to_string(k);
          return GBCG_ERR_INVALID;
        }
      }
    }
  }
  (void)n;
  return GBCG_OK;
}

}  // namespace

extern "C" {

int gbcg_batch_create(gbcg_batch_t* out, int32_t count, const int64_t* row_off, const int32_t* ptr,
                      const int32_t* idx, const double* val, int32_t nrhs, int32_t memory, int32_t tune,
                      void* stream) {
  gbcg::set_last_error("");
  if (!out) return fail(GBCG_ERR_INVALID, "null output handle");
  *out = nullptr;
  if (count < 1) return fail(GBCG_ERR_INVALID, "count must be >= 1");
  if (nrhs < 1 || nrhs > kRhs) return fail(GBCG_ERR_INVALID, "nrhs must be in [1, 8]");
  if (!row_off || !ptr) return fail(GBCG_ERR_INVALID, "null row_off or ptr");
  if (memory != GBCG_HOST && memory != GBCG_DEVICE) return fail(GBCG_ERR_INVALID, "memory must be GBCG_HOST or GBCG_DEVICE");
  const int64_t n = row_off[count];
  if (n < 0 || n >= (int64_t)1 << 31) return fail(GBCG_ERR_INVALID, "total rows must be in [0, 2^31)");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> hptr, hidx;
  std::vector<double> hval;
  if (memory == GBCG_DEVICE) {
    hptr.resize(n + 1);
    BCUDA(cudaMemcpyAsync(hptr.data(), ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaStreamSynchronize(s));
    const int64_t z = hptr[n];
    if (z < 0) return fail(GBCG_ERR_INVALID, "ptr[n] is negative");
    if (z > 0) {
      if (!idx || !val) return fail(GBCG_ERR_INVALID, "null idx/val array");
      hidx.resize(z);
      hval.resize(z);
      BCUDA(cudaMemcpyAsync(hidx.data(), idx, sizeof(int32_t) * z, cudaMemcpyDeviceToHost, s));
      BCUDA(cudaMemcpyAsync(hval.data(), val, sizeof(double) * z, cudaMemcpyDeviceToHost, s));
      BCUDA(cudaStreamSynchronize(s));
    }
    ptr = hptr.data();
    idx = hidx.data();
    val = hval.data();
  }
  if (ptr[n] > 0 && (!idx || !val)) return fail(GBCG_ERR_INVALID, "null idx/val array");
  std::string err;
  if (int rc = validate(count, row_off, ptr, idx, val, err)) return fail(rc, err);
  const int64_t nnz = ptr[n];

  gbcg_batch_s* B = new gbcg_batch_s();
  B->count = count;
  B->nrhs = nrhs;
  B->n_tot = n;
  B->nnz_tot = nnz;
  B->row_off.assign(row_off, row_off + count + 1);
  B->nnz_of.resize(count);
  B->bucket.resize(count);
  for (int i = 0; i < count; ++i) {
    B->nnz_of[i] = (int64_t)ptr[row_off[i + 1]] - ptr[row_off[i]];
    B->bucket[i] = bucket_of(row_off[i + 1] - row_off[i], B->nnz_of[i]);
  }
  // a-priori cluster time: entries x rows^(1/3) (CG iterations of these
  // systems grow with the mesh diameter); replaced by measured times
  B->weight.resize(count);
  for (int i = 0; i < count; ++i)
    B->weight[i] = (double)B->nnz_of[i] * std::cbrt((double)(row_off[i + 1] - row_off[i]));
  auto bail = [&](int code) {
    free_batch(B);
    return code;
  };
  if (cudaGetDevice(&B->dev) != cudaSuccess) return bail(fail(GBCG_ERR_CUDA, "cudaGetDevice failed"));
  const size_t nv = (size_t)std::max<int64_t>(1, n) * kRhs;
  int rc = 0;
  if ((rc = balloc(B, &B->d_inst_row, count + 1)) || (rc = balloc(B, &B->d_ptr, n + 1)) ||
      (rc = balloc(B, &B->d_idx, nnz)) || (rc = balloc(B, &B->d_val64, nnz)) || (rc = balloc(B, &B->d_val32, nnz)) ||
      (rc = balloc(B, &B->d_slot_inst, (size_t)count * kMaxGroup)) ||
      (rc = balloc(B, &B->d_slot_part, (size_t)count * kMaxGroup)) || (rc = balloc(B, &B->d_grp, count)) ||
      (rc = balloc(B, &B->d_gbar, count)) || (rc = balloc(B, &B->d_gpart, (size_t)count * 2 * kMaxGroup * 2 * kRhs)) ||
      (rc = balloc(B, &B->d_err, 1)) || (rc = balloc(B, &B->d_rpw, count)) ||
      (rc = balloc(B, &B->d_R64, nv)) || (rc = balloc(B, (double**)&B->d_R, nv)) ||
      (rc = balloc(B, (double**)&B->d_P, nv)) || (rc = balloc(B, (double**)&B->d_Q, nv)) ||
      (rc = balloc(B, (double**)&B->d_D, nv)) || (rc = balloc(B, &B->d_Bst, (size_t)std::max<int64_t>(1, n) * nrhs)) ||
      (rc = balloc(B, &B->d_Xst, (size_t)std::max<int64_t>(1, n) * nrhs)) || (rc = balloc(B, &B->d_queue, 1)) ||
      (rc = balloc(B, &B->d_out, (size_t)count * nrhs)) || (rc = balloc(B, &B->d_iters, count)) ||
      (rc = balloc(B, &B->d_outer, count)) || (rc = balloc(B, &B->d_t, 2 * (size_t)count)) ||
      (rc = balloc(B, &B->d_args, 1)))
    return bail(rc);
  auto hostalloc = [&](void** p, size_t bytes) -> int {
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) return fail(GBCG_ERR_NOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    return 0;
  };
  if ((rc = hostalloc((void**)&B->h_args, sizeof(BArgs))) ||
      (rc = hostalloc((void**)&B->h_out, sizeof(gbcg_batch_info) * (size_t)count * nrhs)) ||
      (rc = hostalloc((void**)&B->h_iters, sizeof(int32_t) * count)) ||
      (rc = hostalloc((void**)&B->h_outer, sizeof(int32_t) * count)) ||
      (rc = hostalloc((void**)&B->h_t, sizeof(long long) * 2 * count)) ||
      (rc = hostalloc((void**)&B->h_err, sizeof(int))))
    return bail(rc);
  if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&B->ev0) != cudaSuccess || cudaEventCreate(&B->ev1) != cudaSuccess)
    return bail(fail(GBCG_ERR_CUDA, "stream/event creation failed"));
  {
    std::vector<float> v32(nnz);
    for (int64_t k = 0; k < nnz; ++k) v32[k] = (float)val[k];
    cudaError_t e = cudaSuccess;
    auto up = [&](void* d, const void* h, size_t bytes) {
      if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
    };
    up(B->d_inst_row, row_off, sizeof(int64_t) * (count + 1));
    up(B->d_ptr, ptr, sizeof(int32_t) * (n + 1));
    up(B->d_idx, idx, sizeof(int32_t) * nnz);
    up(B->d_val64, val, sizeof(double) * nnz);
    up(B->d_val32, v32.data(), sizeof(float) * nnz);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_out, 0, sizeof(gbcg_batch_info) * (size_t)count * nrhs, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(fail(GBCG_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e)));
  }
  for (int f = 0; f < 2; ++f)
    if ((rc = apply_rpw(B, B->tune[f], f == 1, s))) return bail(rc);
  if ((rc = single_schedule(B, s))) return bail(rc);
  if (tune) {
    if ((rc = autotune(B, true, nullptr, s))) return bail(rc);
    if ((rc = apply_rpw(B, B->tune[1], true, s))) return bail(rc);
  }
  *out = B;
  return GBCG_OK;
}

int gbcg_batch_destroy(gbcg_batch_t B) {
  free_batch(B);
  return GBCG_OK;
}

int gbcg_batch_autotune(gbcg_batch_t B, int32_t precision, gbcg_batch_tuning* rep, void* stream) {
  gbcg::set_last_error("");
  if (!B) return fail(GBCG_ERR_INVALID, "null batch handle");
  if (precision != GBCG_FP64 && precision != GBCG_FP32_IR) return fail(GBCG_ERR_INVALID, "unknown precision");
  const bool f32 = precision == GBCG_FP32_IR;
  if (rep) memset(rep, 0, sizeof(*rep));
  cudaStream_t s = (cudaStream_t)stream;
  if (int rc = autotune(B, f32, rep, s)) return rc;
  if (B->exec[f32]) {  // the captured graph belongs to the old configuration
    cudaGraphExecDestroy(B->exec[f32]);
    B->exec[f32] = nullptr;
  }
  if (rep) {
    const Tuning& T = B->tune[f32];
    rep->threads = T.threads;
    rep->cluster = T.cluster;
    for (int b = 0; b < kBuckets; ++b) rep->rows_per_warp[b] = std::min(T.rpw[b], rpw_limit(f32));
    int nc = 0;
    max_clusters(kernel_for(f32, T.threads), T.threads, T.cluster, &nc);
    rep->clusters = nc;
  }
  return GBCG_OK;
}

int gbcg_batch_set_tuning(gbcg_batch_t B, int32_t precision, const gbcg_batch_tuning* t) {
  gbcg::set_last_error("");
  if (!B || !t) return fail(GBCG_ERR_INVALID, "null argument");
  if (precision != GBCG_FP64 && precision != GBCG_FP32_IR) return fail(GBCG_ERR_INVALID, "unknown precision");
  const bool f32 = precision == GBCG_FP32_IR;
  if (t->threads != 256 && t->threads != 512) return fail(GBCG_ERR_INVALID, "threads must be 256 or 512");
  if (t->cluster != 1 && t->cluster != 2 && t->cluster != 4 && t->cluster != 8 && t->cluster != 16)
    return fail(GBCG_ERR_INVALID, "cluster must be 1, 2, 4, 8 or 16");
  Tuning T;
  T.threads = t->threads;
  T.cluster = t->cluster;
  for (int b = 0; b < kBuckets; ++b) {
    const int r = t->rows_per_warp[b];
    if (r != 1 && r != 2 && r != 4 && r != 8 && r != 16) return fail(GBCG_ERR_INVALID, "rows_per_warp must be 1, 2, 4, 8 or 16");
    if (r > rpw_limit(f32)) return fail(GBCG_ERR_INVALID, "rows_per_warp 16 needs the single-precision inner solve");
    T.rpw[b] = r;
  }
  B->tune[f32] = T;
  B->tuned[f32] = true;
  if (B->exec[f32]) {
    cudaGraphExecDestroy(B->exec[f32]);
    B->exec[f32] = nullptr;
  }
  return GBCG_OK;
}

int gbcg_batch_solve(gbcg_batch_t B, const double* b, double* x, double tol, int32_t maxit,
                     const gbcg_batch_opts* opts, gbcg_batch_info* infos, gbcg_batch_report* rep, void* stream) {
  gbcg::set_last_error("");
  const auto t0 = std::chrono::steady_clock::now();
  if (!B) return fail(GBCG_ERR_INVALID, "null batch handle");
  if (!(tol >= 0.0)) return fail(GBCG_ERR_INVALID, "tol must be >= 0");
  const int precision = opts ? opts->precision : GBCG_FP64;
  if (precision != GBCG_FP64 && precision != GBCG_FP32_IR && precision != GBCG_FP32_RU)
    return fail(GBCG_ERR_INVALID, "unknown precision");
  if (B->n_tot > 0 && (!b || !x)) return fail(GBCG_ERR_INVALID, "null b or x");
  const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  if (bdev != xdev) return fail(GBCG_ERR_INVALID, "b and x must both be device or both be host memory");
  if (bdev && (misaligned16(b) || misaligned16(x)))
    return fail(GBCG_ERR_INVALID, "device b and x must be 16-byte aligned");
  const int memory = bdev ? GBCG_DEVICE : GBCG_HOST;
  const bool f32 = precision != GBCG_FP64;  // both single-precision forms share tuning and graph
  cudaStream_t s = (cudaStream_t)stream;
  if (rep) memset(rep, 0, sizeof(*rep));
  int rc = 0;
  // the double-precision solve without its own tuning takes the single-precision one
  if (!f32 && !B->tuned[0] && B->tuned[1]) {
    B->tune[0] = B->tune[1];
    B->tuned[0] = true;
  }
  if (!B->exec[f32]) {
    if ((rc = apply_rpw(B, B->tune[f32], f32, s))) return rc;
    if ((rc = capture(B, f32))) return rc;
  } else if ((rc = apply_rpw(B, B->tune[f32], f32, s))) {
    return rc;
  }
  // schedule of this solve: group sizes from the expected cluster times
  const int max_group = (opts && opts->max_group > 0) ? opts->max_group : kMaxGroup;
  const int force_group = opts ? opts->force_group : 0;
  {
    std::vector<int8_t> grp;
    std::vector<int32_t> si, sp;
    make_schedule(B, B->clusters[f32], max_group, force_group, grp, si, sp);
    if ((rc = upload_schedule(B, grp, si, sp, s))) return rc;
  }
  const size_t nvb = sizeof(double) * (size_t)B->n_tot * B->nrhs;
  const double* bd = b;
  double* xd = x;
  if (memory == GBCG_HOST) {
    if (nvb) {
      BCUDA(cudaMemcpyAsync(B->d_Bst, b, nvb, cudaMemcpyHostToDevice, s));
      BCUDA(cudaMemcpyAsync(B->d_Xst, x, nvb, cudaMemcpyHostToDevice, s));
    }
    bd = B->d_Bst;
    xd = B->d_Xst;
  }
  BArgs a = base_args(B);
  a.B = bd;
  a.X = xd;
  a.tol = tol;
  a.reliable = precision == GBCG_FP32_RU;
  if (precision == GBCG_FP32_RU)
    a.inner_tol = (opts && opts->inner_tol > 0 && opts->inner_tol < 1) ? opts->inner_tol : 0.1;
  else
    a.inner_tol = f32 ? ((opts && opts->inner_tol > 0) ? opts->inner_tol : 1e-4) : 0.0;
  a.maxit = maxit;
  a.max_outer = (opts && opts->max_outer > 0) ? opts->max_outer : (f32 ? 30 : 4);
  a.force_rpw = 0;
  a.timeout_ns = (long long)((opts && opts->wait_timeout_ms > 0) ? opts->wait_timeout_ms : 1000) * 1000000LL;
  BCUDA(cudaStreamSynchronize(s));  // the previous solve's graph has read h_args
  *B->h_args = a;
  BCUDA(cudaEventRecord(B->ev0, s));
  BCUDA(cudaGraphLaunch(B->exec[f32], s));
  BCUDA(cudaEventRecord(B->ev1, s));
  if (memory == GBCG_HOST && nvb) BCUDA(cudaMemcpyAsync(x, B->d_Xst, nvb, cudaMemcpyDeviceToHost, s));
  BCUDA(cudaStreamSynchronize(s));
  float kms = 0.f;
  BCUDA(cudaEventElapsedTime(&kms, B->ev0, B->ev1));
  int status = GBCG_OK;
  int64_t total = 0, prods = 0;
  int maxits = 0;
  for (int i = 0; i < B->count; ++i) {
    prods += B->h_iters[i];
    for (int k = 0; k < B->nrhs; ++k) {
      const gbcg_batch_info& o = B->h_out[(size_t)i * B->nrhs + k];
      total += o.iterations;
      maxits = std::max(maxits, o.iterations);
      if (status == GBCG_OK && o.status != GBCG_OK) status = o.status;
    }
  }
  if (*B->h_err) {
    status = GBCG_ERR_TIMEOUT;
    gbcg::set_last_error("a multi-cluster group wait ran out; instances not reached report zeros");
  }
  if (infos) memcpy(infos, B->h_out, sizeof(gbcg_batch_info) * (size_t)B->count * B->nrhs);
  if (B->reorder && !(opts && opts->fixed_order) && !*B->h_err) {
    // next solve: measured cluster time (duration x clusters of the group)
    for (int i = 0; i < B->count; ++i) {
      const long long d = B->h_t[2 * i + 1] - B->h_t[2 * i];
      if (d > 0) B->weight[i] = (double)d * B->grp_loaded[i];
    }
  }
  if (rep) {
    const Tuning& T = B->tune[f32];
    rep->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    rep->kernel_ms = kms;
    rep->products = prods;
    rep->iterations = total;
    rep->max_iterations = maxits;
    rep->launches = 1;
    rep->graph = 1;
    rep->threads = T.threads;
    rep->cluster = T.cluster;
    rep->clusters = B->clusters[f32];
    for (int i = 0; i < B->count; ++i) {
      if (B->grp_loaded[i] > 1) rep->groups += 1;
      rep->max_group = std::max<int32_t>(rep->max_group, B->grp_loaded[i]);
    }
    long long lo = 0, hi = 0, busy = 0;
    for (int i = 0; i < B->count; ++i) {
      const long long a0 = B->h_t[2 * i], a1 = B->h_t[2 * i + 1];
      if (i == 0 || a0 < lo) lo = a0;
      if (i == 0 || a1 > hi) hi = a1;
      busy += (a1 - a0) * B->grp_loaded[i];
    }
    rep->span_ms = (double)(hi - lo) * 1e-6;
    rep->busy_fraction = (hi > lo && B->clusters[f32] > 0) ? (double)busy / ((double)(hi - lo) * B->clusters[f32]) : 0.0;
  }
  return status;
}

int gbcg_batch_selftest_group_timeout(gbcg_batch_t B, int32_t timeout_ms, void* stream) {
  gbcg::set_last_error("");
  if (!B) return fail(GBCG_ERR_INVALID, "null batch handle");
  if (timeout_ms <= 0) return fail(GBCG_ERR_INVALID, "timeout_ms must be > 0");
  cudaStream_t s = (cudaStream_t)stream;
  const Tuning& T = B->tune[1];
  int nc = 0;
  if (int rc = max_clusters(kernel_for(true, T.threads), T.threads, T.cluster, &nc)) return rc;
  if (nc < 2) return fail(GBCG_ERR_CUDA, "the self-test needs two co-resident clusters");
  // every instance on one cluster, except the last, a group of two whose
  // second slot is left out of the queue: its first part waits for a
  // partner that never comes
  std::vector<int8_t> grp;
  std::vector<int32_t> si, sp;
  make_schedule(B, 1, 1, 0, grp, si, sp);
  const int last = si.back();
  grp[last] = 2;
  if (int rc = upload_schedule(B, grp, si, sp, s)) return rc;
  if (int rc = apply_rpw(B, T, true, s)) return rc;
  const size_t nv = (size_t)std::max<int64_t>(1, B->n_tot) * B->nrhs;
  double *Bp = nullptr, *Xp = nullptr;
  BCUDA(cudaMalloc(&Bp, sizeof(double) * nv));
  cudaError_t e = cudaMalloc(&Xp, sizeof(double) * nv);
  if (e != cudaSuccess) {
    cudaFree(Bp);
    return fail(GBCG_ERR_NOMEM, "self-test buffers");
  }
  BArgs a = base_args(B);
  a.B = Bp;
  a.X = Xp;
  a.tol = 0.0;
  a.inner_tol = 0.0;
  a.maxit = 2;
  a.max_outer = 1;
  a.timeout_ns = (long long)timeout_ms * 1000000LL;
  *B->h_args = a;
  int rc = 0;
  auto step = [&](cudaError_t c, const char* what) {
    if (!rc && c != cudaSuccess) rc = fail(GBCG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(c));
  };
  step(cudaMemsetAsync(Bp, 0, sizeof(double) * nv, s), "self-test b");
  step(cudaMemsetAsync(Xp, 0, sizeof(double) * nv, s), "self-test x");
  step(cudaMemcpyAsync(B->d_args, B->h_args, sizeof(BArgs), cudaMemcpyHostToDevice, s), "self-test args");
  step(cudaMemsetAsync(B->d_queue, 0, sizeof(int), s), "self-test queue");
  step(cudaMemsetAsync(B->d_err, 0, sizeof(int), s), "self-test error flag");
  step(cudaMemsetAsync(B->d_gbar, 0, sizeof(unsigned) * B->count, s), "self-test group barriers");
  if (!rc) rc = launch(kernel_for(true, T.threads), T.threads, T.cluster, nc, B->d_args, s);
  step(cudaMemcpyAsync(B->h_err, B->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "self-test error read");
  step(cudaStreamSynchronize(s), "self-test sync");
  cudaFree(Bp);
  cudaFree(Xp);
  if (rc) return rc;
  return *B->h_err == kTimeout ? GBCG_ERR_TIMEOUT : GBCG_OK;
}

int gbcg_batch_instance_times(gbcg_batch_t B, int64_t* t_ns, int32_t* products, int32_t* outer_products) {
  if (!B) return fail(GBCG_ERR_INVALID, "null batch handle");
  for (int i = 0; i < B->count; ++i) {
    if (t_ns) {
      t_ns[2 * i] = B->h_t[2 * i];
      t_ns[2 * i + 1] = B->h_t[2 * i + 1];
    }
    if (products) products[i] = B->h_iters[i];
    if (outer_products) outer_products[i] = B->h_outer[i];
  }
  return GBCG_OK;
}

int gbcg_batch_stats(gbcg_batch_t B, gbcg_batch_stats_t* out) {
  if (!B || !out) return fail(GBCG_ERR_INVALID, "null argument");
  memset(out, 0, sizeof(*out));
  out->count = B->count;
  out->nrhs = B->nrhs;
  out->n = B->n_tot;
  out->nnz = B->nnz_tot;
  out->device_bytes = B->bytes;
  // one inner iteration over the whole batch: the single-precision matrix
  // (value + column) and row pointers once, and per row and right-hand side
  // the vector traffic of the fused passes (p gathered once, q written; p, q,
  // x, r read and x, r written; r, p read and p written: 11 accesses)
  out->iter_bytes_fp32 = 8 * B->nnz_tot + 4 * (B->n_tot + B->count) + 11 * 4 * kRhs * B->n_tot;
  out->iter_bytes_fp64 = 12 * B->nnz_tot + 4 * (B->n_tot + B->count) + 11 * 8 * kRhs * B->n_tot;
  for (int f = 0; f < 2; ++f) {
    out->threads[f] = B->tune[f].threads;
    out->cluster[f] = B->tune[f].cluster;
    for (int b = 0; b < kBuckets; ++b) out->rows_per_warp[f][b] = std::min(B->tune[f].rpw[b], rpw_limit(f == 1));
  }
  return GBCG_OK;
}

}  // extern "C"
