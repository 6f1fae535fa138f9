// kernels.cuh -- device code of the GB300 conjugate-gradient library (sm_103a).
//
// Sparse product (Section III, "A p product on line 2"): the sliced row-gather
// layout of layout.h, one warp per slice of 32 rows and one lane per row, as
// in the paper's thread-per-row kernel but with the row data interleaved so
// that a slice is one contiguous block.  Each warp streams its next slice's
// values and column indices into shared memory with a bulk asynchronous copy
// (cp.async.bulk, completion on an mbarrier, L2 evict-first policy) while it
// computes the current one, so the number of bytes in flight does not depend
// on how many warps are resident.  The symmetric format is computed by
// CTA-cooperative tiles (a producer warp streams tile stages; the entries of
// a tile come in conflict-free rounds, so the transpose half U' x is a
// shared-memory scatter without atomics, one barrier per round, and sums
// leaving a tile are added after a grid barrier), or, as a fallback, as a
// second row gather through a transpose plan that reads U's values in place.  The paper used a separate scatter kernel with atomics;
// here every output element is summed in a fixed order, so results are
// bitwise reproducible.
//
// CG iteration (Section III listing): one persistent cooperative launch per
// solve.  Each CTA owns a contiguous range of slices (and so of rows); per
// iteration it runs
//   A: q = A p on its rows, partial p'q            -> grid barrier
//   B: alpha = r'r / p'q; x += alpha p; r -= alpha q; partial r'r -> barrier
//   C: beta = r_k'r_k / r_{k-1}'r_{k-1}; p = r + beta p           -> barrier
// The partial sums of all CTAs are added by every CTA in the same fixed
// order, so every CTA takes the same decisions; the step's scalars (alpha,
// beta, the stopping tests) are formed once per CTA by thread 0 and
// broadcast through shared memory (GB300's FP64 pipe runs at 1/64 rate).  Every wait (grid barrier,
// mbarrier) is bounded by a global-timer limit; on expiry the CTA records
// GBCG_ERR_TIMEOUT and leaves at the next barrier, so nothing can hang.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "layout.h"  // TileDesc: the packed per-tile descriptor of the tiled symmetric layout

#include <type_traits>

namespace gbcg {

constexpr int kCgThreads = 512;
constexpr int kWarps = kCgThreads / 32;
// Tiled symmetric kernels: 15 consumer warps and one producer warp, so every
// persistent kernel runs 16 warps and keeps 128 registers per thread (a 17th
// warp puts five warps on one SM sub-partition and caps registers at 96).
constexpr int kTileThreads = kCgThreads;
constexpr int kTileWarps = kWarps - 1;  // consumer warps of a tile
constexpr int kMaxThreads = kCgThreads;
constexpr int kMaxL = 16;    // slots per row one pipeline stage holds
constexpr int kStages = 2;   // stages per warp
constexpr uint16_t kPlanPad = 0xFFFF;
constexpr int kMaxStages = 3 + 2;  // mbarriers per warp: a single- (3) and a double-precision (2) pipeline

// Layout modes of the product.
enum { kGather = 0, kPlan = 1, kTiles = 2 };

enum DevStatus { kOk = 0, kNotSpd = 2, kMaxit = 3, kNonfinite = 4, kTimeout = 5 };

template <typename V>
struct OpDev {
  int64_t n = 0, nslices = 0, nlong = 0;
  const int64_t* __restrict__ sl_ptr = nullptr;
  const int32_t* __restrict__ col = nullptr;
  const int16_t* __restrict__ col16 = nullptr;  // col - row, when every offset fits (row-gather layout)
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

// Tiled symmetric layout (layout.h, SymTilesHost).
template <typename V>
struct SymDev {
  const TileDesc* __restrict__ desc = nullptr;
  const int32_t* __restrict__ carry_src = nullptr;
  const int32_t* __restrict__ carry_dst = nullptr;
  const int32_t* __restrict__ carry_len = nullptr;
  const int32_t* __restrict__ flush_src = nullptr;
  const int32_t* __restrict__ flush_len = nullptr;
  const int32_t* __restrict__ flush_row = nullptr;
  const int32_t* __restrict__ cta_tile = nullptr;
  const int32_t* __restrict__ tile_slice = nullptr;
  const int32_t* __restrict__ tile_ns = nullptr;
  const int32_t* __restrict__ tile_own = nullptr;
  const int32_t* __restrict__ tile_len = nullptr;
  const int32_t* __restrict__ tile_stride = nullptr;
  const int64_t* __restrict__ tile_ent = nullptr;
  const int64_t* __restrict__ tile_meta = nullptr;
  const int64_t* __restrict__ tile_ext = nullptr;
  const int32_t* __restrict__ tile_win = nullptr;
  const int32_t* __restrict__ win_start = nullptr;
  const int32_t* __restrict__ win_len = nullptr;
  const V* __restrict__ val = nullptr;
  const uint16_t* __restrict__ meta = nullptr;
  const int32_t* __restrict__ in_ptr = nullptr;
  const int32_t* __restrict__ in_row = nullptr;
  const int32_t* __restrict__ in_len = nullptr;
  const int64_t* __restrict__ in_src = nullptr;
  V* part = nullptr;                      // further window partial sums (scratch)
  V* p1 = nullptr;                        // each row's first window partial sum (dense; 0 where none)
};

struct GridBar {
  unsigned long long count;  // arrivals since launch (monotone)
  int32_t status;            // first failure recorded by any CTA
  int32_t where;             // barrier index of that failure
  long long detail[4];       // facts about that failure (addresses, sizes)
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
  SymDev<V> T;
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
  int32_t stream_vec;         // tiled layout: stream the vector passes through shared memory
  long long timeout_ns;
};

// One pipeline stage of a warp: a slice's values then its column indices,
// both slot-major ([slot][lane]).
template <typename V>
struct alignas(16) Stage {
  V val[kMaxL * 32];
  int32_t col[kMaxL * 32];
};
// Stages per warp of the row-gather pipeline: three for single precision,
// two for double precision (FP64-FMA-bound; a third would not fit shared
// memory).  Measured on GB300, a fourth single-precision stage (or copies
// issued further ahead) made the solver slower: the streaming copies share
// the memory system with the latency-critical gathers, and lengthen them.
template <typename V>
__host__ __device__ constexpr int gather_stages() { return sizeof(V) == 4 ? 3 : kStages; }
template <typename V>
constexpr size_t pipe_smem_bytes() { return sizeof(Stage<V>) * gather_stages<V>() * kWarps; }

// Shared memory of the tiled symmetric product: the tile stages (filled by
// bulk copies: values, slots, diagonal, x over the tile's slots) and two
// accumulators over the slots (tiles alternate between them, so one can be
// cleared while the other is still being read).
// Caps of a tile, per precision: a consumer thread takes kRpt rows of the
// tile (rows l and l + 480), so single-precision tiles run up to 30 slices
// (960 rows) and amortise the per-tile work (stage wait, clears, epilogue:
// ~1000-1400 cycles on GB300) over twice the rows; double-precision tiles,
// whose stages are twice as large, stay at 15 slices.
template <typename V> struct TileCaps;
template <> struct TileCaps<float> {
  static constexpr int kRpt = 2, kEnt = 8192, kSlot = 3072;
};
template <> struct TileCaps<double> {
  static constexpr int kRpt = 1, kEnt = 4096, kSlot = 2048;
};
template <typename V>
constexpr int tile_rows() { return 32 * kTileWarps * TileCaps<V>::kRpt; }
constexpr uint16_t kPadSlot = 0x8000;  // slot flag of a padding entry
// A stage: the tile's descriptor (copied in by the producer warp before it
// issues the stage's bulk copies, published to the consumers by the same
// mbarrier phase), then the copied arrays.
template <typename V>
struct alignas(16) TileStage {
  TileDesc desc;
  V val[TileCaps<V>::kEnt];
  uint16_t meta[TileCaps<V>::kEnt + 8];  // slot of each entry (kPadSlot: padding)
  V diag[tile_rows<V>()];
  V xs[TileCaps<V>::kSlot];
};
// Tile stages per CTA: three in each precision (~64 KB each in single,
// ~61 KB in double precision), two in flight while one is consumed, which
// keeps the copies several tiles ahead of the consumers at GB300's HBM rate.
template <typename V>
__host__ __device__ constexpr int tile_stages() { return 3; }
constexpr int kMaxTileStages = 3;  // "full" and "empty" mbarriers per CTA: one pair per stage
template <typename V>
struct alignas(16) TileSmem {
  TileStage<V> st[tile_stages<V>()];
  V acc[2][TileCaps<V>::kSlot];
  uint16_t runs[7 * kDescRun];  // the current tile's inline carry and flush runs (the consumers' copy)
};
static_assert(sizeof(TileDesc) % 16 == 0, "stage payload alignment");
template <typename V>
constexpr size_t sym_smem_bytes() { return sizeof(TileSmem<V>); }
static_assert(sizeof(TileSmem<float>) <= 220 * 1024, "symmetric tiles: shared memory (float)");
static_assert(sizeof(TileSmem<double>) <= 220 * 1024, "symmetric tiles: shared memory (double)");

// Fill counters of the tile stages; like the gather pipeline's they persist
// across calls within one launch.
struct TilePipe {
  uint64_t* bar;      // "full" mbarrier per stage (shared memory): the stage's copies landed
  uint64_t* empty;    // "empty" mbarrier per stage: the consumers are done with it (kMaxTileStages each)
  // per stage b (bit b), kept in registers: parity of the fills issued
  // (producer) and of the fills waited for (consumers), and whether the
  // stage has been filled at all in this launch
  uint32_t iss_par, wait_par, used;
  uint64_t policy;       // matrix streams (read once per product): evict first
  uint64_t policy_x;     // x windows (each x read by up to three tiles' windows): normal, so they
                         // outlive the evict-first matrix stream in L2
  long long limit_ns;
  bool failed;
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
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = gtime();
  while (!mbar_try_wait(bar, parity))
    if (gtime() - t0 > limit_ns) return false;
  return true;
}
// Named barrier 1 over the `count` consumer threads (warps 0..count/32-1).
__device__ __forceinline__ void consumers_sync(int count) {
  asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}
// Same, returning whether `pred` holds on every consumer thread.
__device__ __forceinline__ bool consumers_and(int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(count)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy view of global memory before
// its later bulk copies (data written by plain stores and read by TMA).
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Orders this thread's earlier generic-proxy accesses of shared memory
// before later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
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

template <typename V> struct Vec;
template <> struct Vec<double> { using T = double2; static constexpr int W = 2; };
template <> struct Vec<float> { using T = float4; static constexpr int W = 4; };

// Row product of the lane's row in slice s straight from global memory
// (layout.h).  Symmetric rows sum in increasing column order: transpose half
// (columns < row), diagonal, upper half.
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

// Per-warp pipeline state (uniform across the warp's lanes).
struct Pipe {
  uint64_t* bars;      // nst mbarriers of this warp
  uint32_t nst;        // stages
  uint32_t issued;     // stage fills issued so far
  uint32_t consumed;   // stage fills consumed so far
  uint64_t policy;
  long long limit_ns;
  bool failed;
};

__device__ __forceinline__ void pipe_init(Pipe& pp, uint64_t* bars, uint32_t nst, long long limit_ns) {
  pp.bars = bars;
  pp.nst = nst;
  pp.issued = pp.consumed = 0;
  pp.policy = policy_evict_first();
  pp.limit_ns = limit_ns;
  pp.failed = false;
  if ((threadIdx.x & 31) == 0)
    for (uint32_t i = 0; i < nst; ++i) mbar_init(&bars[i], 1);
  fence_mbar_init();
}

template <typename V>
__device__ __forceinline__ int slice_len(const OpDev<V>& A, int64_t s) {
  return (int)((A.sl_ptr[s + 1] - A.sl_ptr[s]) >> 5);
}

// Offsets and lengths of a warp's slices, 32 at a time: lane l holds the
// warp's slice number 32w + l of window w (slices first, first + nw, ...),
// so one load fetches the metadata of the next 32 fills and issuing a fill
// waits on no load.  len_prev keeps the previous window's lengths for the
// fills still in flight when the issue side moves on.
struct SliceWin {
  int64_t beg = 0;
  int len = 0, len_prev = 0;
  int w = -1;
};

template <typename V>
__device__ __forceinline__ void win_at(const OpDev<V>& A, SliceWin& sw, int j, int64_t first, int64_t s1, int nw) {
  const int w = j >> 5;
  if (w == sw.w) return;
  sw.len_prev = sw.len;
  sw.w = w;
  const int64_t s = first + ((int64_t)w * 32 + (threadIdx.x & 31)) * nw;
  sw.beg = 0;
  sw.len = 0;
  if (s < s1) {
    sw.beg = A.sl_ptr[s];
    sw.len = (int)((A.sl_ptr[s + 1] - sw.beg) >> 5);
  }
}

// Length of the warp's slice number j (issued already: its window is the
// current one or the one before).
__device__ __forceinline__ int win_len(const SliceWin& sw, int j) {
  return __shfl_sync(0xffffffffu, (j >> 5) == sw.w ? sw.len : sw.len_prev, j & 31);
}

// Issue the fill of slice s into the next stage (no-op for empty or
// oversize slices, which are read straight from global memory).
template <typename V>
__device__ __forceinline__ void pipe_issue(const OpDev<V>& A, Stage<V>* stages, Pipe& pp, int64_t s) {
  const int L = slice_len(A, s);
  if (L == 0 || L > kMaxL || pp.failed) return;
  const uint32_t st = pp.issued % pp.nst;
  if ((threadIdx.x & 31) == 0) {
    const bool narrow = A.col16 != nullptr;
    const uint32_t vb = (uint32_t)(L * 32 * sizeof(V));
    const uint32_t cb = (uint32_t)(L * 32 * (narrow ? sizeof(int16_t) : sizeof(int32_t)));
    mbar_arrive_expect_tx(&pp.bars[st], vb + cb);
    bulk_g2s(stages[st].val, A.val + A.sl_ptr[s], vb, &pp.bars[st], pp.policy);
    if (narrow)
      bulk_g2s(stages[st].col, A.col16 + A.sl_ptr[s], cb, &pp.bars[st], pp.policy);
    else
      bulk_g2s(stages[st].col, A.col + A.sl_ptr[s], cb, &pp.bars[st], pp.policy);
  }
  ++pp.issued;
}

// pipe_issue for the warp's slice number j, its offset and length taken from
// the window.
template <typename V>
__device__ __forceinline__ void pipe_issue_win(const OpDev<V>& A, Stage<V>* stages, Pipe& pp, SliceWin& sw, int j,
                                               int64_t first, int64_t s1, int nw) {
  win_at(A, sw, j, first, s1, nw);
  const int L = __shfl_sync(0xffffffffu, sw.len, j & 31);
  const int64_t beg = __shfl_sync(0xffffffffu, sw.beg, j & 31);
  if (L == 0 || L > kMaxL || pp.failed) return;
  const uint32_t st = pp.issued % pp.nst;
  if ((threadIdx.x & 31) == 0) {
    const bool narrow = A.col16 != nullptr;
    const uint32_t vb = (uint32_t)(L * 32 * sizeof(V));
    const uint32_t cb = (uint32_t)(L * 32 * (narrow ? sizeof(int16_t) : sizeof(int32_t)));
    mbar_arrive_expect_tx(&pp.bars[st], vb + cb);
    bulk_g2s(stages[st].val, A.val + beg, vb, &pp.bars[st], pp.policy);
    if (narrow)
      bulk_g2s(stages[st].col, A.col16 + beg, cb, &pp.bars[st], pp.policy);
    else
      bulk_g2s(stages[st].col, A.col + beg, cb, &pp.bars[st], pp.policy);
  }
  ++pp.issued;
}

// Waits (bounded) for every fill still in flight; used before a CTA leaves
// after a failure so no copy lands in released shared memory.
__device__ __forceinline__ void pipe_drain(Pipe& pp) {
  while (pp.consumed < pp.issued) {
    const uint32_t st = pp.consumed % pp.nst, par = (pp.consumed / pp.nst) & 1u;
    mbar_wait(&pp.bars[st], par, pp.limit_ns);
    ++pp.consumed;
  }
}

// Calls f(row, y) or, when f takes three arguments, f(row, y, x_row) with
// x_row = x[row] loaded beside the product's gathers (saving the emitter a
// dependent load of its own row).
template <typename V, class F>
__device__ __forceinline__ void emit_row(F&& f, int64_t row, V y, V xr) {
  if constexpr (std::is_invocable_v<F, int64_t, V, V>)
    f(row, y, xr);
  else
    f(row, y);
}

// Visits the rows of slices [s0, s1) and long rows [l0, l1) of the CTA:
// f(row, (A x)_row[, x_row]) runs on the lane that computed the row.
// Row-gather formats use the per-warp bulk-copy pipeline; the symmetric
// format reads global memory directly.
template <typename V, bool SYM, bool NC, class F>
__device__ __forceinline__ void spmv_rows(const OpDev<V>& A, int64_t s0, int64_t s1, int64_t l0, int64_t l1,
                                          const V* x, Stage<V>* stages, Pipe& pp, int* err, F&& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (SYM) {  // transpose-plan layout
    for (int64_t s = s0 + warp; s < s1; s += nw) {
      const int64_t row = s * 32 + lane;
      const V xr = (std::is_invocable_v<F, int64_t, V, V> && row < A.n) ? ld_vec<NC>(x + row) : V(0);
      const V v = sell_row<V, true, NC, 4>(A, s, lane, x);
      if (row < A.n) emit_row<V>(f, row, v, xr);
    }
  } else if constexpr (NC) {
    // One-shot products take their slices' offsets and lengths from the
    // window (one load per 32 slices rather than one per slice on the issue
    // path): 6% (single) and 11% (double precision) faster on GB300 at 128^3.
    // The persistent solver keeps the per-slice loads below, because there a
    // faster issue path puts more copies in flight, and they lengthen the
    // round trip of the gathers (measured 2-4% slower per iteration).
    const int64_t first = s0 + warp;
    const int J = first < s1 ? (int)((s1 - first + nw - 1) / nw) : 0;  // slices of this warp
    SliceWin sw;
    int j_issue = 0;
    while (j_issue + 1 < (int)pp.nst && j_issue < J)
      pipe_issue_win(A, stages, pp, sw, j_issue++, first, s1, nw);
    for (int j = 0; j < J; ++j) {
      if (j_issue < J) pipe_issue_win(A, stages, pp, sw, j_issue++, first, s1, nw);
      const int64_t s = first + (int64_t)j * nw;
      const int L = win_len(sw, j);
      const int64_t row = s * 32 + lane;
      const V xr = (std::is_invocable_v<F, int64_t, V, V> && row < A.n) ? ld_vec<NC>(x + row) : V(0);
      V acc = V(0);
      if (L > kMaxL) {
        acc = sell_row<V, false, NC, 8>(A, s, lane, x);
      } else if (L > 0 && !pp.failed) {
        const uint32_t st = pp.consumed % pp.nst, par = (pp.consumed / pp.nst) & 1u;
        if (!mbar_wait(&pp.bars[st], par, pp.limit_ns)) {
          pp.failed = true;
          if (lane == 0) atomicCAS(err, 0, (int)kTimeout);
        } else {
          ++pp.consumed;
          const V* __restrict__ sv = stages[st].val;
          V xv[kMaxL];
          if (A.col16) {  // 16-bit offsets from the row (lanes past the last row read x[0])
            const int16_t* __restrict__ sc = reinterpret_cast<const int16_t*>(stages[st].col);
            const V* xb = x + (row < A.n ? row : 0);
#pragma unroll
            for (int k = 0; k < kMaxL; ++k)
              if (k < L) xv[k] = ld_vec<NC>(xb + sc[k * 32 + lane]);
          } else {
            const int32_t* __restrict__ sc = stages[st].col;
#pragma unroll
            for (int k = 0; k < kMaxL; ++k)
              if (k < L) xv[k] = ld_vec<NC>(x + sc[k * 32 + lane]);
          }
#pragma unroll
          for (int k = 0; k < kMaxL; ++k)
            if (k < L) acc = fma_(sv[k * 32 + lane], xv[k], acc);
        }
        __syncwarp();
      }
      if (row < A.n && !((A.long_mask[s] >> lane) & 1u)) emit_row<V>(f, row, acc, xr);
    }
    if (pp.failed) pipe_drain(pp);
  } else {
    int64_t s_issue = s0 + warp;
    for (uint32_t d = 0; d + 1 < pp.nst && s_issue < s1; ++d, s_issue += nw) pipe_issue(A, stages, pp, s_issue);
    for (int64_t s = s0 + warp; s < s1; s += nw) {
      if (s_issue < s1) {
        pipe_issue(A, stages, pp, s_issue);
        s_issue += nw;
      }
      const int L = slice_len(A, s);
      const int64_t row = s * 32 + lane;
      const V xr = (std::is_invocable_v<F, int64_t, V, V> && row < A.n) ? ld_vec<NC>(x + row) : V(0);
      V acc = V(0);
      if (L > kMaxL) {
        acc = sell_row<V, false, NC, 8>(A, s, lane, x);
      } else if (L > 0 && !pp.failed) {
        const uint32_t st = pp.consumed % pp.nst, par = (pp.consumed / pp.nst) & 1u;
        if (!mbar_wait(&pp.bars[st], par, pp.limit_ns)) {
          pp.failed = true;
          if (lane == 0) atomicCAS(err, 0, (int)kTimeout);
        } else {
          ++pp.consumed;
          const V* __restrict__ sv = stages[st].val;
          V xv[kMaxL];
          if (A.col16) {  // 16-bit offsets from the row (lanes past the last row read x[0])
            const int16_t* __restrict__ sc = reinterpret_cast<const int16_t*>(stages[st].col);
            const V* xb = x + (row < A.n ? row : 0);
#pragma unroll
            for (int k = 0; k < kMaxL; ++k)
              if (k < L) xv[k] = ld_vec<NC>(xb + sc[k * 32 + lane]);
          } else {
            const int32_t* __restrict__ sc = stages[st].col;
#pragma unroll
            for (int k = 0; k < kMaxL; ++k)
              if (k < L) xv[k] = ld_vec<NC>(x + sc[k * 32 + lane]);
          }
#pragma unroll
          for (int k = 0; k < kMaxL; ++k)
            if (k < L) acc = fma_(sv[k * 32 + lane], xv[k], acc);
        }
        __syncwarp();
      }
      if (row < A.n && !((A.long_mask[s] >> lane) & 1u)) emit_row<V>(f, row, acc, xr);
    }
    if (pp.failed) pipe_drain(pp);
  }
  for (int64_t li = l0 + warp; li < l1; li += nw) {
    const V v = long_row<V, NC>(A, li, lane, x);
    if (lane == 0) {
      const int64_t row = A.long_row[li];
      emit_row<V>(f, row, v, std::is_invocable_v<F, int64_t, V, V> ? ld_vec<NC>(x + row) : V(0));
    }
  }
}


// ------------------------------------------------- symmetric tiles ---
// for i = lane, lane + 32, ... < len: st(i, ld(i)), with B loads in flight
// per lane before the first store (the loads are independent).
template <int B, class LD, class ST>
__device__ __forceinline__ void batched(int lane, int len, LD&& ld, ST&& st) {
  for (int i0 = 0; i0 < len; i0 += 32 * B) {
    decltype(ld(0)) v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int i = i0 + u * 32 + lane;
      if (i < len) v[u] = ld(i);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int i = i0 + u * 32 + lane;
      if (i < len) st(i, v[u]);
    }
  }
}

// Window w of the tile (inline in the descriptor, else from the global list).
template <typename V>
__device__ __forceinline__ void tile_window(const TileDesc& d, const SymDev<V>& T, int w, int32_t& ws, int32_t& wl) {
  if (w < kDescWin) {
    ws = d.ws[w];
    wl = d.wl[w];
  } else {
    ws = T.win_start[d.win0 + w];
    wl = T.win_len[d.win0 + w];
  }
}

// Issues (producer lane 0) the bulk copies of the tile whose descriptor
// stage bf holds: values, slot blob, diagonal, and the x slots (own rows and
// windows) that are 16-byte aligned; the rest is loaded by tile_tail.
template <typename V>
__device__ __forceinline__ void tile_issue(const OpDev<V>& A, const SymDev<V>& T, TileStage<V>& st, TilePipe& tp,
                                           int bf, const V* x) {
  const TileDesc& d = st.desc;
  uint64_t* bar = &tp.bar[bf];
  const uint32_t vb = (uint32_t)(d.E8 * sizeof(V)), mb = (uint32_t)(d.E8 * sizeof(uint16_t));
  const uint32_t db = (uint32_t)(d.nsl * 32 * sizeof(V));
  const bool own_bulk = (d.rows & 3) == 0;
  uint32_t bytes = vb + mb + db + (own_bulk ? (uint32_t)(d.rows * sizeof(V)) : 0u);
  for (int w = 0; w < d.nwin; ++w) {
    int32_t ws, wl;
    tile_window(d, T, w, ws, wl);
    if (((ws | wl) & 3) == 0) bytes += (uint32_t)(wl * sizeof(V));
  }
  fence_proxy_async_global();
  mbar_arrive_expect_tx(bar, bytes);
  if (vb) bulk_g2s(st.val, T.val + d.e0, vb, bar, tp.policy);
  if (mb) bulk_g2s(st.meta, T.meta + d.m0, mb, bar, tp.policy);
  bulk_g2s(st.diag, A.diag + d.row0, db, bar, tp.policy);
  if (own_bulk && d.rows > 0) bulk_g2s(st.xs, x + d.row0, (uint32_t)(d.rows * sizeof(V)), bar, tp.policy_x);
  int32_t slot = d.own;
  for (int w = 0; w < d.nwin; ++w) {
    int32_t ws, wl;
    tile_window(d, T, w, ws, wl);
    if (((ws | wl) & 3) == 0 && wl > 0) bulk_g2s(st.xs + slot, x + ws, (uint32_t)(wl * sizeof(V)), bar, tp.policy_x);
    slot += wl;
  }
  tp.iss_par ^= 1u << bf;
  tp.used |= 1u << bf;
}

// Plain loads (consumer threads) of the x slots tile_issue left out: rows or
// windows not 16-byte aligned, which occur only at the end of the matrix.
template <typename V, bool NC>
__device__ __forceinline__ void tile_tail(const SymDev<V>& T, TileStage<V>& st, const V* x, int nthreads) {
  const TileDesc& d = st.desc;
  if ((d.rows & 3) != 0)
    for (int i = threadIdx.x; i < d.rows; i += nthreads) st.xs[i] = ld_vec<NC>(x + d.row0 + i);
  int32_t slot = d.own;
  for (int w = 0; w < d.nwin; ++w) {
    int32_t ws, wl;
    tile_window(d, T, w, ws, wl);
    if (((ws | wl) & 3) != 0)
      for (int i = threadIdx.x; i < wl; i += nthreads) st.xs[slot + i] = ld_vec<NC>(x + ws + i);
    slot += wl;
  }
}

// Symmetric product over the CTA's tiles (a producer warp streams tiles into
// the stages; 15 consumer warps cooperate on each tile, one lane per row).
// In round k every row takes its round-k entry (i, j): the direct sum
// (U x)_i gains U_ij x_j from the staged x, and slot j's accumulator gains
// U_ij x_i; the layout guarantees that no two entries of a round target the
// same slot, and a barrier separates the rounds, so each slot's sum is formed
// in round order without atomics.  The accumulator of a tile starts with what
// the previous tile of the CTA carried into it (window rows both tiles
// cover).  Then f(row, own part of (A x)_row, x_i, D_i x_i, (U x)_i) runs on
// the row's lane; window slots are carried into the next tile's accumulator
// or leave as partial sums.  Uniform control flow: every consumer thread
// takes every barrier.
template <typename V, bool NC, class F>
__device__ __forceinline__ void sym_tiles(const OpDev<V>& A, const SymDev<V>& T, const V* x, TileSmem<V>* sm,
                                          TilePipe& tp, int* err, F&& f) {
  constexpr int NST = tile_stages<V>();
  constexpr int NC_THREADS = 32 * kTileWarps;  // consumers: warps 0..14; warp 15 produces
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, c = blockIdx.x;
  const int32_t t0 = T.cta_tile[c], t1 = T.cta_tile[c + 1];
  if (t0 >= t1) return;
  if (warp == kTileWarps) {
    // producer: lane 0 waits for a free stage and issues its copies; lanes
    // 0..15 bring the tile's descriptor into the stage first.  Descriptors
    // are loaded kDescAhead tiles ahead into a register ring (lane l holds
    // the l-th 16 bytes of each): with only the next one in flight, the
    // producer issued one tile per DRAM round trip (~1 us), which bounded the
    // product (measured 1.3 us per tile against ~0.4 us of consumer work).
    constexpr int kDescVecs = (int)(sizeof(TileDesc) / 16);
    constexpr int kDescAhead = 6;
    int4 dq[kDescAhead];
#pragma unroll
    for (int k = 0; k < kDescAhead; ++k) {
      dq[k] = make_int4(0, 0, 0, 0);
      if (lane < kDescVecs && t0 + k < t1) dq[k] = __ldg(reinterpret_cast<const int4*>(T.desc + t0 + k) + lane);
    }
    for (int32_t t = t0; t < t1; ++t) {
      const int b = (int)((t - t0) % NST);
      int ok = !tp.failed;
      if (lane == 0 && ok && ((tp.used >> b) & 1u) &&
          !mbar_wait(&tp.empty[b], ((tp.iss_par >> b) & 1u) ^ 1u, tp.limit_ns)) {
        ok = 0;
        if (atomicCAS(err, 0, (int)kTimeout) == 0) err[1] = 400000000 + (int)(t % 1000000) * 10 + b;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        tp.failed = true;
        break;
      }
      __syncwarp();  // lane 0's wait for the free stage is ordered before the lanes' writes
      TileStage<V>& st = sm->st[b];
      if (lane < kDescVecs) reinterpret_cast<int4*>(&st.desc)[lane] = dq[0];
#pragma unroll
      for (int k = 0; k + 1 < kDescAhead; ++k) dq[k] = dq[k + 1];
      if (lane < kDescVecs && t + kDescAhead < t1)
        dq[kDescAhead - 1] = __ldg(reinterpret_cast<const int4*>(T.desc + t + kDescAhead) + lane);
      __syncwarp();
      if (lane == 0) tile_issue(A, T, st, tp, b, x);
      __syncwarp();
    }
    // the CTA must not move on while its copies are in flight: wait
    // (bounded) for the last fill of every stage to land
    if (lane == 0)
      for (int b = 0; b < NST; ++b)
        if ((tp.used >> b) & 1u) mbar_wait(&tp.bar[b], ((tp.iss_par >> b) & 1u) ^ 1u, tp.limit_ns);
    __syncwarp();
    return;
  }
  // the first tile's accumulator starts at zero (the barrier of the first
  // tile orders this before its rounds)
  for (int v4 = threadIdx.x; v4 < (int)(TileCaps<V>::kSlot * sizeof(V) / 16); v4 += NC_THREADS)
    reinterpret_cast<int4*>(sm->acc[0])[v4] = make_int4(0, 0, 0, 0);
  for (int32_t t = t0; t < t1; ++t) {
    const int j = (int)(t - t0), bf = j % NST;
    TileStage<V>& st = sm->st[bf];
    V* __restrict__ acc = sm->acc[j & 1];
    V* __restrict__ acc_next = sm->acc[(j + 1) & 1];
    bool ok = !tp.failed;
    if (ok) {
      ok = mbar_wait(&tp.bar[bf], (tp.wait_par >> bf) & 1u, tp.limit_ns);
      if (!ok && atomicCAS(err, 0, (int)kTimeout) == 0) err[1] = 300000000 + (int)(t % 1000000) * 10 + bf;
    }
    if (ok && st.desc.tail) tile_tail<V, NC>(T, st, x, NC_THREADS);
    ok = consumers_and(NC_THREADS, ok);
    if (!ok) {
      tp.failed = true;
      continue;
    }
    tp.wait_par ^= 1u << bf;
    // the tile's geometry into registers (the descriptor goes with the stage)
    const TileDesc& d = st.desc;
    const int g_rows = d.rows, g_D = d.D, g_S = d.S, g_own = d.own, R = d.R;
    const int g_nc = d.nc, g_nf = d.nf, g_c0 = d.carry0, g_f0 = d.flush0;
    const int64_t g_row0 = d.row0, g_ext0 = d.ext0;
    // the next tile's accumulator is cleared here, its carried values are
    // written after this tile's rounds; this tile's inline runs are kept for
    // the end of the tile (the stage is released before)
    for (int v4 = threadIdx.x; v4 < (int)(TileCaps<V>::kSlot * sizeof(V) / 16); v4 += NC_THREADS)
      reinterpret_cast<int4*>(acc_next)[v4] = make_int4(0, 0, 0, 0);
    if (threadIdx.x < 7 * kDescRun) sm->runs[threadIdx.x] = (&d.cs[0])[threadIdx.x];  // cs, cd, cl, fs, fl, fr
    const uint16_t* __restrict__ slot = st.meta;
    const V* __restrict__ val = st.val;
    const V* __restrict__ xs = st.xs;
    // rounds: in round k each row's round-k entry (i, j) adds U_ij x_j to
    // the row's direct sum and U_ij x_i to slot j's accumulator; no two
    // entries of a round share a slot (over all the tile's rows), so the
    // scatter needs no atomics, and the barrier after each round orders the
    // additions into a slot.  Thread t takes rows t and t + 480 (single
    // precision) or row t (double precision).
    constexpr int RPT = TileCaps<V>::kRpt;
    V xi[RPT], dg[RPT], direct[RPT];
    bool mine[RPT];
#pragma unroll
    for (int h = 0; h < RPT; ++h) {
      const int row = threadIdx.x + h * NC_THREADS;
      mine[h] = row < g_rows;
      xi[h] = mine[h] ? xs[row] : V(0);
      dg[h] = mine[h] ? st.diag[row] : V(0);
      direct[h] = V(0);
    }
    {
      // each round's entries are loaded one round ahead, before the current
      // round's chain of dependent shared-memory accesses
      uint32_t sn[RPT];
      V vn[RPT];
#pragma unroll
      for (int h = 0; h < RPT; ++h) {
        const int e = threadIdx.x + h * NC_THREADS;
        sn[h] = mine[h] && g_D > 0 ? (uint32_t)slot[e] : (uint32_t)kPadSlot;
        vn[h] = mine[h] && g_D > 0 ? val[e] : V(0);
      }
      for (int k = 0; k < g_D; ++k) {
        uint32_t s16[RPT];
        V v[RPT];
#pragma unroll
        for (int h = 0; h < RPT; ++h) {
          s16[h] = sn[h];
          v[h] = vn[h];
          if (mine[h] && k + 1 < g_D) {
            const int e = threadIdx.x + h * NC_THREADS + (k + 1) * R;
            sn[h] = slot[e];
            vn[h] = val[e];
          }
        }
#pragma unroll
        for (int h = 0; h < RPT; ++h)
          if (!(s16[h] & kPadSlot)) {
            direct[h] = fma_(v[h], xs[s16[h]], direct[h]);
            acc[s16[h]] = fma_(v[h], xi[h], acc[s16[h]]);
          }
        consumers_sync(NC_THREADS);
      }
    }
    if (g_D == 0) consumers_sync(NC_THREADS);  // every read of the stage is done
    // the stage is free: release it to the producer
    if (threadIdx.x == 0) mbar_arrive(&tp.empty[bf]);
#pragma unroll
    for (int h = 0; h < RPT; ++h)
      if (mine[h]) {
        const int row = threadIdx.x + h * NC_THREADS;
        const V dxi = dg[h] * xi[h];
        f(g_row0 + row, dxi + direct[h] + acc[row], xi[h], dxi, direct[h]);
      }
    // window slots: carried into the next tile's accumulator, or out as
    // partial sums (runs past the inline ones come from the global lists)
    const uint16_t* cs = sm->runs;
    for (int u = 0; u < g_nc; ++u) {
      const int s0 = u < kDescRun ? cs[u] : T.carry_src[g_c0 + u];
      const int d0 = u < kDescRun ? cs[kDescRun + u] : T.carry_dst[g_c0 + u];
      const int len = u < kDescRun ? cs[2 * kDescRun + u] : T.carry_len[g_c0 + u];
      for (int i = threadIdx.x; i < len; i += NC_THREADS) acc_next[d0 + i] = acc[s0 + i];
    }
    // a direct run writes its rows' first partial sums to the dense array;
    // the others go to the compact one
    V* __restrict__ part = T.part + g_ext0 - g_own;
    const int32_t* frow = reinterpret_cast<const int32_t*>(cs + 5 * kDescRun);
    for (int u = 0; u < g_nf; ++u) {
      const int s0 = u < kDescRun ? cs[3 * kDescRun + u] : T.flush_src[g_f0 + u];
      const int len = u < kDescRun ? cs[4 * kDescRun + u] : T.flush_len[g_f0 + u];
      const int r0 = u < kDescRun ? frow[u] : T.flush_row[g_f0 + u];
      V* __restrict__ dst = r0 >= 0 ? T.p1 + r0 - s0 : part;
      for (int i = threadIdx.x; i < len; i += NC_THREADS) dst[s0 + i] = acc[s0 + i];
    }
    (void)g_S;
  }
}

// Adds the listed window partial sums (a row's second and later ones) to y
// over the CTA's tiles (warp w takes tiles t0 + w, t0 + w + 16, ...), runs in
// the layout's fixed order.
template <typename V>
__device__ __forceinline__ void sym_incoming(const SymDev<V>& T, V* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, c = blockIdx.x;
  for (int32_t t = T.cta_tile[c] + warp; t < T.cta_tile[c + 1]; t += nw) {
    const int64_t row0 = (int64_t)T.tile_slice[t] * 32;
    for (int32_t u = T.in_ptr[t]; u < T.in_ptr[t + 1]; ++u) {
      const int64_t rr = row0 + T.in_row[u], src = T.in_src[u];
      const int len = T.in_len[u];
      batched<8>(lane, len, [&](int l) { return y[rr + l] + T.part[src + l]; }, [&](int l, V v) { y[rr + l] = v; });
      __syncwarp();
    }
  }
}

__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float4 vadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// y += the dense first partial sums over rows [r0, r1) of the CTA (after
// sym_incoming: the product of the tiled layout is then complete).  16-byte
// vectors, U per thread in flight (r0 is a multiple of 32): 4 in the
// standalone product, 1 inside the solvers, whose registers are taken.
template <typename V, int U = 4>
__device__ __forceinline__ void add_first_partials(const SymDev<V>& T, V* y, int64_t r0, int64_t r1) {
  using VT = typename Vec<V>::T;
  constexpr int W = Vec<V>::W;
  const int64_t g0 = r0 / W, g1 = r1 / W, bd = blockDim.x;
  const VT* __restrict__ pv = reinterpret_cast<const VT*>(T.p1);
  VT* __restrict__ yv = reinterpret_cast<VT*>(y);
  for (int64_t g = g0 + threadIdx.x; g < g1; g += U * bd) {
    VT a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (g + u * bd < g1) {
        a[u] = yv[g + u * bd];
        b[u] = pv[g + u * bd];
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (g + u * bd < g1) yv[g + u * bd] = vadd(a[u], b[u]);
  }
  for (int64_t i = g1 * W + threadIdx.x; i < r1; i += bd) y[i] += T.p1[i];
}

__device__ __forceinline__ void tile_pipe_init(TilePipe& tp, uint64_t* bars, long long limit_ns) {
  tp.bar = bars;
  tp.empty = bars + kMaxTileStages;
  tp.iss_par = tp.wait_par = tp.used = 0;
  tp.policy = policy_evict_first();
  tp.policy_x = policy_evict_normal();
  tp.limit_ns = limit_ns;
  tp.failed = false;
  if (threadIdx.x == 0)
    for (int b = 0; b < 2 * kMaxTileStages; ++b) mbar_init(&bars[b], 1);
  fence_mbar_init();
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
// f0(sum) runs on thread 0 before the broadcast: scalars derived from the sum
// (step lengths, square roots, tests) are formed once per CTA and published
// through shared memory, not by every thread on GB300's 1/64-rate FP64 pipe.
template <class F0>
__device__ __forceinline__ double grid_sum(const double* part, int G, double* red, F0&& f0) {
  if (threadIdx.x < 32) {
    // every load first (one round trip for G <= 256), then the additions in
    // the same order as one strided loop would make them
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = threadIdx.x + 32 * u;
      v[u] = i < G ? part[i] : 0.0;
    }
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (threadIdx.x + 32 * u < G) t += v[u];
    for (int i = threadIdx.x + 256; i < G; i += 32) t += part[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) {
      red[32] = t;
      f0(t);
    }
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}
__device__ __forceinline__ double grid_sum(const double* part, int G, double* red) {
  return grid_sum(part, G, red, [](double) {});
}

// (err points at GridBar::status; err[1] is GridBar::where, a code naming
// the wait that ran out.)

// Bounded grid barrier.  Returns false (uniformly within the CTA) when the
// wait ran out or another CTA already failed.
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned long long& target, long long timeout_ns,
                                             int* sflag, int where) {
  __syncthreads();  // the CTA's writes before thread 0's release
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int ok = 1;
    // arrival with release semantics (no separate fence, no returned value);
    // the acquire loads of the spin order everything after the barrier
    red_release_add(&gb->count, 1ull);
    const long long t0 = gtime();
    for (unsigned spins = 1;; ++spins) {
      if (ld_acquire(&gb->count) >= target) break;
      if ((spins & 63u) == 0) {
        if (ld_relaxed(&gb->status) != 0) { ok = 0; break; }
        if (gtime() - t0 > timeout_ns) {
          if (atomicCAS(&gb->status, 0, (int)kTimeout) == 0) gb->where = where;
          ok = 0;
          break;
        }
      }
    }
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

// -------------------------------------------------- one-shot kernels ---
// Shared-memory carving of the product kernels for layout mode FMT.
template <typename V, int FMT>
constexpr size_t product_smem() {
  return FMT == kGather ? pipe_smem_bytes<V>() : FMT == kTiles ? sym_smem_bytes<V>() : 0;
}

// Computes A x into y for the CTA's rows: complete for kGather / kPlan; for
// kTiles the CTA's own part, the window partial sums going to T.p1 (a row's
// first) and T.part (further ones), added by sym_incoming and
// add_first_partials after every CTA is done.
template <typename V, int FMT, bool NC>
__device__ __forceinline__ void product_rows(const OpDev<V>& A, const SymDev<V>& T, int64_t s0, int64_t s1,
                                             int64_t l0, int64_t l1, const V* x, V* y, unsigned char* smem,
                                             Pipe& pp, TilePipe& tp, int* err) {
  if constexpr (FMT == kTiles) {
    TileSmem<V>* sm = reinterpret_cast<TileSmem<V>*>(smem);
    sym_tiles<V, NC>(A, T, x, sm, tp, err, [&](int64_t row, V qo, V, V, V) { y[row] = qo; });
  } else {
    Stage<V>* stages = reinterpret_cast<Stage<V>*>(smem) + (threadIdx.x >> 5) * gather_stages<V>();
    spmv_rows<V, FMT == kPlan, NC>(A, s0, s1, l0, l1, x, stages, pp, err, [&](int64_t row, V v) { y[row] = v; });
  }
}

// y = A x on the persistent grid's partition (first pass for kTiles).
template <typename V, int FMT>
__global__ void __launch_bounds__(FMT == kTiles ? kTileThreads : kCgThreads, 1)
    k_rows(OpDev<V> A, SymDev<V> T, const int32_t* __restrict__ cta_slice, const int32_t* __restrict__ cta_long,
           const V* __restrict__ x, V* __restrict__ y, int* err, long long limit_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bars[kMaxThreads / 32][kMaxStages];
  __shared__ uint64_t tbar[2 * kMaxTileStages];
  Pipe pp;
  pipe_init(pp, bars[threadIdx.x >> 5], gather_stages<V>(), limit_ns);
  TilePipe tp;
  tile_pipe_init(tp, tbar, limit_ns);
  __syncthreads();
  const int c = blockIdx.x;
  product_rows<V, FMT, true>(A, T, cta_slice[c], cta_slice[c + 1], cta_long[c], cta_long[c + 1], x, y, smem_raw,
                             pp, tp, err);
}

// Second pass: for kTiles adds the partial sums (the listed ones, then the
// dense first ones); with MODE 1 then forms r = b - y in place (double
// precision) with per-CTA sums of r'r.
template <typename V, int FMT, int MODE>
__global__ void __launch_bounds__(kCgThreads, 1)
    k_finish(SymDev<V> T, const int32_t* __restrict__ cta_slice, int64_t n, const V* __restrict__ b,
             V* __restrict__ y, double* __restrict__ part) {
  __shared__ double red[33];
  const int c = blockIdx.x;
  const int64_t r0 = (int64_t)cta_slice[c] * 32;
  const int64_t r1 = (int64_t)cta_slice[c + 1] * 32 < n ? (int64_t)cta_slice[c + 1] * 32 : n;
  if constexpr (FMT == kTiles) {
    sym_incoming<V>(T, y);
    __syncthreads();
    if constexpr (MODE == 0) add_first_partials<V>(T, y, r0, r1);
  }
  if constexpr (MODE == 1) {
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      V yi = y[i];
      if constexpr (FMT == kTiles) yi += T.p1[i];
      const V t = b[i] - yi;
      y[i] = t;
      acc = fma((double)t, (double)t, acc);
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) part[c] = s;
  }
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

// Value update of a handle: slot i of a device value array takes input
// value map[i] (0 where map[i] < 0: padding), in double precision into d64
// and in single precision into d32 (either may be null).
__global__ void k_place_values(const int32_t* __restrict__ map, int64_t len, const double* __restrict__ src,
                               double* __restrict__ d64, float* __restrict__ d32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = map[i];
    const double v = k >= 0 ? src[k] : 0.0;
    if (d64) d64[i] = v;
    if (d32) d32[i] = (float)v;
  }
}

// x += a * double(d)
__global__ void k_axpy_f32(double a, const float* __restrict__ d, int64_t n, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, (double)d[i], x[i]);
}

// ------------------------------------------------- persistent solver ---
// Vector pass over rows [r0, r1) with 16-byte accesses.  ld(i) loads the
// group of W elements from i into a register tuple and st(i, tuple) finishes
// it; each thread keeps two groups in flight (both loaded before either is
// finished), or one with ONE.  The tail runs element-wise through f1(i).
template <typename V, bool ONE = false, class LD, class ST, class F1>
__device__ __forceinline__ void rows_vec(int64_t r0, int64_t r1, LD&& ld, ST&& st, F1&& f1) {
  constexpr int W = Vec<V>::W;
  const int64_t g0 = r0 / W, g1 = r1 / W;  // r0 is a multiple of 32
  const int64_t bd = blockDim.x;
  if constexpr (ONE) {
    for (int64_t g = g0 + threadIdx.x; g < g1; g += bd) st(g * W, ld(g * W));
  } else
  for (int64_t g = g0 + threadIdx.x; g < g1; g += 2 * bd) {
    const bool two = g + bd < g1;
    auto t0 = ld(g * W);
    decltype(t0) t1;
    if (two) t1 = ld((g + bd) * W);
    st(g * W, t0);
    if (two) st((g + bd) * W, t1);
  }
  for (int64_t i = g1 * W + threadIdx.x; i < r1; i += blockDim.x) f1(i);
}

template <typename VT>
struct Quad {
  VT a, b, c, d;
};

// ------------------------------------------------ streamed vector passes ---
// A vector pass of a tiled solver streams its input vectors through shared
// memory (the tile stages' space, idle between products): one thread issues
// bulk copies of 8 KB chunks of the arrays (2048 float or 1024 double rows),
// kVecBufs chunks ahead, so an SM keeps up to kVecBufs x NA x 8 KB of reads in
// flight without holding them in registers.  A register-pipelined pass (two
// 16-byte groups per thread and array) kept far less in flight and streamed
// the 256^3 system's vectors at about 4.8 TB/s.
constexpr int kVecChunkBytes = 8192;  // per array and chunk
constexpr int kVecBufs = 4;           // chunks in flight
template <typename V>
__host__ __device__ constexpr int vec_chunk() { return kVecChunkBytes / (int)sizeof(V); }
struct VecPipe {
  uint64_t* bar;  // one mbarrier per buffer (shared memory)
  uint32_t par;   // per buffer (bit b): parity of its next completion, kept alike by every thread
  uint64_t policy;
  long long limit_ns;
};
__device__ __forceinline__ void vec_pipe_init(VecPipe& vp, uint64_t* bars, long long limit_ns) {
  vp.bar = bars;
  vp.par = 0;
  vp.policy = policy_evict_normal();
  vp.limit_ns = limit_ns;
  if (threadIdx.x == 0)
    for (int b = 0; b < kVecBufs; ++b) mbar_init(&bars[b], 1);
  fence_mbar_init();
}
template <int NA>
__host__ __device__ constexpr size_t stream_smem_bytes() { return (size_t)kVecBufs * NA * kVecChunkBytes; }

// f(i, v) for every 16-byte group of W rows at row i of [r0, rv), rv = r0 +
// W floor((r1 - r0) / W), with v[k] = src[k][i .. i + W - 1] (r0 a multiple
// of 32, every src[k] 16-byte aligned); tail(i) for each row of [rv, r1).
// Every thread of the CTA calls it.  Returns false, with the timeout
// recorded in err, when a chunk did not land within the pipe's limit; the
// copies still in flight are waited for (bounded) first.
template <typename V, int NA, class F, class FT>
__device__ __forceinline__ bool stream_rows(const V* const (&src)[NA], int64_t r0, int64_t r1, V* buf, VecPipe& vp,
                                            int* err, F&& f, FT&& tail) {
  using VT = typename Vec<V>::T;
  constexpr int W = Vec<V>::W, kVecChunk = vec_chunk<V>();
  const int64_t rv = r0 + ((r1 - r0) & ~(int64_t)(W - 1));
  const int64_t nch = (rv - r0 + kVecChunk - 1) / kVecChunk;
  fence_proxy_async_shared();  // the buffers' earlier generic writes (tile accumulators) come first
  __syncthreads();
  auto issue = [&](int64_t j) {
    const int b = (int)(j % kVecBufs);
    const int64_t a = r0 + j * kVecChunk;
    const uint32_t bytes = (uint32_t)((rv - a < kVecChunk ? rv - a : kVecChunk) * (int64_t)sizeof(V));
    mbar_arrive_expect_tx(&vp.bar[b], (uint32_t)NA * bytes);
#pragma unroll
    for (int k = 0; k < NA; ++k) bulk_g2s(buf + (b * NA + k) * kVecChunk, src[k] + a, bytes, &vp.bar[b], vp.policy);
  };
  if (threadIdx.x == 0) {
    fence_proxy_async_global();  // the arrays were written by plain stores before the last grid barrier
    for (int64_t j = 0; j < nch && j < kVecBufs; ++j) issue(j);
  }
  bool ok = true;
  int64_t j = 0;
  for (; j < nch; ++j) {
    const int b = (int)(j % kVecBufs);
    ok = mbar_wait(&vp.bar[b], (vp.par >> b) & 1u, vp.limit_ns);
    if (ok) {
      const int64_t a = r0 + j * kVecChunk;
      const int groups = (int)(rv - a < kVecChunk ? rv - a : kVecChunk) / W;
      for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        VT v[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) v[k] = reinterpret_cast<const VT*>(buf + (b * NA + k) * kVecChunk)[g];
        f(a + W * (int64_t)g, v);
      }
    }
    ok = __syncthreads_and(ok);  // buffer b is free on every thread, or some wait ran out
    if (!ok) break;
    vp.par ^= 1u << b;
    if (threadIdx.x == 0 && j + kVecBufs < nch) issue(j + kVecBufs);
  }
  if (!ok) {
    // chunks j .. min(j + kVecBufs, nch) - 1 were issued: wait (bounded) for
    // them to land before anything else uses the buffers
    if (threadIdx.x == 0) {
      if (atomicCAS(err, 0, (int)kTimeout) == 0) err[1] = 500000000 + (int)(j % 1000000);
      for (int64_t i = j; i < nch && i < j + kVecBufs; ++i) {
        const int b = (int)(i % kVecBufs);
        mbar_wait(&vp.bar[b], (vp.par >> b) & 1u, vp.limit_ns);
        vp.par ^= 1u << b;
      }
    }
    return false;
  }
  for (int64_t i = rv + threadIdx.x; i < r1; i += blockDim.x) tail(i);
  return true;
}

// OUTER = false: inner single-precision solve from x = 0 (rhs in b), no
// true-residual confirmation.  OUTER = true: the full solve of Section III
// from the caller's x0 with the confirm/restart step.
template <typename V, int FMT, bool OUTER>
__global__ void __launch_bounds__(FMT == kTiles ? kTileThreads : kCgThreads, 1) k_cg(CgArgs<V> a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bars[kMaxThreads / 32][kMaxStages];
  __shared__ double red[33];
  __shared__ int sflag;
  __shared__ struct {
    double alpha, beta;
    int code, nonfinite, conv;
  } sc;  // the step's scalars, formed by thread 0 (grid_sum's epilogue)
  using VT = typename Vec<V>::T;
  constexpr int W = Vec<V>::W;
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t s0 = a.cta_slice[c], s1 = a.cta_slice[c + 1];
  const int64_t l0 = a.cta_long[c], l1 = a.cta_long[c + 1];
  const int64_t r0 = s0 * 32;
  const int64_t r1 = s1 * 32 < a.A.n ? s1 * 32 : a.A.n;
  const OpDev<V>& A = a.A;
  const SymDev<V>& T = a.T;
  V* __restrict__ x = a.x;
  V* __restrict__ r = a.r;
  V* __restrict__ p = a.p;
  V* __restrict__ q = a.q;
  const V* __restrict__ b = a.b;
  double* part0 = a.part;
  double* part1 = a.part + G;
  __shared__ uint64_t tbar[2 * kMaxTileStages];
  Pipe pp;
  pipe_init(pp, bars[threadIdx.x >> 5], gather_stages<V>(), a.timeout_ns);
  TilePipe tp;
  tile_pipe_init(tp, tbar, a.timeout_ns);
  __shared__ uint64_t vbar[kVecBufs];
  VecPipe vp;
  if constexpr (FMT == kTiles) vec_pipe_init(vp, vbar, a.timeout_ns);
  static_assert(FMT != kTiles || stream_smem_bytes<5>() <= sizeof(TileSmem<V>), "vector stream buffers");
  __syncthreads();
  int* err = &a.bar->status;
  unsigned long long target = 0;
  int nbar = 0;
  int status = kOk;
  int k = 0, restarts = 0;
  double rr = 0.0, nb = 0.0, rel_true = 0.0;
  bool conv = false;

  // q = A xin over the CTA's rows, complete (kTiles: across a grid barrier)
  auto full_product = [&](const V* xin) -> bool {
    product_rows<V, FMT, false>(A, T, s0, s1, l0, l1, xin, q, smem_raw, pp, tp, err);
    if constexpr (FMT == kTiles) {
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return false;
      sym_incoming<V>(T, q);
      __syncthreads();
      add_first_partials<V, 1>(T, q, r0, r1);
    }
    __syncthreads();
    return true;
  };

  // init: r = b - A x0, p = r, r'r and b'b
  {
    V pr = V(0), pb = V(0);
    if constexpr (OUTER) {
      if (!full_product(x)) return;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const V bi = b[i];
        const V t = bi - q[i];
        r[i] = t;
        p[i] = t;
        pr = fma_(t, t, pr);
        pb = fma_(bi, bi, pb);
      }
    } else {
      rows_vec<V>(
          r0, r1, [&](int64_t i) { return *reinterpret_cast<const VT*>(b + i); },
          [&](int64_t i, VT bv) {
            *reinterpret_cast<VT*>(x + i) = VT{};
            *reinterpret_cast<VT*>(r + i) = bv;
            *reinterpret_cast<VT*>(p + i) = bv;
            const V* e = reinterpret_cast<const V*>(&bv);
#pragma unroll
            for (int j = 0; j < W; ++j) pr = fma_(e[j], e[j], pr);
          },
          [&](int64_t i) {
            const V bi = b[i];
            x[i] = V(0);
            r[i] = bi;
            p[i] = bi;
            pr = fma_(bi, bi, pr);
          });
      pb = pr;
    }
    // r'r and b'b go to the third and fourth partial-sum slots: the first
    // iteration writes p'q to part0 (and r'r to part1) with no barrier after
    // these sums, while a slower CTA may still be adding them up
    double* part2 = a.part + 2 * G;
    double* part3 = a.part + 3 * G;
    const double s_rr = block_sum((double)pr, red);
    if (threadIdx.x == 0) part2[c] = s_rr;
    const double s_bb = block_sum((double)pb, red);
    if (threadIdx.x == 0) part3[c] = s_bb;
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    rr = grid_sum(part2, G, red);
    nb = sqrt(grid_sum(part3, G, red));
  }
  if (nb == 0.0) {  // b = 0: x = 0
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[i] = V(0);
    rr = 0.0;
    goto finish;
  }
  conv = sqrt(rr) / nb <= a.tol;
  for (;;) {
    while (k < a.maxit && !conv) {
      // A: q = A p, p'q
      V ppq = V(0);
      if constexpr (FMT == kTiles) {
        // p'Ap = p'Dp + 2 p'Up from the rows' own parts: no incoming sums needed
        TileSmem<V>* sm = reinterpret_cast<TileSmem<V>*>(smem_raw);
        sym_tiles<V, false>(A, T, p, sm, tp, err, [&](int64_t row, V qo, V xi, V dxi, V direct) {
          q[row] = qo;
          ppq = fma_(xi, fma_(V(2), direct, dxi), ppq);
        });
      } else {
        Stage<V>* stages = reinterpret_cast<Stage<V>*>(smem_raw) + (threadIdx.x >> 5) * gather_stages<V>();
        spmv_rows<V, FMT == kPlan, false>(A, s0, s1, l0, l1, p, stages, pp, err, [&](int64_t row, V v, V pr) {
          q[row] = v;
          ppq = fma_(pr, v, ppq);
        });
      }
      {
        const double s = block_sum((double)ppq, red);
        if (threadIdx.x == 0) part0[c] = s;
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
      grid_sum(part0, G, red, [&](double pq) {
        sc.code = !isfinite(pq) ? kNonfinite : !(pq > 0.0) ? kNotSpd : kOk;
        sc.alpha = rr / pq;
      });
      if (sc.code != kOk) { status = sc.code; goto finish; }
      const double alpha = sc.alpha;
      if constexpr (FMT == kTiles) {
        sym_incoming<V>(T, q);
        __syncthreads();
      }
      // B: x += alpha p, r -= alpha q, r'r
      {
        const V al = (V)alpha;
        V prr = V(0);
        bool streamed = false;
        if constexpr (FMT == kTiles) {
          // vectors larger than the L2: p, q, the first partials, x and r
          // stream through shared memory (the same rows per thread, in the
          // same order, as the register-pipelined pass below)
          if (a.stream_vec) {
            const V* const src[5] = {p, q, T.p1, x, r};
            const bool ok = stream_rows<V, 5>(
                src, r0, r1, reinterpret_cast<V*>(smem_raw), vp, err,
                [&](int64_t i, const VT (&v)[5]) {
                  const V* pe = reinterpret_cast<const V*>(&v[0]);
                  const V* qe = reinterpret_cast<const V*>(&v[1]);
                  const V* fe = reinterpret_cast<const V*>(&v[2]);
                  const V* xe = reinterpret_cast<const V*>(&v[3]);
                  const V* re = reinterpret_cast<const V*>(&v[4]);
                  VT xn, rn;
                  V* xo = reinterpret_cast<V*>(&xn);
                  V* ro = reinterpret_cast<V*>(&rn);
#pragma unroll
                  for (int j = 0; j < W; ++j) {
                    xo[j] = fma_(al, pe[j], xe[j]);
                    ro[j] = fma_(-al, qe[j] + fe[j], re[j]);
                    prr = fma_(ro[j], ro[j], prr);
                  }
                  *reinterpret_cast<VT*>(x + i) = xn;
                  *reinterpret_cast<VT*>(r + i) = rn;
                },
                [&](int64_t i) {
                  x[i] = fma_(al, p[i], x[i]);
                  const V ri = fma_(-al, q[i] + T.p1[i], r[i]);
                  r[i] = ri;
                  prr = fma_(ri, ri, prr);
                });
            if (!ok) return;
            streamed = true;
          }
        }
        // (one 16-byte group per thread at a time in the double-precision
        // tiled solve, whose registers are otherwise taken)
        if (!streamed)
        rows_vec<V, FMT == kTiles && OUTER && sizeof(V) == 8>(
            r0, r1,
            [&](int64_t i) {
              VT qv = *reinterpret_cast<const VT*>(q + i);
              if constexpr (FMT == kTiles) qv = vadd(qv, *reinterpret_cast<const VT*>(T.p1 + i));
              return Quad<VT>{*reinterpret_cast<const VT*>(p + i), qv, *reinterpret_cast<const VT*>(x + i),
                              *reinterpret_cast<const VT*>(r + i)};
            },
            [&](int64_t i, Quad<VT> t) {
              const V* pe = reinterpret_cast<const V*>(&t.a);
              const V* qe = reinterpret_cast<const V*>(&t.b);
              V* xe = reinterpret_cast<V*>(&t.c);
              V* re = reinterpret_cast<V*>(&t.d);
#pragma unroll
              for (int j = 0; j < W; ++j) {
                xe[j] = fma_(al, pe[j], xe[j]);
                re[j] = fma_(-al, qe[j], re[j]);
                prr = fma_(re[j], re[j], prr);
              }
              *reinterpret_cast<VT*>(x + i) = t.c;
              *reinterpret_cast<VT*>(r + i) = t.d;
            },
            [&](int64_t i) {
              x[i] = fma_(al, p[i], x[i]);
              V qi = q[i];
              if constexpr (FMT == kTiles) qi += T.p1[i];
              const V ri = fma_(-al, qi, r[i]);
              r[i] = ri;
              prr = fma_(ri, ri, prr);
            });
        const double s = block_sum((double)prr, red);
        if (threadIdx.x == 0) part1[c] = s;
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
      const double rr_new = grid_sum(part1, G, red, [&](double s) {
        sc.nonfinite = !isfinite(s);
        sc.beta = s / rr;
        sc.conv = sqrt(s) / nb <= a.tol;
      });
      ++k;
      if (sc.nonfinite) { status = kNonfinite; rr = rr_new; goto finish; }
      const double beta = sc.beta;
      rr = rr_new;
      conv = sc.conv;
      if (conv) break;
      // C: p = r + beta p
      {
        const V be = (V)beta;
        bool streamed = false;
        if constexpr (FMT == kTiles) {
          if (a.stream_vec) {
            const V* const src[2] = {p, r};
            const bool ok = stream_rows<V, 2>(
                src, r0, r1, reinterpret_cast<V*>(smem_raw), vp, err,
                [&](int64_t i, const VT (&v)[2]) {
                  const V* pe = reinterpret_cast<const V*>(&v[0]);
                  const V* re = reinterpret_cast<const V*>(&v[1]);
                  VT pn;
                  V* po = reinterpret_cast<V*>(&pn);
#pragma unroll
                  for (int j = 0; j < W; ++j) po[j] = fma_(be, pe[j], re[j]);
                  *reinterpret_cast<VT*>(p + i) = pn;
                },
                [&](int64_t i) { p[i] = fma_(be, p[i], r[i]); });
            if (!ok) return;
            streamed = true;
          }
        }
        if (!streamed)
        rows_vec<V>(
            r0, r1,
            [&](int64_t i) {
              return Quad<VT>{*reinterpret_cast<const VT*>(p + i), *reinterpret_cast<const VT*>(r + i), VT{}, VT{}};
            },
            [&](int64_t i, Quad<VT> t) {
              V* pe = reinterpret_cast<V*>(&t.a);
              const V* re = reinterpret_cast<const V*>(&t.b);
#pragma unroll
              for (int j = 0; j < W; ++j) pe[j] = fma_(be, pe[j], re[j]);
              *reinterpret_cast<VT*>(p + i) = t.a;
            },
            [&](int64_t i) { p[i] = fma_(be, p[i], r[i]); });
      }
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    }
    if constexpr (!OUTER) {
      if (!conv) status = kMaxit;
      break;
    } else {
      // confirm on the true residual; restart the recurrence from it otherwise
      if (!full_product(x)) return;
      V ptt = V(0);
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const V t = b[i] - q[i];
        r[i] = t;
        ptt = fma_(t, t, ptt);
      }
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
      conv = sqrt(rr) / nb <= a.tol;
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

// Extra vectors of the single-reduction CG: s = A p, z = A s, and w = A r
// double-buffered (the product of an iteration reads one buffer while the
// update writes the other).
template <typename V>
struct PcgArgs {
  CgArgs<V> c;
  V* s;
  V* z;
  V* w0;
  V* w1;
};

// Single-reduction ("pipelined") CG: the Chronopoulos-Gear recurrences of the
// Section III iteration in the Ghysels-Vanroose arrangement.  Each iteration
// is ONE pass over the CTA's rows -- the product q = A w fused, row by row,
// with z = q + beta z, s = w + beta s, p = r + beta p, x += alpha p,
// r -= alpha s, w' = w - alpha z and the partial sums of r'r and w'r -- and
// ONE grid barrier, after which every CTA forms alpha and beta from the same
// sums in the same order.  (k_cg needs three barriers per iteration.)  The
// partial sums alternate between two halves of the partial-sum array, so a
// CTA never overwrites sums another CTA may still be reading.  The full
// solve from x0 with true-residual confirmation and restarts (from
// r = b - A x), in double precision: in single precision the recurrences
// drift past any useful inner tolerance.  p'Ap comes from the
// recurrence delta - beta gamma / alpha_old, which cancels near the
// attainable residual: a non-positive value after the first step of a run
// ends the run into the confirmation instead of reporting NOT_SPD.
// Row-gather layouts only (kGather, kPlan): their product needs no barrier
// of its own.
template <typename V, int FMT>
__global__ void __launch_bounds__(kCgThreads, 1) k_pcg(PcgArgs<V> pa) {
  static_assert(FMT != kTiles, "the tiled symmetric product needs a barrier of its own");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bars[kMaxThreads / 32][kMaxStages];
  __shared__ double red[33];
  __shared__ struct {
    double alpha, beta;
    int code;
  } sc;
  __shared__ int sflag;
  const CgArgs<V>& a = pa.c;
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
  V* __restrict__ sv = pa.s;
  V* __restrict__ zv = pa.z;
  V* wb[2] = {pa.w0, pa.w1};
  const V* __restrict__ b = a.b;
  Pipe pp;
  pipe_init(pp, bars[threadIdx.x >> 5], gather_stages<V>(), a.timeout_ns);
  __syncthreads();
  int* err = &a.bar->status;
  Stage<V>* stages = reinterpret_cast<Stage<V>*>(smem_raw) + (threadIdx.x >> 5) * gather_stages<V>();
  unsigned long long target = 0;
  int nbar = 0, status = kOk, k = 0, restarts = 0, par = 0, cur = 0;
  double gamma = 0.0, delta = 0.0, nb = 0.0, rel_true = 0.0;
  // partial-sum half `h`: sums j = 0, 1 (and 2 for b'b) of every CTA
  auto slot = [&](int h, int j) { return a.part + (int64_t)(3 * h + j) * G; };
  auto publish = [&](int h, double v0, double v1, double v2) -> bool {
    const double s_0 = block_sum(v0, red);
    if (threadIdx.x == 0) slot(h, 0)[c] = s_0;
    const double s_1 = block_sum(v1, red);
    if (threadIdx.x == 0) slot(h, 1)[c] = s_1;
    const double s_2 = block_sum(v2, red);
    if (threadIdx.x == 0) slot(h, 2)[c] = s_2;
    return grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++);
  };
  for (bool first_run = true;; first_run = false) {
    // r = b - A x; then w = A r with r'r, w'r (and b'b)
    spmv_rows<V, FMT == kPlan, false>(A, s0, s1, l0, l1, x, stages, pp, err, [&](int64_t row, V v) { q[row] = v; });
    __syncthreads();
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) r[i] = b[i] - q[i];
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    {
      V pg = V(0), pd = V(0), pb = V(0);
      V* __restrict__ w = wb[cur];
      spmv_rows<V, FMT == kPlan, false>(A, s0, s1, l0, l1, r, stages, pp, err, [&](int64_t row, V v) {
        w[row] = v;
        const V ri = r[row];
        pg = fma_(ri, ri, pg);
        pd = fma_(v, ri, pd);
      });
      if (first_run)
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) pb = fma_(b[i], b[i], pb);
      if (!publish(par, (double)pg, (double)pd, (double)pb)) return;
      gamma = grid_sum(slot(par, 0), G, red);
      delta = grid_sum(slot(par, 1), G, red);
      if (first_run) nb = sqrt(grid_sum(slot(par, 2), G, red));
      par ^= 1;
    }
    if (nb == 0.0) {  // b = 0: x = 0
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[i] = V(0);
      gamma = 0.0;
      goto finish;
    }
    {
      double gamma_old = 0.0, alpha_old = 0.0;
      bool first = true;
      for (;;) {
        // the step's scalars once per CTA (thread 0), not by every thread on
        // the 1/64-rate FP64 pipe: 0 step, 1 not finite, 2 leave the run, 3 not SPD
        if (threadIdx.x == 0) {
          int code = 0;
          double al0 = 0.0, be0 = 0.0;
          if (!isfinite(gamma) || !isfinite(delta)) {
            code = 1;
          } else if (sqrt(gamma) / nb <= a.tol || k >= a.maxit) {
            code = 2;
          } else {
            be0 = first ? 0.0 : gamma / gamma_old;
            const double den = first ? delta : delta - be0 * gamma / alpha_old;  // p'Ap
            if (!isfinite(den)) code = 1;
            // first step: den = r'Ar, A is not positive definite; later the
            // recurrence for p'Ap has cancelled (near the attainable residual):
            // confirm and restart from the true residual
            else if (!(den > 0.0)) code = first ? 3 : 2;
            else al0 = gamma / den;
          }
          sc.code = code;
          sc.alpha = al0;
          sc.beta = be0;
        }
        __syncthreads();
        if (sc.code == 1) { status = kNonfinite; goto finish; }
        if (sc.code == 3) { status = kNotSpd; goto finish; }
        if (sc.code == 2) break;
        const double beta = sc.beta;
        const double alpha = sc.alpha;
        const V al = (V)alpha, be = (V)beta;
        const V* __restrict__ w = wb[cur];
        V* __restrict__ wn = wb[cur ^ 1];
        V pg = V(0), pd = V(0);
        spmv_rows<V, FMT == kPlan, false>(A, s0, s1, l0, l1, w, stages, pp, err, [&](int64_t row, V qv, V wi) {
          const V ri = r[row];
          const V zi = first ? qv : fma_(be, zv[row], qv);
          const V si = first ? wi : fma_(be, sv[row], wi);
          const V pi = first ? ri : fma_(be, p[row], ri);
          zv[row] = zi;
          sv[row] = si;
          p[row] = pi;
          x[row] = fma_(al, pi, x[row]);
          const V rn = fma_(-al, si, ri);
          const V wnv = fma_(-al, zi, wi);
          r[row] = rn;
          wn[row] = wnv;
          pg = fma_(rn, rn, pg);
          pd = fma_(wnv, rn, pd);
        });
        if (!publish(par, (double)pg, (double)pd, 0.0)) return;
        gamma_old = gamma;
        alpha_old = alpha;
        gamma = grid_sum(slot(par, 0), G, red);
        delta = grid_sum(slot(par, 1), G, red);
        par ^= 1;
        cur ^= 1;
        ++k;
        first = false;
      }
    }
    {
      // confirm on the true residual; restart the recurrences from it otherwise
      spmv_rows<V, FMT == kPlan, false>(A, s0, s1, l0, l1, x, stages, pp, err, [&](int64_t row, V v) { q[row] = v; });
      __syncthreads();
      V ptt = V(0);
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const V t = b[i] - q[i];
        ptt = fma_(t, t, ptt);
      }
      if (!publish(par, (double)ptt, 0.0, 0.0)) return;
      const double tt = grid_sum(slot(par, 0), G, red);
      par ^= 1;
      rel_true = sqrt(tt) / nb;
      if (!isfinite(tt)) { status = kNonfinite; break; }
      if (rel_true <= a.tol) break;
      if (k >= a.maxit || restarts >= a.max_restarts) { status = kMaxit; break; }
      ++restarts;
    }
  }
finish:
  if (c == 0 && threadIdx.x == 0) {
    a.st->rr = gamma;
    a.st->nb = nb;
    a.st->rel_true = rel_true;
    a.st->k = k;
    a.st->restarts = restarts;
    a.st->status = status;
  }
}

// Mixed precision with reliable updates.  Single-precision CG iterations on
// A32 (the three phases of k_cg's inner solve) build a correction d; when the
// recurrence residual has fallen by the factor delta since the last update,
// or reaches tol, or the iteration bound is met, the correction is added to
// the double-precision x (x += d, d = 0) and the single-precision residual is
// replaced by the double-precision b - A x, formed by the double-precision
// product in the same launch.  The search direction is kept: the Krylov space
// is not restarted.  Converged when an update's true residual is <= tol ||b||.
struct RuArgs {
  CgArgs<float> c;        // float operator; x = correction d, r, p, q
  OpDev<double> A64;      // the same layout with double values
  SymDev<double> T64;     // and its tiles (kTiles)
  double* x64;            // caller's x (in: x0)
  const double* b64;
  double* q64;            // double product scratch
  double delta;
};

// Bytes of one warp's share of the stage buffers, used in turn by the
// single-precision and the double-precision product.
__host__ __device__ constexpr size_t ru_warp_stage_bytes() {
  return gather_stages<float>() * sizeof(Stage<float>) > gather_stages<double>() * sizeof(Stage<double>)
             ? gather_stages<float>() * sizeof(Stage<float>)
             : gather_stages<double>() * sizeof(Stage<double>);
}

// Tiled symmetric layout: the single- and double-precision products share
// the tile pipeline and its shared memory (TileSmem<double> over
// TileSmem<float>); each product drains its fills and grid barriers separate
// them, so no fill of one lands in a stage the other is reading.
template <int FMT>
__global__ void __launch_bounds__(FMT == kTiles ? kTileThreads : kCgThreads, 1) k_cg_ru(RuArgs ra) {
  static_assert(gather_stages<float>() + gather_stages<double>() <= kMaxStages, "mbarrier sets");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bars[kMaxThreads / 32][kMaxStages];
  __shared__ double red[33];
  __shared__ int sflag;
  __shared__ struct {
    float al, be;
    int code, upd;
  } sc;  // the step's scalars, formed by thread 0 (grid_sum's epilogue)
  const CgArgs<float>& a = ra.c;
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t s0 = a.cta_slice[c], s1 = a.cta_slice[c + 1];
  const int64_t l0 = a.cta_long[c], l1 = a.cta_long[c + 1];
  const int64_t r0 = s0 * 32;
  const int64_t r1 = s1 * 32 < a.A.n ? s1 * 32 : a.A.n;
  float* __restrict__ d = a.x;
  float* __restrict__ r = a.r;
  float* __restrict__ p = a.p;
  float* __restrict__ q = a.q;
  double* __restrict__ x64 = ra.x64;
  const double* __restrict__ b64 = ra.b64;
  double* __restrict__ q64 = ra.q64;
  const int warp = threadIdx.x >> 5;
  unsigned char* wst = smem_raw + (size_t)warp * ru_warp_stage_bytes();
  Stage<float>* st32 = reinterpret_cast<Stage<float>*>(wst);
  Stage<double>* st64 = reinterpret_cast<Stage<double>*>(wst);
  Pipe pp32, pp64;
  pipe_init(pp32, bars[warp], gather_stages<float>(), a.timeout_ns);
  pipe_init(pp64, bars[warp] + gather_stages<float>(), gather_stages<double>(), a.timeout_ns);
  __shared__ uint64_t tbar[2 * kMaxTileStages];
  TilePipe tp;
  if constexpr (FMT == kTiles) tile_pipe_init(tp, tbar, a.timeout_ns);
  __shared__ uint64_t vbar[kVecBufs];
  VecPipe vp;
  if constexpr (FMT == kTiles) vec_pipe_init(vp, vbar, a.timeout_ns);
  static_assert(stream_smem_bytes<5>() <= sizeof(TileSmem<float>), "vector stream buffers");
  __syncthreads();
  int* err = &a.bar->status;
  double* part0 = a.part;
  double* part1 = a.part + G;
  double* part2 = a.part + 2 * G;
  unsigned long long target = 0;
  int nbar = 0, status = kOk, k = 0, updates = 0;
  double rr = 0.0, nb = 0.0, rel = 0.0, rmax = 0.0;
  bool first_update = true;

  // x += d, d = 0; r = float(b - A64 x); rr = r'r; rel = ||b - A x|| / ||b||
  auto update = [&]() -> bool {
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      x64[i] += (double)d[i];
      d[i] = 0.f;
    }
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return false;
    if constexpr (FMT == kTiles) {
      TileSmem<double>* sm = reinterpret_cast<TileSmem<double>*>(smem_raw);
      sym_tiles<double, false>(ra.A64, ra.T64, x64, sm, tp, err,
                               [&](int64_t row, double qo, double, double, double) { q64[row] = qo; });
      if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return false;
      sym_incoming<double>(ra.T64, q64);
    } else {
      spmv_rows<double, FMT == kPlan, false>(ra.A64, s0, s1, l0, l1, x64, st64, pp64, err,
                                             [&](int64_t row, double v) { q64[row] = v; });
    }
    __syncthreads();
    double ptt = 0.0, pbb = 0.0;
    float prr = 0.f;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double bi = b64[i];
      double qi = q64[i];
      if constexpr (FMT == kTiles) qi += ra.T64.p1[i];
      const double t = bi - qi;
      const float tf = (float)t;
      r[i] = tf;
      ptt = fma(t, t, ptt);
      prr = fmaf(tf, tf, prr);
      if (first_update) pbb = fma(bi, bi, pbb);
    }
    const double s_tt = block_sum(ptt, red);
    if (threadIdx.x == 0) part0[c] = s_tt;
    const double s_rr = block_sum((double)prr, red);
    if (threadIdx.x == 0) part1[c] = s_rr;
    if (first_update) {
      const double s_bb = block_sum(pbb, red);
      if (threadIdx.x == 0) part2[c] = s_bb;
    }
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return false;
    const double tt = grid_sum(part0, G, red);
    rr = grid_sum(part1, G, red);
    if (first_update) nb = sqrt(grid_sum(part2, G, red));
    first_update = false;
    rel = nb > 0.0 ? sqrt(tt) / nb : 0.0;
    rmax = sqrt(rr);
    return true;
  };

  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) d[i] = 0.f;
  if (!update()) return;
  if (nb == 0.0) {  // b = 0: x = 0
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x64[i] = 0.0;
    rel = 0.0;
    goto finish;
  }
  if (!isfinite(rel)) { status = kNonfinite; goto finish; }
  if (rel <= a.tol) goto finish;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) p[i] = r[i];
  if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
  status = kMaxit;
  while (k < a.maxit) {
    // A: q = A32 p, p'q
    {
      float ppq = 0.f;
      if constexpr (FMT == kTiles) {
        // p'Ap = p'Dp + 2 p'Up from the rows' own parts: no incoming sums needed
        TileSmem<float>* sm = reinterpret_cast<TileSmem<float>*>(smem_raw);
        sym_tiles<float, false>(a.A, a.T, p, sm, tp, err, [&](int64_t row, float qo, float xi, float dxi, float direct) {
          q[row] = qo;
          ppq = fmaf(xi, fmaf(2.f, direct, dxi), ppq);
        });
      } else {
        spmv_rows<float, FMT == kPlan, false>(a.A, s0, s1, l0, l1, p, st32, pp32, err,
                                              [&](int64_t row, float v, float pr) {
                                                q[row] = v;
                                                ppq = fmaf(pr, v, ppq);
                                              });
      }
      const double sp = block_sum((double)ppq, red);
      if (threadIdx.x == 0) part0[c] = sp;
    }
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    grid_sum(part0, G, red, [&](double pq) {
      sc.code = !isfinite(pq) ? kNonfinite : !(pq > 0.0) ? kNotSpd : kOk;
      sc.al = (float)(rr / pq);
    });
    if (sc.code != kOk) { status = sc.code; break; }
    const float al = sc.al;
    if constexpr (FMT == kTiles) {  // the transpose parts other CTAs computed for these rows
      sym_incoming<float>(a.T, q);
      __syncthreads();
    }
    // B: d += alpha p, r -= alpha q, r'r  (16-byte accesses, as k_cg; on the
    // tiled layout q_i = own part + first partial, and when the vectors
    // outgrow the L2, p, q, the first partials, d and r stream through
    // shared memory)
    if (FMT == kTiles && ra.c.stream_vec) {
      float prr = 0.f;
      const float* const src[5] = {p, q, a.T.p1, d, r};
      const bool ok = stream_rows<float, 5>(
          src, r0, r1, reinterpret_cast<float*>(smem_raw), vp, err,
          [&](int64_t i, const float4 (&v)[5]) {
            const float* pe = reinterpret_cast<const float*>(&v[0]);
            const float* qe = reinterpret_cast<const float*>(&v[1]);
            const float* fe = reinterpret_cast<const float*>(&v[2]);
            const float* de = reinterpret_cast<const float*>(&v[3]);
            const float* re = reinterpret_cast<const float*>(&v[4]);
            float4 dn, rn;
            float* dno = reinterpret_cast<float*>(&dn);
            float* rno = reinterpret_cast<float*>(&rn);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              dno[j] = fmaf(al, pe[j], de[j]);
              rno[j] = fmaf(-al, qe[j] + fe[j], re[j]);
              prr = fmaf(rno[j], rno[j], prr);
            }
            *reinterpret_cast<float4*>(d + i) = dn;
            *reinterpret_cast<float4*>(r + i) = rn;
          },
          [&](int64_t i) {
            d[i] = fmaf(al, p[i], d[i]);
            const float ri = fmaf(-al, q[i] + a.T.p1[i], r[i]);
            r[i] = ri;
            prr = fmaf(ri, ri, prr);
          });
      if (!ok) return;
      const double sr = block_sum((double)prr, red);
      if (threadIdx.x == 0) part1[c] = sr;
    } else {
      float prr = 0.f;
      rows_vec<float>(
          r0, r1,
          [&](int64_t i) {
            float4 qv = *reinterpret_cast<const float4*>(q + i);
            if constexpr (FMT == kTiles) qv = vadd(qv, *reinterpret_cast<const float4*>(a.T.p1 + i));
            return Quad<float4>{*reinterpret_cast<const float4*>(p + i), qv, *reinterpret_cast<const float4*>(d + i),
                                *reinterpret_cast<const float4*>(r + i)};
          },
          [&](int64_t i, Quad<float4> t) {
            const float* pe = reinterpret_cast<const float*>(&t.a);
            const float* qe = reinterpret_cast<const float*>(&t.b);
            float* de = reinterpret_cast<float*>(&t.c);
            float* re = reinterpret_cast<float*>(&t.d);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              de[j] = fmaf(al, pe[j], de[j]);
              re[j] = fmaf(-al, qe[j], re[j]);
              prr = fmaf(re[j], re[j], prr);
            }
            *reinterpret_cast<float4*>(d + i) = t.c;
            *reinterpret_cast<float4*>(r + i) = t.d;
          },
          [&](int64_t i) {
            d[i] = fmaf(al, p[i], d[i]);
            float qi = q[i];
            if constexpr (FMT == kTiles) qi += a.T.p1[i];
            const float ri = fmaf(-al, qi, r[i]);
            r[i] = ri;
            prr = fmaf(ri, ri, prr);
          });
      const double sr = block_sum((double)prr, red);
      if (threadIdx.x == 0) part1[c] = sr;
    }
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
    // 0: iterate; 1: update first (the recurrence residual fell by delta,
    // reached tol, or the iteration bound is met); 2: not finite
    double rr_new = grid_sum(part1, G, red, [&](double s) {
      sc.upd = !isfinite(s) ? 2 : (sqrt(s) < ra.delta * rmax || sqrt(s) <= a.tol * nb || k + 1 >= a.maxit) ? 1 : 0;
      sc.be = (float)(s / rr);
    });
    ++k;
    if (sc.upd == 2) { status = kNonfinite; break; }
    float be = sc.be;
    if (sc.upd == 1) {
      const double rr_keep = rr;
      if (!update()) return;
      ++updates;
      if (!isfinite(rel)) { status = kNonfinite; goto finish; }
      if (rel <= a.tol) { status = kOk; goto finish; }
      if (k >= a.maxit) { status = kMaxit; goto finish; }
      rr_new = rr;  // the replaced residual's r'r (update() set rr and rmax)
      rr = rr_keep;
      be = (float)(rr_new / rr);
    }
    rr = rr_new;
    // C: p = r + beta p
    if (FMT == kTiles && ra.c.stream_vec) {
      const float* const src[2] = {p, r};
      const bool ok = stream_rows<float, 2>(
          src, r0, r1, reinterpret_cast<float*>(smem_raw), vp, err,
          [&](int64_t i, const float4 (&v)[2]) {
            const float* pe = reinterpret_cast<const float*>(&v[0]);
            const float* re = reinterpret_cast<const float*>(&v[1]);
            float4 pn;
            float* pno = reinterpret_cast<float*>(&pn);
#pragma unroll
            for (int j = 0; j < 4; ++j) pno[j] = fmaf(be, pe[j], re[j]);
            *reinterpret_cast<float4*>(p + i) = pn;
          },
          [&](int64_t i) { p[i] = fmaf(be, p[i], r[i]); });
      if (!ok) return;
    } else {
      rows_vec<float>(
          r0, r1,
          [&](int64_t i) {
            return Quad<float4>{*reinterpret_cast<const float4*>(p + i), *reinterpret_cast<const float4*>(r + i),
                                float4{}, float4{}};
          },
          [&](int64_t i, Quad<float4> t) {
            float* pe = reinterpret_cast<float*>(&t.a);
            const float* re = reinterpret_cast<const float*>(&t.b);
#pragma unroll
            for (int j = 0; j < 4; ++j) pe[j] = fmaf(be, pe[j], re[j]);
            *reinterpret_cast<float4*>(p + i) = t.a;
          },
          [&](int64_t i) { p[i] = fmaf(be, p[i], r[i]); });
    }
    if (!grid_barrier(a.bar, target, a.timeout_ns, &sflag, nbar++)) return;
  }
  // left by a breakdown: keep the last correction
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x64[i] += (double)d[i];
finish:
  if (c == 0 && threadIdx.x == 0) {
    a.st->rr = rr;
    a.st->nb = nb;
    a.st->rel_true = rel;
    a.st->k = k;
    a.st->restarts = updates;
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
