// gbcg.cu -- C ABI of the GB300 conjugate-gradient library (include/gbcg.h).
//
// Host driver: validates and lays out the matrix (layout.cpp), owns the
// device copies and the solve workspace, and launches the kernels of
// kernels.cuh.  Nothing here computes on the host: every step of a product
// or a solve runs in the library's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gbcg.h"
#include "kernels.cuh"
#include "layout.h"

using namespace gbcg;

static_assert(kTilePad == kPadSlot, "the layout's padding flag is the kernels'");
static_assert(TileCaps<float>::kSlot < kPadSlot && TileCaps<double>::kSlot < kPadSlot,
              "slot numbers stay below the padding flag");

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(...)                                                                               \
  do {                                                                                              \
    cudaError_t e_ = (__VA_ARGS__);                                                                     \
    if (e_ != cudaSuccess)                                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? GBCG_ERR_NOMEM : GBCG_ERR_CUDA,                 \
                  std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                              \
  } while (0)

template <typename T>
int dalloc(T** p, size_t count, int64_t& bytes) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) return fail(GBCG_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  bytes += (int64_t)(count * sizeof(T));
  return 0;
}

template <typename T>
int upload(T** p, const std::vector<T>& h, cudaStream_t s, int64_t& bytes) {
  if (int rc = dalloc(p, h.size(), bytes)) return rc;
  if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return 0;
}

std::vector<float> to_f32(const std::vector<double>& v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}

// Tile caps of each precision's layout (the kernels' TileCaps).
constexpr int kTileSlices32 = kTileWarps * TileCaps<float>::kRpt, kTileSlices64 = kTileWarps * TileCaps<double>::kRpt;

int env_int(const char* name, int dflt) {
  const char* s = getenv(name);
  return (s && *s) ? atoi(s) : dflt;
}

}  // namespace

namespace gbcg {
// Sets the calling thread's message for gbcg_last_error() (also used by the
// allocation-free entry point in static_solve.cu).
void set_last_error(const std::string& m) { g_last_error = m; }
}  // namespace gbcg

// One tiled symmetric layout on the device (layout.h, SymTilesHost): the
// single-precision product and the double-precision product each have their
// own (tiles of up to 30 and 15 slices), over the same CTA row ranges.
struct DevTiles {
  int32_t *cta_tile = nullptr, *tile_slice = nullptr, *tile_ns = nullptr, *tile_own = nullptr, *tile_len = nullptr,
          *tile_stride = nullptr, *tile_win = nullptr, *win_start = nullptr, *win_len = nullptr;
  int64_t *tile_ent = nullptr, *tile_meta = nullptr, *tile_ext = nullptr, *in_src = nullptr;
  uint16_t* meta = nullptr;
  TileDesc* desc = nullptr;
  int32_t *carry_src = nullptr, *carry_dst = nullptr, *carry_len = nullptr, *flush_src = nullptr, *flush_len = nullptr,
          *flush_row = nullptr;
  int32_t *in_ptr = nullptr, *in_row = nullptr, *in_len = nullptr;
  void* val = nullptr;   // float or double values, in the layout's order
  void* part = nullptr;  // further window partial sums, same type
  void* p1 = nullptr;    // each row's first window partial sum, n values (zero where a row has none)
  int64_t ntiles = 0, next = 0, slots = 0;

  void release() {
    void* p[] = {cta_tile, tile_slice, tile_ns, tile_own, tile_len, tile_stride, tile_win, win_start, win_len,
                 tile_ent, tile_meta, tile_ext, in_src, meta, desc, carry_src, carry_dst, carry_len, flush_src,
                 flush_len, flush_row, in_ptr, in_row, in_len, val, part, p1};
    for (void* d : p)
      if (d) cudaFree(d);
    *this = DevTiles();
  }
  template <typename V>
  SymDev<V> dev() const {
    SymDev<V> t;
    t.desc = desc;
    t.carry_src = carry_src;
    t.carry_dst = carry_dst;
    t.carry_len = carry_len;
    t.flush_src = flush_src;
    t.flush_len = flush_len;
    t.flush_row = flush_row;
    t.p1 = (V*)p1;
    t.cta_tile = cta_tile;
    t.tile_slice = tile_slice;
    t.tile_ns = tile_ns;
    t.tile_own = tile_own;
    t.tile_len = tile_len;
    t.tile_stride = tile_stride;
    t.tile_ent = tile_ent;
    t.tile_meta = tile_meta;
    t.tile_ext = tile_ext;
    t.tile_win = tile_win;
    t.win_start = win_start;
    t.win_len = win_len;
    t.val = (const V*)val;
    t.meta = meta;
    t.in_ptr = in_ptr;
    t.in_row = in_row;
    t.in_len = in_len;
    t.in_src = in_src;
    t.part = (V*)part;
    return t;
  }
};

// Uploads one tiled layout; V is the type of its values.
template <typename V>
int upload_tiles(DevTiles& D, const SymTilesHost& Tl, int64_t n, cudaStream_t s, int64_t& B) {
  D.ntiles = (int64_t)Tl.tile_ns.size();
  D.next = Tl.tile_ext.back();
  D.slots = (int64_t)Tl.val.size();
  if (int rc = upload(&D.cta_tile, Tl.cta_tile, s, B)) return rc;
  if (int rc = upload(&D.tile_slice, Tl.tile_slice, s, B)) return rc;
  if (int rc = upload(&D.tile_ns, Tl.tile_ns, s, B)) return rc;
  if (int rc = upload(&D.tile_own, Tl.tile_own, s, B)) return rc;
  if (int rc = upload(&D.tile_len, Tl.tile_len, s, B)) return rc;
  if (int rc = upload(&D.tile_stride, Tl.tile_stride, s, B)) return rc;
  if (int rc = upload(&D.tile_ent, Tl.tile_ent, s, B)) return rc;
  if (int rc = upload(&D.tile_meta, Tl.tile_meta, s, B)) return rc;
  if (int rc = upload(&D.tile_ext, Tl.tile_ext, s, B)) return rc;
  if (int rc = upload(&D.tile_win, Tl.tile_win, s, B)) return rc;
  if (int rc = upload(&D.win_start, Tl.win_start, s, B)) return rc;
  if (int rc = upload(&D.win_len, Tl.win_len, s, B)) return rc;
  if (int rc = upload(&D.meta, Tl.meta, s, B)) return rc;
  if (int rc = upload(&D.in_ptr, Tl.in_ptr, s, B)) return rc;
  if (int rc = upload(&D.in_row, Tl.in_row, s, B)) return rc;
  if (int rc = upload(&D.in_len, Tl.in_len, s, B)) return rc;
  if (int rc = upload(&D.in_src, Tl.in_src, s, B)) return rc;
  if (int rc = upload(&D.desc, Tl.desc, s, B)) return rc;
  if (int rc = upload(&D.carry_src, Tl.carry_src, s, B)) return rc;
  if (int rc = upload(&D.carry_dst, Tl.carry_dst, s, B)) return rc;
  if (int rc = upload(&D.carry_len, Tl.carry_len, s, B)) return rc;
  if (int rc = upload(&D.flush_src, Tl.flush_src, s, B)) return rc;
  if (int rc = upload(&D.flush_len, Tl.flush_len, s, B)) return rc;
  if (int rc = upload(&D.flush_row, Tl.flush_row, s, B)) return rc;
  V* val = nullptr;
  if constexpr (sizeof(V) == 4) {
    if (int rc = upload(&val, to_f32(Tl.val), s, B)) return rc;
  } else {
    if (int rc = upload(&val, Tl.val, s, B)) return rc;
  }
  D.val = val;
  V* part = nullptr;
  if (int rc = dalloc(&part, (size_t)std::max<int64_t>(D.next, 1), B)) return rc;
  D.part = part;
  // rows that receive no first partial sum keep this zero for good
  V* p1 = nullptr;
  if (int rc = dalloc(&p1, (size_t)std::max<int64_t>(n, 1), B)) return rc;
  D.p1 = p1;
  CUDA_TRY(cudaMemsetAsync(p1, 0, sizeof(V) * (size_t)std::max<int64_t>(n, 1), s));
  return 0;
}

struct gbcg_matrix_s {
  int32_t format = 0, index_base = 0;
  int64_t n = 0, nnz_input = 0, nnz_full = 0, slots = 0, plan_slots = 0;
  // the caller's pattern, kept for value updates; device value slot -> input
  // entry maps (-1 on padding), built at the first update
  std::vector<int32_t> h_ptr, h_idx;
  int32_t *u_map_main = nullptr, *u_map_long = nullptr, *u_map_diag = nullptr;
  int64_t u_len_main = 0, u_len_long = 0, u_len_diag = 0;
  double* u_stage = nullptr;
  int64_t nslices = 0, nlong = 0, bytes = 0;
  int sym = 0;
  int mode = kGather;       // kGather (CSR/CSC), kPlan or kTiles (symmetric)
  int64_t l2_bytes = 0;     // the device's L2 size
  // tiled symmetric layouts (device): single- and double-precision products
  DevTiles t32, t64;
  int32_t *u_map_t32 = nullptr;  // value map of the single-precision tiles (u_map_main: double-precision)
  int64_t u_len_t32 = 0;
  // layout (device)
  int64_t* sl_ptr = nullptr;
  int32_t* col = nullptr;
  int16_t* col16 = nullptr;  // 16-bit column offsets (row-gather layout, when they fit)
  double* val64 = nullptr;
  float* val32 = nullptr;
  uint32_t* long_mask = nullptr;
  int32_t* long_row = nullptr;
  int64_t* long_ptr = nullptr;
  int32_t* long_col = nullptr;
  double* long_val64 = nullptr;
  float* long_val32 = nullptr;
  double* diag64 = nullptr;
  float* diag32 = nullptr;
  int64_t* pl_ptr = nullptr;
  int32_t* pl_i = nullptr;
  uint16_t* pl_k = nullptr;
  // persistent-solver partition
  int grid = 1;
  int32_t* cta_slice = nullptr;
  int32_t* cta_long = nullptr;
  // workspace
  double *r = nullptr, *p = nullptr, *q = nullptr, *bstage = nullptr, *xstage = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr, *rhs32 = nullptr;
  // single-reduction CG (double precision): s = A p, z = A s, w = A r (two buffers)
  double *s64 = nullptr, *z64 = nullptr, *w64a = nullptr, *w64b = nullptr;
  double* part = nullptr;   // max(2 * grid, one-shot blocks)
  double* sums = nullptr;   // small scalars
  int64_t part_len = 0;
  GridBar* bar = nullptr;
  CgState* st = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // brackets of the persistent launches
  // pinned host mirrors
  CgState* st_h = nullptr;
  GridBar* bar_h = nullptr;
  double* sums_h = nullptr;

  template <typename V>
  OpDev<V> op() const;
  template <typename V>
  SymDev<V> tiles() const {
    return sizeof(V) == 4 ? t32.dev<V>() : t64.dev<V>();
  }
  int spmv_blocks() const { return (int)std::max<int64_t>(1, (nslices + nlong + 7) / 8); }
};

template <>
OpDev<double> gbcg_matrix_s::op<double>() const {
  OpDev<double> o;
  o.n = n;
  o.nslices = nslices;
  o.nlong = nlong;
  o.sl_ptr = sl_ptr;
  o.col = col;
  o.col16 = col16;
  o.val = val64;
  o.long_mask = long_mask;
  o.long_row = long_row;
  o.long_ptr = long_ptr;
  o.long_col = long_col;
  o.long_val = long_val64;
  o.diag = diag64;
  o.pl_ptr = pl_ptr;
  o.pl_i = pl_i;
  o.pl_k = pl_k;
  return o;
}
template <>
OpDev<float> gbcg_matrix_s::op<float>() const {
  OpDev<float> o;
  o.n = n;
  o.nslices = nslices;
  o.nlong = nlong;
  o.sl_ptr = sl_ptr;
  o.col = col;
  o.col16 = col16;
  o.val = val32;
  o.long_mask = long_mask;
  o.long_row = long_row;
  o.long_ptr = long_ptr;
  o.long_col = long_col;
  o.long_val = long_val32;
  o.diag = diag32;
  o.pl_ptr = pl_ptr;
  o.pl_i = pl_i;
  o.pl_k = pl_k;
  return o;
}

namespace {

void free_matrix(gbcg_matrix_s* M) {
  if (!M) return;
  void* dev[] = {M->sl_ptr, M->col, M->col16, M->val64, M->val32, M->long_mask, M->long_row, M->long_ptr, M->long_col,
                 M->long_val64, M->long_val32, M->diag64, M->diag32, M->pl_ptr, M->pl_i, M->pl_k,
                 M->cta_slice, M->cta_long, M->r, M->p, M->q, M->bstage, M->xstage, M->r32, M->p32, M->q32,
                 M->d32, M->rhs32, M->part, M->sums, M->bar, M->st, M->u_map_main, M->u_map_long, M->u_map_diag,
                 M->u_map_t32, M->u_stage, M->s64, M->z64, M->w64a, M->w64b};
  M->t32.release();
  M->t64.release();
  for (void* d : dev)
    if (d) cudaFree(d);
  if (M->st_h) cudaFreeHost(M->st_h);
  if (M->bar_h) cudaFreeHost(M->bar_h);
  if (M->sums_h) cudaFreeHost(M->sums_h);
  if (M->ev0) cudaEventDestroy(M->ev0);
  if (M->ev1) cudaEventDestroy(M->ev1);
  delete M;
}

// Threads per CTA: the tiled symmetric kernels add a producer warp.
constexpr int block_of(int fmt) { return fmt == kTiles ? kTileThreads : kCgThreads; }

template <typename V, int FMT, bool OUTER>
int occupancy_of(int& per_sm) {
  const size_t sm = product_smem<V, FMT>();
  CUDA_TRY(cudaFuncSetAttribute(k_cg<V, FMT, OUTER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg<V, FMT, OUTER>, block_of(FMT), sm));
  return 0;
}

// Shared memory of the reliable-update kernel: the per-warp stages of both
// precisions' gather pipelines, or (kTiles) the larger of the two tile
// pipelines' carvings, used in turn.
template <int FMT>
constexpr size_t ru_smem() {
  return FMT == kTiles ? std::max(sym_smem_bytes<float>(), sym_smem_bytes<double>())
                       : (size_t)kWarps * ru_warp_stage_bytes();
}

template <int FMT>
int ru_occupancy_of(int& per_sm) {
  CUDA_TRY(cudaFuncSetAttribute(k_cg_ru<FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ru_smem<FMT>()));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_ru<FMT>, block_of(FMT), ru_smem<FMT>()));
  return 0;
}

template <int FMT>
int pcg_occupancy_of(int& per_sm) {
  if constexpr (FMT == kTiles) {
    per_sm = 1 << 20;
    return 0;
  } else {
    const size_t sm = product_smem<double, FMT>();
    CUDA_TRY(cudaFuncSetAttribute(k_pcg<double, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<double, FMT>, kCgThreads, sm));
    return 0;
  }
}

template <typename V, int FMT>
int prepare_rows() {
  CUDA_TRY(cudaFuncSetAttribute(k_rows<V, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)product_smem<V, FMT>()));
  return 0;
}

// Co-resident CTAs per SM of the persistent solver in layout mode FMT (and
// the shared-memory attributes of the kernels of that mode).
template <int FMT>
int solver_occupancy(int& per_sm) {
  int a = 0, b = 0, c = 0, e = 0;
  if (int rc = occupancy_of<double, FMT, true>(a)) return rc;
  if (int rc = occupancy_of<float, FMT, false>(b)) return rc;
  if (int rc = pcg_occupancy_of<FMT>(c)) return rc;
  if (int rc = ru_occupancy_of<FMT>(e)) return rc;
  if (int rc = prepare_rows<double, FMT>()) return rc;
  if (int rc = prepare_rows<float, FMT>()) return rc;
  per_sm = std::min(std::min(a, b), std::min(c, e));
  return 0;
}

int mode_occupancy(int mode, int& per_sm) {
  return mode == kTiles ? solver_occupancy<kTiles>(per_sm)
                        : mode == kPlan ? solver_occupancy<kPlan>(per_sm) : solver_occupancy<kGather>(per_sm);
}

// The kernels read and write vectors with 16-byte loads and bulk copies.
bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename V, int FMT, bool OUTER>
cudaError_t launch_cg(const CgArgs<V>& args, int grid, cudaStream_t s) {
  void* kargs[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)k_cg<V, FMT, OUTER>, dim3(grid), dim3(block_of(FMT)), kargs,
                                     product_smem<V, FMT>(), s);
}

template <typename V, bool OUTER>
cudaError_t launch_cg_fmt(const gbcg_matrix_s* M, const CgArgs<V>& a, cudaStream_t s) {
  switch (M->mode) {
    case kTiles: return launch_cg<V, kTiles, OUTER>(a, M->grid, s);
    case kPlan: return launch_cg<V, kPlan, OUTER>(a, M->grid, s);
    default: return launch_cg<V, kGather, OUTER>(a, M->grid, s);
  }
}

template <int FMT>
cudaError_t launch_pcg(const PcgArgs<double>& args, int grid, cudaStream_t s) {
  void* kargs[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)k_pcg<double, FMT>, dim3(grid), dim3(kCgThreads), kargs,
                                     product_smem<double, FMT>(), s);
}

// The single-reduction CG on the handle's layout (row-gather layouts only;
// the caller has checked the mode).
cudaError_t launch_pcg_fmt(const gbcg_matrix_s* M, const CgArgs<double>& c, cudaStream_t s) {
  PcgArgs<double> a;
  a.c = c;
  a.s = M->s64;
  a.z = M->z64;
  a.w0 = M->w64a;
  a.w1 = M->w64b;
  return M->mode == kPlan ? launch_pcg<kPlan>(a, M->grid, s) : launch_pcg<kGather>(a, M->grid, s);
}

template <int FMT>
cudaError_t launch_ru(const RuArgs& args, int grid, cudaStream_t s) {
  void* kargs[] = {(void*)&args};
  return cudaLaunchCooperativeKernel((const void*)k_cg_ru<FMT>, dim3(grid), dim3(block_of(FMT)), kargs,
                                     ru_smem<FMT>(), s);
}

// Product y = A x (MODE 0), or r = b - A x into y with per-CTA partial sums
// of r'r in part (MODE 1, double precision), on the persistent partition.
template <typename V, int FMT, int MODE>
cudaError_t launch_product(const gbcg_matrix_s* M, const V* x, const V* b, V* y, cudaStream_t s) {
  k_rows<V, FMT><<<M->grid, block_of(FMT), product_smem<V, FMT>(), s>>>(
      M->op<V>(), M->tiles<V>(), M->cta_slice, M->cta_long, x, y, &M->bar->status, 1000000000LL);
  if (FMT == kTiles || MODE == 1)
    k_finish<V, FMT, MODE><<<M->grid, kCgThreads, 0, s>>>(M->tiles<V>(), M->cta_slice, M->n, b, y, M->part);
  return cudaGetLastError();
}

template <typename V, int MODE>
cudaError_t launch_product_fmt(const gbcg_matrix_s* M, const V* x, const V* b, V* y, cudaStream_t s) {
  switch (M->mode) {
    case kTiles: return launch_product<V, kTiles, MODE>(M, x, b, y, s);
    case kPlan: return launch_product<V, kPlan, MODE>(M, x, b, y, s);
    default: return launch_product<V, kGather, MODE>(M, x, b, y, s);
  }
}

// The device-side half of gbcg_solve_async: the solver state as the fields
// of gbcg_info (status mapped as status_from_device maps it on the host).
__global__ void k_export_info(const CgState* st, const GridBar* gb, gbcg_device_info* out, int ru) {
  int status;
  if (gb->status != 0) {
    status = GBCG_ERR_TIMEOUT;
  } else {
    switch (st->status) {
      case kOk: status = GBCG_OK; break;
      case kNotSpd: status = GBCG_ERR_NOT_SPD; break;
      case kMaxit: status = GBCG_ERR_MAXIT; break;
      case kNonfinite: status = GBCG_ERR_NONFINITE; break;
      default: status = GBCG_ERR_TIMEOUT; break;
    }
  }
  out->status = status;
  out->iterations = st->k;
  out->outer = st->restarts;
  out->pad_ = 0;
  out->rel_res_true = st->nb > 0 ? st->rel_true : 0.0;
  out->rel_res_recursive = ru ? st->rel_true : (st->nb > 0 ? sqrt(st->rr) / st->nb : 0.0);
}

int status_from_device(const CgState& st, const GridBar& gb) {
  if (gb.status != 0) return GBCG_ERR_TIMEOUT;
  switch (st.status) {
    case kOk: return GBCG_OK;
    case kNotSpd: return GBCG_ERR_NOT_SPD;
    case kMaxit: return GBCG_ERR_MAXIT;
    case kNonfinite: return GBCG_ERR_NONFINITE;
    default: return GBCG_ERR_TIMEOUT;
  }
}

long long timeout_ns_of(const gbcg_opts* o) {
  int ms = (o && o->wait_timeout_ms > 0) ? o->wait_timeout_ms : 1000;
  return (long long)ms * 1000000LL;
}

template <typename V>
CgArgs<V> make_args(const gbcg_matrix_s* M, V* x, V* r, V* p, V* q, const V* b, double tol, int maxit,
                    int max_restarts, long long timeout_ns) {
  CgArgs<V> a;
  a.A = M->op<V>();
  a.T = M->tiles<V>();
  a.x = x;
  a.r = r;
  a.p = p;
  a.q = q;
  a.b = b;
  a.part = M->part;
  a.bar = M->bar;
  a.st = M->st;
  a.cta_slice = M->cta_slice;
  a.cta_long = M->cta_long;
  a.tol = tol;
  a.maxit = maxit;
  a.max_restarts = max_restarts;
  // on the tiled layout the vector passes stream through shared memory when
  // the five vectors of the r update (5 values per row) outgrow the L2; from
  // L2 the register-pipelined passes are faster (reliable updates: 46.2
  // against 44.7 us per iteration at 128^3, 320 against 351 at 256^3).
  // GBCG_STREAM_VEC=0/1 forces either (tests)
  a.stream_vec = M->mode == kTiles && (int64_t)(5 * sizeof(V)) * M->n > M->l2_bytes ? 1 : 0;
  if (const int f = env_int("GBCG_STREAM_VEC", -1); f >= 0 && M->mode == kTiles) a.stream_vec = f ? 1 : 0;
  a.timeout_ns = timeout_ns;
  return a;
}

// Reads the solver state and barrier word back (one synchronisation).
int read_state(gbcg_matrix_s* M, cudaStream_t s) {
  CUDA_TRY(cudaMemcpyAsync(M->st_h, M->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(M->bar_h, M->bar, sizeof(GridBar), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return 0;
}

// Enqueues the double-precision persistent solve (either variant): the
// barrier reset and the launch, bracketed by the handle's events when timed.
cudaError_t enqueue_fp64(gbcg_matrix_s* M, const double* b, double* x, double tol, int maxit, const gbcg_opts* o,
                         bool timed, cudaStream_t s) {
  const int max_restarts = (o && o->max_restarts > 0) ? o->max_restarts : 3;
  cudaError_t e = cudaMemsetAsync(M->bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  CgArgs<double> a = make_args<double>(M, x, M->r, M->p, M->q, b, tol, maxit, max_restarts, timeout_ns_of(o));
  if (timed && (e = cudaEventRecord(M->ev0, s)) != cudaSuccess) return e;
  e = (o && o->variant == GBCG_PIPELINED) ? launch_pcg_fmt(M, a, s) : launch_cg_fmt<double, true>(M, a, s);
  if (e != cudaSuccess) return e;
  return timed ? cudaEventRecord(M->ev1, s) : cudaSuccess;
}

int solve_fp64(gbcg_matrix_s* M, const double* b, double* x, double tol, int maxit, const gbcg_opts* o,
               gbcg_info* info, cudaStream_t s) {
  CUDA_TRY(enqueue_fp64(M, b, x, tol, maxit, o, true, s));
  if (int rc = read_state(M, s)) return rc;
  float kms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&kms, M->ev0, M->ev1));
  info->kernel_ms = kms;
  info->kernel_launches = 1;
  info->launches = 1;
  const int status = status_from_device(*M->st_h, *M->bar_h);
  info->iterations = M->st_h->k;
  info->outer = M->st_h->restarts;
  info->status = status;
  info->rel_res_recursive = M->st_h->nb > 0 ? std::sqrt(M->st_h->rr) / M->st_h->nb : 0.0;
  info->rel_res_true = M->st_h->nb > 0 ? M->st_h->rel_true : 0.0;
  if (status == GBCG_ERR_TIMEOUT)
    g_last_error = "device-side wait ran out (barrier " + std::to_string(M->bar_h->where) + "; " +
                   std::to_string(M->bar_h->detail[0]) + " " + std::to_string(M->bar_h->detail[1]) + " " +
                   std::to_string(M->bar_h->detail[2]) + " " + std::to_string(M->bar_h->detail[3]) + ")";
  return status;
}

// Single-precision iterations with double-precision reliable updates: one
// persistent launch, on any layout.
cudaError_t enqueue_ru(gbcg_matrix_s* M, const double* b, double* x, double tol, int maxit, const gbcg_opts* o,
                       bool timed, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(M->bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  RuArgs a;
  a.c = make_args<float>(M, M->d32, M->r32, M->p32, M->q32, nullptr, tol, maxit, 0, timeout_ns_of(o));
  a.A64 = M->op<double>();
  a.T64 = M->tiles<double>();
  a.x64 = x;
  a.b64 = b;
  a.q64 = M->q;
  a.delta = (o && o->inner_tol > 0.0 && o->inner_tol < 1.0) ? o->inner_tol : 0.1;
  if (timed && (e = cudaEventRecord(M->ev0, s)) != cudaSuccess) return e;
  e = M->mode == kTiles  ? launch_ru<kTiles>(a, M->grid, s)
      : M->mode == kPlan ? launch_ru<kPlan>(a, M->grid, s)
                         : launch_ru<kGather>(a, M->grid, s);
  if (e != cudaSuccess) return e;
  return timed ? cudaEventRecord(M->ev1, s) : cudaSuccess;
}

int solve_ru(gbcg_matrix_s* M, const double* b, double* x, double tol, int maxit, const gbcg_opts* o,
             gbcg_info* info, cudaStream_t s) {
  CUDA_TRY(enqueue_ru(M, b, x, tol, maxit, o, true, s));
  if (int rc = read_state(M, s)) return rc;
  float kms = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&kms, M->ev0, M->ev1));
  info->kernel_ms = kms;
  info->kernel_launches = 1;
  info->launches = 1;
  const int status = status_from_device(*M->st_h, *M->bar_h);
  info->iterations = M->st_h->k;
  info->outer = M->st_h->restarts;
  info->status = status;
  info->rel_res_recursive = M->st_h->rel_true;
  info->rel_res_true = M->st_h->rel_true;
  if (status == GBCG_ERR_TIMEOUT) g_last_error = "device-side wait ran out (reliable-update solve)";
  return status;
}

int dot_to_host(gbcg_matrix_s* M, const double* a, const double* b, double& out, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(M->part_len, std::max<int64_t>(1, (M->n + 255) / 256));
  k_dot_part<<<blocks, 256, 0, s>>>(a, b, M->n, M->part);
  k_sum_part<<<1, 256, 0, s>>>(M->part, blocks, M->sums);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(M->sums_h, M->sums, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  out = M->sums_h[0];
  return 0;
}

int residual_to_host(gbcg_matrix_s* M, const double* b, const double* x, double& rr, cudaStream_t s) {
  CUDA_TRY(launch_product_fmt<double, 1>(M, x, b, M->r, s));
  k_sum_part<<<1, 256, 0, s>>>(M->part, M->grid, M->sums);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(M->sums_h, M->sums, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  rr = M->sums_h[0];
  return 0;
}

// Single-precision inner CG with double-precision iterative refinement.
int solve_ir(gbcg_matrix_s* M, const double* b, double* x, double tol, int maxit, const gbcg_opts* o,
             gbcg_info* info, cudaStream_t s) {
  const int max_outer = (o && o->max_outer > 0) ? o->max_outer : 30;
  const double inner_tol = (o && o->inner_tol > 0) ? o->inner_tol : 1e-4;
  const long long tns = timeout_ns_of(o);
  const int64_t n = M->n;
  const int gsz = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (n + 255) / 256));
  double bb = 0.0;
  if (int rc = dot_to_host(M, b, b, bb, s)) return rc;
  info->launches += 2;  // k_dot_part + k_sum_part
  const double nb = std::sqrt(bb);
  int used = 0, outer = 0, status = GBCG_ERR_MAXIT;
  double rel = 0.0;
  if (nb == 0.0) {
    CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    status = GBCG_OK;
  } else {
    for (;;) {
      double rr = 0.0;
      if (int rc = residual_to_host(M, b, x, rr, s)) return rc;
      info->launches += 3;  // k_rows + k_finish + k_sum_part
      rel = std::sqrt(rr) / nb;
      if (!std::isfinite(rel)) { status = GBCG_ERR_NONFINITE; break; }
      if (rel <= tol) { status = GBCG_OK; break; }
      if (outer >= max_outer || used >= maxit) { status = GBCG_ERR_MAXIT; break; }
      const double nr = std::sqrt(rr);
      k_scale_to_f32<<<gsz, 256, 0, s>>>(M->r, 1.0 / nr, n, M->rhs32);
      CUDA_TRY(cudaGetLastError());
      CUDA_TRY(cudaMemsetAsync(M->bar, 0, sizeof(GridBar), s));
      CgArgs<float> a = make_args<float>(M, M->d32, M->r32, M->p32, M->q32, M->rhs32, inner_tol, maxit - used, 0, tns);
      CUDA_TRY(cudaEventRecord(M->ev0, s));
      CUDA_TRY(launch_cg_fmt<float, false>(M, a, s));
      CUDA_TRY(cudaEventRecord(M->ev1, s));
      if (int rc = read_state(M, s)) return rc;
      float kms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&kms, M->ev0, M->ev1));
      info->kernel_ms += kms;
      info->kernel_launches += 1;
      info->launches += 2;  // k_scale_to_f32 + inner k_cg
      if (M->bar_h->status != 0) {
        status = GBCG_ERR_TIMEOUT;
        g_last_error = "device-side wait ran out (inner solve)";
        break;
      }
      used += M->st_h->k;
      ++outer;
      if ((M->st_h->status == kNotSpd || M->st_h->status == kNonfinite) && M->st_h->k == 0) {
        status = M->st_h->status == kNotSpd ? GBCG_ERR_NOT_SPD : GBCG_ERR_NONFINITE;
        break;
      }
      k_axpy_f32<<<gsz, 256, 0, s>>>(nr, M->d32, n, x);
      CUDA_TRY(cudaGetLastError());
      info->launches += 1;
    }
  }
  info->iterations = used;
  info->outer = outer;
  info->status = status;
  info->rel_res_recursive = rel;
  info->rel_res_true = rel;
  return status;
}

template <typename V>
int spmv_any(gbcg_matrix_t A, const V* x, V* y, cudaStream_t s) {
  if (!A) return fail(GBCG_ERR_INVALID, "null matrix handle");
  if (A->n == 0) return GBCG_OK;
  if (!x || !y) return fail(GBCG_ERR_INVALID, "null vector");
  if (misaligned16(x) || misaligned16(y)) return fail(GBCG_ERR_INVALID, "x and y must be 16-byte aligned");
  CUDA_TRY(launch_product_fmt<V, 0>(A, x, nullptr, y, s));
  return GBCG_OK;
}

}  // namespace

extern "C" {

int gbcg_create(gbcg_matrix_t* out, int32_t format, int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                const double* val, int32_t index_base, int32_t memory, void* stream) {
  g_last_error.clear();
  if (!out) return fail(GBCG_ERR_INVALID, "null output handle");
  *out = nullptr;
  if (n < 0 || nnz < 0) return fail(GBCG_ERR_INVALID, "n and nnz must be non-negative");
  if (memory != GBCG_HOST && memory != GBCG_DEVICE) return fail(GBCG_ERR_INVALID, "memory must be GBCG_HOST or GBCG_DEVICE");
  if (!ptr) return fail(GBCG_ERR_INVALID, "null ptr array");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> hptr, hidx;
  std::vector<double> hval;
  if (memory == GBCG_DEVICE) {  // bring the caller's arrays to the host for the layout build
    hptr.resize(n + 1);
    CUDA_TRY(cudaMemcpyAsync(hptr.data(), ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    if (nnz > 0) {
      if (!idx || !val) return fail(GBCG_ERR_INVALID, "null idx/val array");
      hidx.resize(nnz);
      hval.resize(nnz);
      CUDA_TRY(cudaMemcpyAsync(hidx.data(), idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaMemcpyAsync(hval.data(), val, sizeof(double) * nnz, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    ptr = hptr.data();
    idx = hidx.data();
    val = hval.data();
  }
  LayoutHost L;
  std::string err;
  int rc = build_layout(format, n, nnz, ptr, idx, val, index_base, L, err);
  if (rc) return fail(rc, err);
  // debug mode: full CSR/CSC inputs must be symmetric (CG's premise)
  if (format != GBCG_SYM_CSR_UPPER && env_int("GBCG_CHECK_SYMMETRY", 0) != 0 &&
      (rc = check_symmetry(n, nnz, ptr, idx, val, index_base, err)) != 0)
    return fail(rc, err);

  gbcg_matrix_s* M = new gbcg_matrix_s();
  M->format = format;
  M->n = n;
  M->nnz_input = nnz;
  M->nnz_full = L.nnz_full;
  M->sym = format == GBCG_SYM_CSR_UPPER;
  M->nslices = L.A.nslices;
  M->nlong = (int64_t)L.A.long_row.size();
  M->slots = L.A.sl_ptr.empty() ? 0 : L.A.sl_ptr.back();
  M->plan_slots = L.plan.pl_ptr.empty() ? 0 : L.plan.pl_ptr.back();
  M->index_base = index_base;
  M->h_ptr.assign(ptr, ptr + n + 1);
  M->h_idx.assign(idx, idx + nnz);
  auto bail = [&](int code) {
    free_matrix(M);
    return code;
  };
#define TRY(x)                  \
  do {                          \
    if (int rc_ = (x)) return bail(rc_); \
  } while (0)
  int64_t& B = M->bytes;
  // persistent-solver grid: every co-resident CTA that gets a slice.  Even a
  // few slices per CTA beat fewer, fuller CTAs: at 25 230 rows on GB300, 152
  // CTAs against 50 run a reliable-update iteration in 11.2 against 12.0 us
  // (full CSR) and 16.4 against 18.7 us (symmetric tiles)
  int dev = 0, sms = 0, per_sm = 0;
  int l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
    return bail(fail(GBCG_ERR_CUDA, "cannot query the device"));
  M->l2_bytes = l2;
  const char* sym_mode = getenv("GBCG_SYM_LAYOUT");
  M->mode = !M->sym ? kGather : (sym_mode && !strcmp(sym_mode, "plan")) ? kPlan : kTiles;
  auto choose_grid = [&]() -> int {
    if (int rc = mode_occupancy(M->mode, per_sm)) return rc;
    if (per_sm < 1) return fail(GBCG_ERR_CUDA, "the persistent solver kernel cannot be resident");
    per_sm = std::min(per_sm, std::max(1, env_int("GBCG_CTAS_PER_SM", 2)));
    const int64_t want = M->nslices;
    const int env_grid = env_int("GBCG_GRID", 0);
    M->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, want));
    if (env_grid > 0) M->grid = std::min(env_grid, per_sm * sms);
    return 0;
  };
  TRY(choose_grid());
  SymTilesHost T32, T64;
  if (M->mode == kTiles &&
      (!build_sym_tiles(L, M->grid, TileCaps<float>::kSlot, TileCaps<float>::kEnt, kTileSlices32, T32) ||
       !build_sym_tiles(L, M->grid, TileCaps<double>::kSlot, TileCaps<double>::kEnt, kTileSlices64, T64))) {
    M->mode = kPlan;  // a single slice exceeds what a tile holds
    TRY(choose_grid());
  }
  std::vector<int32_t> cs, cl(M->grid + 1, 0);
  if (M->mode == kTiles) {
    // both layouts cut the rows at the same CTA boundaries (the vector
    // phases of a solve run over those rows)
    cs.resize(M->grid + 1);
    for (int c = 0; c <= M->grid; ++c) {
      cs[c] = T64.tile_slice[T64.cta_tile[c]];
      if (cs[c] != T32.tile_slice[T32.cta_tile[c]])
        return bail(fail(GBCG_ERR_INVALID, "tile layouts of the two precisions cut the rows differently"));
    }
    TRY(upload_tiles<float>(M->t32, T32, n, s, B));
    TRY(upload_tiles<double>(M->t64, T64, n, s, B));
    M->slots = M->t64.slots;
    M->plan_slots = 0;
    TRY(upload(&M->long_mask, std::vector<uint32_t>(std::max<int64_t>(M->nslices, 1), 0u), s, B));
  } else {
    TRY(upload(&M->sl_ptr, L.A.sl_ptr, s, B));
    TRY(upload(&M->col, L.A.col, s, B));
    if (!L.A.col16.empty() && M->mode == kGather && env_int("GBCG_WIDE_INDEX", 0) == 0)
      TRY(upload(&M->col16, L.A.col16, s, B));
    TRY(upload(&M->val64, L.A.val, s, B));
    TRY(upload(&M->val32, to_f32(L.A.val), s, B));
    TRY(upload(&M->long_mask, L.A.long_mask, s, B));
    TRY(upload(&M->long_row, L.A.long_row, s, B));
    TRY(upload(&M->long_ptr, L.A.long_ptr, s, B));
    TRY(upload(&M->long_col, L.A.long_col, s, B));
    TRY(upload(&M->long_val64, L.A.long_val, s, B));
    TRY(upload(&M->long_val32, to_f32(L.A.long_val), s, B));
    if (M->mode == kPlan) {
      TRY(upload(&M->pl_ptr, L.plan.pl_ptr, s, B));
      TRY(upload(&M->pl_i, L.plan.pl_i, s, B));
      TRY(upload(&M->pl_k, L.plan.pl_k, s, B));
    }
    cs = partition_slices(L, M->grid);
    for (int c = 0; c <= M->grid; ++c) {  // long rows go to the CTA that owns their row
      const int64_t row0 = (int64_t)cs[c] * 32;
      cl[c] = (int32_t)(std::lower_bound(L.A.long_row.begin(), L.A.long_row.end(), row0) - L.A.long_row.begin());
    }
    cl[M->grid] = (int32_t)M->nlong;
  }
  if (M->sym) {
    TRY(upload(&M->diag64, L.diag, s, B));
    TRY(upload(&M->diag32, to_f32(L.diag), s, B));
  }
  TRY(upload(&M->cta_slice, cs, s, B));
  TRY(upload(&M->cta_long, cl, s, B));
  // workspace
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  TRY(dalloc(&M->r, nn, B));
  TRY(dalloc(&M->p, nn, B));
  TRY(dalloc(&M->q, nn, B));
  TRY(dalloc(&M->bstage, nn, B));
  TRY(dalloc(&M->xstage, nn, B));
  TRY(dalloc(&M->r32, nn, B));
  TRY(dalloc(&M->p32, nn, B));
  TRY(dalloc(&M->q32, nn, B));
  TRY(dalloc(&M->d32, nn, B));
  TRY(dalloc(&M->rhs32, nn, B));
  if (M->mode != kTiles) {  // the single-reduction CG's vectors
    TRY(dalloc(&M->s64, nn, B));
    TRY(dalloc(&M->z64, nn, B));
    TRY(dalloc(&M->w64a, nn, B));
    TRY(dalloc(&M->w64b, nn, B));
  }
  M->part_len = std::max<int64_t>({6 * (int64_t)M->grid, (int64_t)M->spmv_blocks(), 4096});
  TRY(dalloc(&M->part, (size_t)M->part_len, B));
  TRY(dalloc(&M->sums, 8, B));
  TRY(dalloc(&M->bar, 1, B));
  TRY(dalloc(&M->st, 1, B));
  if (cudaMallocHost((void**)&M->st_h, sizeof(CgState)) != cudaSuccess ||
      cudaMallocHost((void**)&M->bar_h, sizeof(GridBar)) != cudaSuccess ||
      cudaMallocHost((void**)&M->sums_h, 8 * sizeof(double)) != cudaSuccess)
    return bail(fail(GBCG_ERR_NOMEM, "cudaMallocHost failed"));
  if (cudaEventCreate(&M->ev0) != cudaSuccess || cudaEventCreate(&M->ev1) != cudaSuccess)
    return bail(fail(GBCG_ERR_CUDA, "cudaEventCreate failed"));
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(GBCG_ERR_CUDA, "upload failed"));
#undef TRY
  *out = M;
  return GBCG_OK;
}

int gbcg_destroy(gbcg_matrix_t A) {
  free_matrix(A);
  return GBCG_OK;
}

int gbcg_spmv(gbcg_matrix_t A, const double* x, double* y, void* stream) {
  g_last_error.clear();
  return spmv_any<double>(A, x, y, (cudaStream_t)stream);
}

int gbcg_spmv_f32(gbcg_matrix_t A, const float* x, float* y, void* stream) {
  g_last_error.clear();
  return spmv_any<float>(A, x, y, (cudaStream_t)stream);
}

namespace {

// The combinations of precision, variant and layout a solve accepts.
int check_solve_opts(const gbcg_matrix_s* A, const gbcg_opts* opts) {
  if (opts && (opts->precision != GBCG_FP64 && opts->precision != GBCG_FP32_IR && opts->precision != GBCG_FP32_RU))
    return fail(GBCG_ERR_INVALID, "unknown precision");
  if (opts && opts->precision == GBCG_FP32_RU && opts->variant == GBCG_PIPELINED)
    return fail(GBCG_ERR_INVALID, "the single-reduction variant is double precision only");
  if (opts && opts->variant != GBCG_STANDARD && opts->variant != GBCG_PIPELINED)
    return fail(GBCG_ERR_INVALID, "unknown variant");
  if (opts && opts->variant == GBCG_PIPELINED && opts->precision == GBCG_FP32_IR)
    return fail(GBCG_ERR_INVALID,
                "the single-reduction variant is double precision only: in single precision its recurrences "
                "drift past any useful inner tolerance");
  if (opts && opts->variant == GBCG_PIPELINED && A->mode == kTiles)
    return fail(GBCG_ERR_INVALID,
                "the single-reduction variant runs on row-gather layouts (CSR, CSC, or symmetric storage with "
                "GBCG_SYM_LAYOUT=plan); the tiled symmetric product needs a barrier of its own");
  return GBCG_OK;
}

}  // namespace

int gbcg_solve(gbcg_matrix_t A, const double* b, double* x, double tol, int32_t maxit, const gbcg_opts* opts,
               gbcg_info* info, void* stream) {
  g_last_error.clear();
  gbcg_info local;
  if (!info) info = &local;
  memset(info, 0, sizeof(*info));
  if (!A) return fail(GBCG_ERR_INVALID, "null matrix handle");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(GBCG_ERR_INVALID, "tol must be finite and >= 0");
  if (int rc = check_solve_opts(A, opts)) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n;
  if (n == 0) {
    info->status = GBCG_OK;
    return GBCG_OK;
  }
  if (!b || !x) return fail(GBCG_ERR_INVALID, "null vector");
  if (maxit <= 0) maxit = (int32_t)std::min<int64_t>(n, 0x7fffffff);
  const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  if (bdev != xdev) return fail(GBCG_ERR_INVALID, "b and x must both be device or both be host memory");
  if (bdev && (misaligned16(b) || misaligned16(x)))
    return fail(GBCG_ERR_INVALID, "device b and x must be 16-byte aligned");
  const double* bd = b;
  double* xd = x;
  if (!bdev) {  // host vectors: stage through the buffers allocated at create time
    CUDA_TRY(cudaMemcpyAsync(A->bstage, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(A->xstage, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    bd = A->bstage;
    xd = A->xstage;
  }
  int status;
  if (opts && opts->precision == GBCG_FP32_IR)
    status = solve_ir(A, bd, xd, tol, maxit, opts, info, s);
  else if (opts && opts->precision == GBCG_FP32_RU)
    status = solve_ru(A, bd, xd, tol, maxit, opts, info, s);
  else
    status = solve_fp64(A, bd, xd, tol, maxit, opts, info, s);
  if (status == GBCG_ERR_CUDA || status == GBCG_ERR_NOMEM) return status;
  if (!bdev) {
    CUDA_TRY(cudaMemcpyAsync(x, A->xstage, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

int gbcg_solve_async(gbcg_matrix_t A, const double* b, double* x, double tol, int32_t maxit, const gbcg_opts* opts,
                     gbcg_device_info* dinfo, void* stream) {
  g_last_error.clear();
  if (!A) return fail(GBCG_ERR_INVALID, "null matrix handle");
  if (!dinfo) return fail(GBCG_ERR_INVALID, "null device info");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(GBCG_ERR_INVALID, "tol must be finite and >= 0");
  if (int rc = check_solve_opts(A, opts)) return rc;
  if (opts && opts->precision == GBCG_FP32_IR)
    return fail(GBCG_ERR_INVALID, "the refinement steers its passes from the host: no asynchronous form");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n;
  if (n == 0) {
    CUDA_TRY(cudaMemsetAsync(dinfo, 0, sizeof(gbcg_device_info), s));  // GBCG_OK, nothing to do
    return GBCG_OK;
  }
  if (!b || !x) return fail(GBCG_ERR_INVALID, "null vector");
  if (misaligned16(b) || misaligned16(x)) return fail(GBCG_ERR_INVALID, "b and x must be 16-byte aligned");
  if (maxit <= 0) maxit = (int32_t)std::min<int64_t>(n, 0x7fffffff);
  const bool ru = opts && opts->precision == GBCG_FP32_RU;
  CUDA_TRY(ru ? enqueue_ru(A, b, x, tol, maxit, opts, false, s) : enqueue_fp64(A, b, x, tol, maxit, opts, false, s));
  k_export_info<<<1, 1, 0, s>>>(A->st, A->bar, dinfo, ru ? 1 : 0);
  CUDA_TRY(cudaGetLastError());
  return GBCG_OK;
}

int gbcg_stats(gbcg_matrix_t A, gbcg_matrix_stats* out) {
  if (!A || !out) return fail(GBCG_ERR_INVALID, "null argument");
  memset(out, 0, sizeof(*out));
  out->n = A->n;
  out->nnz_input = A->nnz_input;
  out->nnz_full = A->nnz_full;
  out->stored_slots = A->slots;
  out->plan_slots = A->plan_slots;
  out->long_rows = A->nlong;
  out->device_bytes = A->bytes;
  const int64_t n = A->n, m = A->nnz_input;
  // the product's matrix stream: value + column index per entry (2-byte
  // offsets in the row-gather layout when they fit), row pointers, x, y
  const int64_t ib = A->col16 ? 2 : 4;
  out->spmv_bytes_fp64 = (8 + ib) * m + 4 * (n + 1) + 16 * n;
  out->spmv_bytes_fp32 = (4 + ib) * m + 4 * (n + 1) + 8 * n;
  out->index_bytes = (int32_t)ib;
  out->format = A->format;
  out->grid_ctas = A->grid;
  out->layout = A->mode;
  out->tiles = (int32_t)A->t64.ntiles;  // the double-precision layout's (the single-precision one has about half)
  out->ext_slots = A->t64.next;
  return GBCG_OK;
}

int gbcg_update_values(gbcg_matrix_t A, const double* val, int32_t memory, void* stream) {
  g_last_error.clear();
  if (!A) return fail(GBCG_ERR_INVALID, "null matrix handle");
  if (memory != GBCG_HOST && memory != GBCG_DEVICE) return fail(GBCG_ERR_INVALID, "memory must be GBCG_HOST or GBCG_DEVICE");
  const int64_t nnz = A->nnz_input;
  if (nnz == 0) return GBCG_OK;
  if (!val) return fail(GBCG_ERR_INVALID, "null value array");
  cudaStream_t s = (cudaStream_t)stream;
  if (!A->u_map_main && !A->u_map_long && !A->u_map_diag) {
    // the layout of the same pattern with value k + 1 at input entry k: every
    // device value slot then names the input entry it holds (0: padding)
    std::vector<double> iv(nnz);
    for (int64_t k = 0; k < nnz; ++k) iv[k] = (double)(k + 1);
    LayoutHost L;
    std::string err;
    if (int rc = build_layout(A->format, A->n, nnz, A->h_ptr.data(), A->h_idx.data(), iv.data(), A->index_base, L, err))
      return fail(rc, "rebuilding the value map: " + err);
    SymTilesHost T32, T64;
    if (A->mode == kTiles &&
        (!build_sym_tiles(L, A->grid, TileCaps<float>::kSlot, TileCaps<float>::kEnt, kTileSlices32, T32) ||
         !build_sym_tiles(L, A->grid, TileCaps<double>::kSlot, TileCaps<double>::kEnt, kTileSlices64, T64)))
      return fail(GBCG_ERR_INVALID, "rebuilding the value map: tiles differ from the handle's");
    auto to_map = [](const std::vector<double>& v) {
      std::vector<int32_t> m(v.size());
      for (size_t i = 0; i < v.size(); ++i) m[i] = (int32_t)v[i] - 1;
      return m;
    };
    int64_t& B = A->bytes;
    if (A->mode == kTiles) {
      if ((int64_t)T64.val.size() != A->t64.slots || (int64_t)T32.val.size() != A->t32.slots)
        return fail(GBCG_ERR_INVALID, "value map: tile size mismatch");
      if (int rc = upload(&A->u_map_main, to_map(T64.val), s, B)) return rc;
      A->u_len_main = (int64_t)T64.val.size();
      if (int rc = upload(&A->u_map_t32, to_map(T32.val), s, B)) return rc;
      A->u_len_t32 = (int64_t)T32.val.size();
    } else {
      if (int rc = upload(&A->u_map_main, to_map(L.A.val), s, B)) return rc;
      A->u_len_main = (int64_t)L.A.val.size();
      if (!L.A.long_val.empty()) {
        if (int rc = upload(&A->u_map_long, to_map(L.A.long_val), s, B)) return rc;
        A->u_len_long = (int64_t)L.A.long_val.size();
      }
    }
    if (A->sym) {
      if (int rc = upload(&A->u_map_diag, to_map(L.diag), s, B)) return rc;
      A->u_len_diag = (int64_t)L.diag.size();
    }
    if (int rc = dalloc(&A->u_stage, (size_t)nnz, B)) return rc;
  }
  const double* src = val;
  if (memory == GBCG_HOST) {
    CUDA_TRY(cudaMemcpyAsync(A->u_stage, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    src = A->u_stage;
  }
  auto run = [&](const int32_t* map, int64_t len, double* d64, float* d32) -> int {
    if (!map || len == 0) return 0;
    const int blocks = (int)std::min<int64_t>(4096, (len + 255) / 256);
    k_place_values<<<blocks, 256, 0, s>>>(map, len, src, d64, d32);
    CUDA_TRY(cudaGetLastError());
    return 0;
  };
  if (A->mode == kTiles) {
    if (int rc = run(A->u_map_main, A->u_len_main, (double*)A->t64.val, nullptr)) return rc;
    if (int rc = run(A->u_map_t32, A->u_len_t32, nullptr, (float*)A->t32.val)) return rc;
  } else {
    if (int rc = run(A->u_map_main, A->u_len_main, A->val64, A->val32)) return rc;
    if (int rc = run(A->u_map_long, A->u_len_long, A->long_val64, A->long_val32)) return rc;
  }
  if (A->sym)
    if (int rc = run(A->u_map_diag, A->u_len_diag, A->diag64, A->diag32)) return rc;
  return GBCG_OK;
}

const char* gbcg_status_string(int status) {
  switch (status) {
    case GBCG_OK: return "GBCG_OK";
    case GBCG_ERR_INVALID: return "GBCG_ERR_INVALID";
    case GBCG_ERR_NOT_SPD: return "GBCG_ERR_NOT_SPD";
    case GBCG_ERR_MAXIT: return "GBCG_ERR_MAXIT";
    case GBCG_ERR_NONFINITE: return "GBCG_ERR_NONFINITE";
    case GBCG_ERR_TIMEOUT: return "GBCG_ERR_TIMEOUT";
    case GBCG_ERR_CUDA: return "GBCG_ERR_CUDA";
    case GBCG_ERR_NOMEM: return "GBCG_ERR_NOMEM";
    default: return "GBCG_UNKNOWN_STATUS";
  }
}

const char* gbcg_last_error(void) { return g_last_error.c_str(); }

int gbcg_selftest_wait_timeout(int32_t ctas, int32_t timeout_ms, void* stream) {
  g_last_error.clear();
  if (timeout_ms <= 0 || timeout_ms > 10000) return fail(GBCG_ERR_INVALID, "timeout_ms must be in (0, 10000]");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wait_selftest, 32, 0));
  if (ctas <= 0) ctas = 2 * sms;
  if (ctas < 2 || ctas > per_sm * sms) return fail(GBCG_ERR_INVALID, "ctas out of the co-resident range");
  GridBar* gb = nullptr;
  GridBar* gh = nullptr;
  CUDA_TRY(cudaMalloc(&gb, sizeof(GridBar)));
  if (cudaMallocHost(&gh, sizeof(GridBar)) != cudaSuccess) {
    cudaFree(gb);
    return fail(GBCG_ERR_NOMEM, "cudaMallocHost failed");
  }
  long long tns = (long long)timeout_ms * 1000000LL;
  void* kargs[] = {(void*)&gb, (void*)&tns};
  cudaError_t e = cudaMemsetAsync(gb, 0, sizeof(GridBar), s);
  if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void*)k_wait_selftest, dim3(ctas), dim3(32), kargs, 0, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gh, gb, sizeof(GridBar), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const int st = gh->status;
  cudaFree(gb);
  cudaFreeHost(gh);
  if (e != cudaSuccess) return fail(GBCG_ERR_CUDA, cudaGetErrorString(e));
  if (st == kTimeout) return fail(GBCG_ERR_TIMEOUT, "barrier wait ran out as designed");
  return GBCG_OK;
}

}  // extern "C"
