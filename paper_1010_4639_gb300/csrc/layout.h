// layout.h -- host-side construction of the device layouts of a sparse matrix.
//
// Row-gather layout ("SELL-32"): rows are grouped in slices of 32 consecutive
// rows; slice s stores its rows' entries slot-major, i.e. the k-th entry of
// row 32s + l lives at sl_ptr[s] + 32k + l.  One warp computes one slice with
// one lane per row (the paper's thread-per-row "trivial" kernel of Section
// III), and a warp's 32 loads of one slot fall into one contiguous 256-byte
// (double) or 128-byte (int32, float) segment.  Each slice is as long as its
// longest row; shorter rows are padded with zero values whose column is the
// row itself (so the padded load hits a line the row already uses).
//
// Rows much longer than the typical row ("long rows") are taken out of the
// slices and computed warp-per-row from a plain CSR copy, so one long row
// does not pad its 31 neighbours.
//
// Symmetric storage (Section III: A = L + D + U with U' = L) keeps the strict
// upper triangle U in the sliced layout, the diagonal D as a vector, and a
// transpose plan: for every row j, the list of (i, k) with U_ij being the k-th
// stored entry of row i, in increasing i.  The plan is itself sliced, so the
// transpose half U' x is a second row gather that reads U's values in place:
// no entry is stored twice and no floating-point atomics are needed.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace gbcg {

struct SellHost {
  int64_t nslices = 0;
  std::vector<int64_t> sl_ptr;     // nslices + 1, in slots, multiples of 32
  std::vector<int32_t> col;        // slots
  std::vector<int16_t> col16;      // slots: col - row when every slot's offset fits 16 bits (else empty);
                                   // 0 on padding and on lanes past the last row
  std::vector<double> val;         // slots
  std::vector<uint32_t> long_mask; // nslices: lanes whose row is a long row
  std::vector<int32_t> long_row;   // long rows, increasing
  std::vector<int64_t> long_ptr;   // nlong + 1
  std::vector<int32_t> long_col;
  std::vector<double> long_val;
};

struct PlanHost {
  std::vector<int64_t> pl_ptr;     // nslices + 1
  std::vector<int32_t> pl_i;       // source row i
  std::vector<uint16_t> pl_k;      // slot of U_ij in row i; 0xFFFF = padding
};

// Tiled symmetric layout.  Rows are split into contiguous ranges, one per CTA
// of the persistent grid, and each range into tiles of whole slices (up to
// 15 for double precision, one per consumer warp; up to 30 for single
// precision, two per consumer warp).  A tile's column space -- its own rows (padded to a
// multiple of 4), then 16-byte-aligned windows of the rows beyond it that its
// upper entries reach -- is numbered by slots indexing a shared-memory copy
// of x and a shared-memory accumulator.  Each strict upper entry is stored
// once (value and 16-bit slot).  The entries are edge-coloured (rows x slots,
// a bipartite graph) into D rounds, D the larger of the longest row and the
// most-hit slot: in each round a row has at most one entry and a slot
// receives at most one.  Entry (round k, local row l) sits at position
// k * R + l, R = 32 * slices; positions without an entry
// are padding (value 0, slot flagged with kTilePad).  The product runs the
// rounds in order with a barrier between them: each row adds U_ij x_j to its
// own sum (direct half) and U_ij x_i to slot j's accumulator (transpose
// half) -- a scatter without conflicts or atomics, every sum in a fixed
// order.  After a tile, a window slot whose row the next tile of the same
// CTA also covers is carried into that tile's accumulator (carry runs); the
// other window slots leave the tile as partial sums (flush runs).  A row's
// first partial sum goes straight to the row's entry of a dense array (zero
// for rows that never receive one), added by the pass that reads the
// product; further ones go to a compact array, and "incoming runs" list, per
// target tile and in a fixed order, which of those to add to which rows.
constexpr uint16_t kTilePad = 0x8000;  // slot flag of a padding entry (the kernels' kPadSlot)

// Everything the tile pipeline needs about one tile, packed so that the
// producer loads it in one round trip and copies it into the tile's stage.
// Windows and runs beyond the inline capacity are read from the global lists
// (win_start/win_len, carry_*, flush_*) starting at win0, carry0, flush0.
constexpr int kDescWin = 8;  // windows held inline
constexpr int kDescRun = 8;  // carry runs and flush runs held inline
struct alignas(16) TileDesc {
  int64_t e0;                    // first entry of the tile (values; a multiple of 8)
  int64_t m0;                    // first u16 of its slot blob (a multiple of 8)
  int64_t row0;                  // first own row
  int64_t ext0;                  // first partial sum of its window slots
  int32_t rows, nsl, D, S, own, R, E8;  // rows, slices, rounds, slots, padded own rows, round stride, entries
  int32_t nwin, nc, nf;          // windows, carry runs, flush runs
  int32_t win0, carry0, flush0;  // first index of each in the global lists
  int32_t tail;                  // some x slot is not 16-byte aligned: loaded with plain loads
  int32_t pad0_;
  int32_t ws[kDescWin], wl[kDescWin];                   // window start rows and lengths
  uint16_t cs[kDescRun], cd[kDescRun], cl[kDescRun];    // carry runs: slot, slot in the next tile, length
  uint16_t fs[kDescRun], fl[kDescRun];                  // flush runs: slot, length
  int32_t fr[kDescRun];                                 // flush runs: first target row (direct), or -1
  int32_t pad1_[4];
};
static_assert(sizeof(TileDesc) == 288, "tile descriptor size");
// the kernels copy the five run arrays as one block of 5 * kDescRun u16
static_assert(offsetof(TileDesc, fl) == offsetof(TileDesc, cs) + 4 * kDescRun * sizeof(uint16_t) &&
                  offsetof(TileDesc, fr) == offsetof(TileDesc, cs) + 5 * kDescRun * sizeof(uint16_t),
              "run arrays: the kernels copy cs .. fr as one block");

struct SymTilesHost {
  int32_t slot_cap = 0, ent_cap = 0;
  std::vector<int32_t> cta_tile;   // G + 1: tile range of each CTA
  std::vector<int32_t> tile_slice; // T + 1: first slice of each tile
  std::vector<int32_t> tile_ns;    // T: slot count (padded own rows + windows)
  std::vector<int32_t> tile_own;   // T: own rows padded to a multiple of 4
  std::vector<int32_t> tile_len;   // T: rounds D (the round-k entry of local row l at k * R + l)
  std::vector<int32_t> tile_stride;  // T: round stride R = 32 * slices
  std::vector<int64_t> tile_ent;   // T + 1: first entry of each tile (multiples of 8)
  std::vector<int64_t> tile_meta;  // T + 1: first u16 of each tile's index blob (multiples of 8)
  std::vector<int64_t> tile_ext;   // T + 1: first partial sum of each tile
  std::vector<int32_t> tile_win;   // T + 1: window range of each tile
  std::vector<int32_t> win_start;  // global first row of each window
  std::vector<int32_t> win_len;    // rows of each window
  std::vector<double> val;         // entry values (0 on padding)
  std::vector<uint16_t> meta;      // per tile: slots[E8] (kTilePad set on padding)
  std::vector<int32_t> tile_carry; // T + 1: carry runs of each tile
  std::vector<int32_t> carry_src;  // first window slot of the run in the tile
  std::vector<int32_t> carry_dst;  // its slot in the next tile of the same CTA
  std::vector<int32_t> carry_len;
  std::vector<int32_t> tile_flush; // T + 1: flush runs of each tile
  std::vector<int32_t> flush_src;  // first window slot of the run
  std::vector<int32_t> flush_len;
  std::vector<int32_t> flush_row;  // direct run: its first target row (the rows' first partial sums, written
                                   // to a dense per-row array); -1: partial sums tile_ext + slot - own
  std::vector<TileDesc> desc;      // T: packed per-tile descriptor
  std::vector<int32_t> in_ptr;     // T + 1: incoming runs of each tile
  std::vector<int32_t> in_row;     // run start, as a row offset inside the target tile
  std::vector<int32_t> in_len;     // run length
  std::vector<int64_t> in_src;     // first partial-sum index of the run
};

struct LayoutHost {
  int32_t format = 0;
  int64_t n = 0;
  int64_t nnz_input = 0;
  int64_t nnz_full = 0;            // entries of the full operator
  SellHost A;                      // full operator (CSR/CSC) or strict upper U (symmetric)
  std::vector<double> diag;        // symmetric only: nslices * 32, zero padded
  PlanHost plan;                   // symmetric only
  // strict upper rows of the symmetric input (kept for the tile builder)
  std::vector<int64_t> urp;
  std::vector<int32_t> urc;
  std::vector<double> urv;
};

// Validates the input (0- or 1-based) and builds the layout.  Returns 0 or a
// gbcg_status error code, with a message in `err`.
int build_layout(int32_t format, int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                 const double* val, int32_t index_base, LayoutHost& out, std::string& err);

// Checks that a full CSR or CSC input (validated) is exactly symmetric,
// pattern and values: entry (i, j) equals entry (j, i) bit for bit.  O(nnz + n)
// host work (a counting-sort transpose).  Returns 0, or kErrInvalid with the
// first asymmetric entry in `err`.
int check_symmetry(int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx, const double* val,
                   int32_t index_base, std::string& err);

// Builds the tiled symmetric layout of L (symmetric input) into `out` for
// `ctas` CTAs, with at most `max_slices` slices, `slot_cap` slots and
// `ent_cap` padded entries per tile.  The CTA row ranges depend only on L
// and `ctas`, so layouts built with different caps share them.  Returns
// false (`out` left empty) when a single slice already exceeds a cap.
bool build_sym_tiles(const LayoutHost& L, int ctas, int slot_cap, int ent_cap, int max_slices, SymTilesHost& out);

// Contiguous slice ranges for `parts` workers, balanced by stored slots
// (plus plan slots for the symmetric layout).  Returns parts + 1 offsets.
std::vector<int32_t> partition_slices(const LayoutHost& L, int parts);
// Long rows split evenly over `parts` workers (parts + 1 offsets).
std::vector<int32_t> partition_long(const LayoutHost& L, int parts);

}  // namespace gbcg
