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
// of the persistent grid, and each range into tiles of at most 16 whole
// slices (one per warp).  A tile's column space -- its own rows (padded to a
// multiple of 4), then 16-byte-aligned windows of the rows beyond it that its
// upper entries reach -- is numbered by 16-bit slots indexing a shared-memory
// copy of x.  Each strict upper entry is stored once (value and slot); entry
// k of the tile's local row l sits at position k * R + l, R a power of two, so
// the row of any position is position & (R - 1) (rows padded to the tile's
// longest row L).  A transpose index lists, for every slot, the positions of
// the entries that target it, in increasing source row: the transpose half
// U'x of a tile is then a gather sum_e val[e] * x[row(e)] over shared memory,
// in a fixed order, without atomics.  Window sums leave the
// tile as partial sums; "incoming runs" list, per target tile and in a fixed
// order, which partial sums to add to which of its rows.
struct SymTilesHost {
  int32_t slot_cap = 0, ent_cap = 0;
  std::vector<int32_t> cta_tile;   // G + 1: tile range of each CTA
  std::vector<int32_t> tile_slice; // T + 1: first slice of each tile
  std::vector<int32_t> tile_ns;    // T: slot count (padded own rows + windows)
  std::vector<int32_t> tile_own;   // T: own rows padded to a multiple of 4
  std::vector<int32_t> tile_len;   // T: padded row length L (entry k of local row l at k * R + l)
  std::vector<int32_t> tile_rlog;  // T: log2 of R = 32 * (slices rounded up to a power of 2)
  std::vector<int64_t> tile_ent;   // T + 1: first entry of each tile (multiples of 8)
  std::vector<int64_t> tile_meta;  // T + 1: first u16 of each tile's index blob (multiples of 8)
  std::vector<int64_t> tile_ext;   // T + 1: first partial sum of each tile
  std::vector<int32_t> tile_win;   // T + 1: window range of each tile
  std::vector<int32_t> win_start;  // global first row of each window
  std::vector<int32_t> win_len;    // rows of each window
  std::vector<double> val;         // entry values (0 on padding)
  std::vector<uint16_t> meta;      // per tile: slots[E8], transpose index[E8], index offsets[S+1 rounded to 8]
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
  SymTilesHost tiles;              // symmetric only, when built
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

// Builds the tiled symmetric layout for `ctas` CTAs, with at most
// `slot_cap` slots and `ent_cap` padded entries per tile.  Returns false
// (layout left empty) when a single slice already exceeds a cap.
bool build_sym_tiles(LayoutHost& L, int ctas, int slot_cap, int ent_cap);

// Contiguous slice ranges for `parts` workers, balanced by stored slots
// (plus plan slots for the symmetric layout).  Returns parts + 1 offsets.
std::vector<int32_t> partition_slices(const LayoutHost& L, int parts);
// Long rows split evenly over `parts` workers (parts + 1 offsets).
std::vector<int32_t> partition_long(const LayoutHost& L, int parts);

}  // namespace gbcg
