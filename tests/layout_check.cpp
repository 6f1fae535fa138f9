// layout_check.cpp -- host-side check of the tiled symmetric layout
// (layout.cpp, build_sym_tiles), run by tests/test_layout_tiles.py without a
// GPU.  Reads a symmetric-upper CSR matrix (0-based) from a binary file,
// builds the layout for a given number of CTAs, and checks:
//   - every strict upper entry is stored exactly once, with its value, at
//     position k * R + l of its tile (l = its local row), and every other
//     position of the tile is padding (value 0, padding flag set);
//   - in every round of every tile no two entries target the same slot;
//   - slots, rounds and entries stay within the caps the kernels assume;
//   - each slot names the right column (own rows, then the windows);
//   - every window slot is either carried to the same row's slot in the
//     next tile of the same CTA or flushed as a partial sum; a direct
//     flush run writes the first partial sums of consecutive rows into the
//     dense per-row array (each row at most once), and the incoming runs
//     cover every other flushed partial sum exactly once;
// then replays the kernels' order of operations on the host (rounds,
// accumulators, dense first partials, partial sums, incoming runs) in double
// precision and
// compares y with a row-by-row symmetric product, entry by entry within the
// componentwise rounding bound.  Prints one line of statistics, or FAIL.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../paper_1010_4639_gb300/csrc/layout.h"

using namespace gbcg;

static int fail(const char* what, long long a = -1, long long b = -1) {
  printf("FAIL %s %lld %lld\n", what, a, b);
  return 1;
}

int main(int argc, char** argv) {
  if (argc < 3) return fail("usage: layout_check matrix.bin ctas [max_slices slot_cap ent_cap]");
  FILE* f = fopen(argv[1], "rb");
  if (!f) return fail("open");
  int64_t n = 0, nnz = 0;
  if (fread(&n, 8, 1, f) != 1 || fread(&nnz, 8, 1, f) != 1) return fail("header");
  std::vector<int32_t> ptr(n + 1), idx(nnz);
  std::vector<double> val(nnz), x(n);
  if (fread(ptr.data(), 4, n + 1, f) != (size_t)(n + 1) || fread(idx.data(), 4, nnz, f) != (size_t)nnz ||
      fread(val.data(), 8, nnz, f) != (size_t)nnz || fread(x.data(), 8, n, f) != (size_t)n)
    return fail("body");
  fclose(f);
  const int ctas = atoi(argv[2]);
  const int max_slices = argc > 3 ? atoi(argv[3]) : 15;
  const int slot_cap = argc > 4 ? atoi(argv[4]) : 2048, ent_cap = argc > 5 ? atoi(argv[5]) : 4096;
  LayoutHost L;
  std::string err;
  if (build_layout(1, n, nnz, ptr.data(), idx.data(), val.data(), 0, L, err)) return fail(err.c_str());
  SymTilesHost T;
  if (!build_sym_tiles(L, ctas, slot_cap, ent_cap, max_slices, T)) {
    printf("NOTILES\n");
    return 0;
  }
  // the CTA row ranges do not depend on the caps
  SymTilesHost T15;
  if (!build_sym_tiles(L, ctas, 2048, 4096, 15, T15)) return fail("reference tiles");
  for (int c = 0; c <= ctas; ++c)
    if (T.tile_slice[T.cta_tile[c]] != T15.tile_slice[T15.cta_tile[c]]) return fail("CTA ranges differ", c);
  const int32_t NT = (int32_t)T.tile_ns.size();
  if ((int)T.cta_tile.size() != ctas + 1 || T.cta_tile[ctas] != NT) return fail("cta_tile");
  std::vector<int64_t> seen(L.urc.size(), 0);
  std::vector<double> y(n, 0.0), part(T.tile_ext[NT], 0.0), p1(n, 0.0);
  std::vector<int32_t> p1_hit(n, 0);
  if (T.flush_row.size() != T.flush_src.size()) return fail("flush_row size");
  std::vector<int32_t> win_hit(T.tile_ext[NT], 0), flushed(T.tile_ext[NT], 0);
  int64_t max_d = 0, max_s = 0, pads = 0, stored = 0, carried = 0, max_runs = 0, max_wins = 0;
  std::vector<int> cta_of(NT, -1);
  for (int c = 0; c < ctas; ++c)
    for (int32_t t = T.cta_tile[c]; t < T.cta_tile[c + 1]; ++t) cta_of[t] = c;
  auto columns = [&](int32_t t) {  // slot -> global row of tile t
    const int64_t a = 32 * (int64_t)T.tile_slice[t], b = std::min<int64_t>(n, 32 * (int64_t)T.tile_slice[t + 1]);
    std::vector<int64_t> col(T.tile_ns[t], -1);
    for (int64_t sl = 0; sl < b - a; ++sl) col[sl] = a + sl;
    int64_t sl = T.tile_own[t];
    for (int32_t w = T.tile_win[t]; w < T.tile_win[t + 1]; ++w)
      for (int32_t r = 0; r < T.win_len[w]; ++r) col[sl++] = T.win_start[w] + r;
    return col;
  };
  std::vector<std::pair<int64_t, double>> carry_in;  // (slot, value) for the next tile
  for (int32_t t = 0; t < NT; ++t) {
    const int64_t s0 = T.tile_slice[t], s1 = T.tile_slice[t + 1];
    const int64_t a = 32 * s0, b = std::min<int64_t>(n, 32 * s1), rows = b - a;
    const int64_t D = T.tile_len[t], S = T.tile_ns[t], own = T.tile_own[t];
    const int64_t R = T.tile_stride[t];
    if (s1 - s0 > max_slices || R != 32 * (s1 - s0) || D * R > ent_cap || S > slot_cap || own != ((rows + 3) & ~3))
      return fail("caps", t, D * R);
    const int64_t e0 = T.tile_ent[t], E8 = T.tile_ent[t + 1] - e0, m0 = T.tile_meta[t];
    if (E8 != ((D * R + 7) & ~int64_t(7)) || T.tile_meta[t + 1] - m0 != E8 || (e0 & 7) || (m0 & 7))
      return fail("blob", t);
    // slot -> global column
    std::vector<int64_t> col_of(S, -1);
    for (int64_t sl = 0; sl < rows; ++sl) col_of[sl] = a + sl;
    int64_t sl = own;
    for (int32_t w = T.tile_win[t]; w < T.tile_win[t + 1]; ++w) {
      if ((T.win_start[w] & 3) != 0) return fail("window alignment", t, w);
      for (int32_t r = 0; r < T.win_len[w]; ++r) col_of[sl++] = T.win_start[w] + r;
    }
    if (sl != S) return fail("slot count", t, sl);
    max_d = std::max(max_d, D);
    max_s = std::max(max_s, S);
    // the packed descriptor agrees with the lists
    const TileDesc& dd = T.desc[t];
    if (dd.e0 != e0 || dd.m0 != m0 || dd.row0 != a || dd.ext0 != T.tile_ext[t] || dd.rows != rows ||
        dd.nsl != s1 - s0 || dd.D != D || dd.S != S || dd.own != own || dd.R != R || dd.E8 != E8 ||
        dd.nwin != T.tile_win[t + 1] - T.tile_win[t] || dd.nc != T.tile_carry[t + 1] - T.tile_carry[t] ||
        dd.nf != T.tile_flush[t + 1] - T.tile_flush[t] || dd.win0 != T.tile_win[t] ||
        dd.carry0 != T.tile_carry[t] || dd.flush0 != T.tile_flush[t])
      return fail("descriptor", t);
    for (int w = 0; w < std::min(dd.nwin, kDescWin); ++w)
      if (dd.ws[w] != T.win_start[dd.win0 + w] || dd.wl[w] != T.win_len[dd.win0 + w]) return fail("descriptor windows", t);
    for (int u = 0; u < std::min(dd.nc, kDescRun); ++u)
      if (dd.cs[u] != T.carry_src[dd.carry0 + u] || dd.cd[u] != T.carry_dst[dd.carry0 + u] ||
          dd.cl[u] != T.carry_len[dd.carry0 + u])
        return fail("descriptor carry runs", t);
    for (int u = 0; u < std::min(dd.nf, kDescRun); ++u)
      if (dd.fs[u] != T.flush_src[dd.flush0 + u] || dd.fl[u] != T.flush_len[dd.flush0 + u] ||
          dd.fr[u] != T.flush_row[dd.flush0 + u])
        return fail("descriptor flush runs", t);
    max_runs = std::max<int64_t>(max_runs, std::max(dd.nc, dd.nf));
    max_wins = std::max<int64_t>(max_wins, dd.nwin);
    // entries: the stored ones, once each, in their row; rounds conflict-free
    std::vector<double> acc(S, 0.0), direct(rows, 0.0);
    if (t > 0 && cta_of[t - 1] != cta_of[t] && !carry_in.empty()) return fail("carry across CTAs", t);
    for (auto& cv : carry_in) acc[cv.first] = cv.second;
    carry_in.clear();
    for (int64_t k = 0; k < D; ++k) {
      std::vector<char> used(S, 0);
      for (int64_t l = 0; l < R; ++l) {
        const int64_t e = k * R + l;
        const uint16_t s16 = T.meta[m0 + e];
        const double v = T.val[e0 + e];
        if (s16 & kTilePad) {
          if (v != 0.0 || (s16 & ~kTilePad) != l) return fail("padding", t, e);
          ++pads;
          continue;
        }
        if (l >= rows || s16 >= S) return fail("slot range", t, e);
        if (used[s16]) return fail("round conflict", t, e);
        used[s16] = 1;
        const int64_t i = a + l, j = col_of[s16];
        // find the stored entry (i, j)
        int64_t q = L.urp[i];
        while (q < L.urp[i + 1] && L.urc[q] != j) ++q;
        if (q == L.urp[i + 1] || L.urv[q] != v) return fail("entry", i, j);
        ++seen[q];
        ++stored;
        direct[l] += v * x[j];       // the kernel's FMAs round once; the bound below covers both
        acc[s16] += v * x[i];
      }
    }
    for (int64_t e = D * R; e < E8; ++e)
      if (!(T.meta[m0 + e] & kTilePad) || T.val[e0 + e] != 0.0) return fail("tail padding", t, e);
    for (int64_t l = 0; l < rows; ++l) y[a + l] = L.diag[a + l] * x[a + l] + direct[l] + acc[l];
    // every window slot: carried to the same row in the next tile of the CTA, or flushed
    std::vector<int> fate(S, 0);
    const bool has_next = t + 1 < NT && cta_of[t + 1] == cta_of[t];
    const std::vector<int64_t> next_col = has_next ? columns(t + 1) : std::vector<int64_t>();
    for (int32_t u = T.tile_carry[t]; u < T.tile_carry[t + 1]; ++u)
      for (int32_t i = 0; i < T.carry_len[u]; ++i) {
        const int64_t src = T.carry_src[u] + i, dst = T.carry_dst[u] + i;
        if (!has_next || src < own || src >= S || dst < 0 || dst >= (int64_t)next_col.size() ||
            next_col[dst] != col_of[src])
          return fail("carry", t, src);
        ++fate[src];
        carry_in.push_back({dst, acc[src]});
        ++carried;
      }
    for (int32_t u = T.tile_flush[t]; u < T.tile_flush[t + 1]; ++u)
      for (int32_t i = 0; i < T.flush_len[u]; ++i) {
        const int64_t src = T.flush_src[u] + i;
        if (src < own || src >= S) return fail("flush", t, src);
        ++fate[src];
        if (T.flush_row[u] >= 0) {  // direct: the row's first partial sum, in the dense array
          const int64_t r = (int64_t)T.flush_row[u] + i;
          if (r != col_of[src] || r >= n || p1_hit[r]++ != 0) return fail("direct flush", t, src);
          p1[r] = acc[src];
          continue;
        }
        if (p1_hit[col_of[src]] == 0) return fail("overflow partial before a direct one", t, src);
        part[T.tile_ext[t] + src - own] = acc[src];
        flushed[T.tile_ext[t] + src - own] = 1;
      }
    for (int64_t s2 = own; s2 < S; ++s2)
      if (fate[s2] != 1) return fail("window slot fate", t, s2);
  }
  for (size_t q = 0; q < seen.size(); ++q)
    if (seen[q] != 1) return fail("entry count", (long long)q, seen[q]);
  // incoming runs, in each target tile's fixed order
  for (int32_t t = 0; t < NT; ++t) {
    const int64_t row0 = 32 * (int64_t)T.tile_slice[t];
    for (int32_t u = T.in_ptr[t]; u < T.in_ptr[t + 1]; ++u)
      for (int32_t l = 0; l < T.in_len[u]; ++l) {
        y[row0 + T.in_row[u] + l] += part[T.in_src[u] + l];
        win_hit[T.in_src[u] + l]++;
      }
  }
  int64_t partials = 0, directs = 0;
  for (int64_t i = 0; i < n; ++i) {
    y[i] += p1[i];
    directs += p1_hit[i];
  }
  for (size_t i = 0; i < win_hit.size(); ++i) {
    if (win_hit[i] != flushed[i]) return fail("incoming coverage", (long long)i, win_hit[i]);
    partials += flushed[i];
  }
  // against the row-by-row product, componentwise
  std::vector<double> z(n, 0.0), scale(n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      const int64_t j = idx[k];
      z[i] += val[k] * x[j];
      scale[i] += std::fabs(val[k] * x[j]);
      if (j != i) {
        z[j] += val[k] * x[i];
        scale[j] += std::fabs(val[k] * x[i]);
      }
    }
  for (int64_t i = 0; i < n; ++i)
    if (std::fabs(y[i] - z[i]) > 1e-13 * scale[i]) return fail("product", i);
  // balance of the CTA ranges under the tile cost the partition assumes:
  // the tile's rounds plus six rounds' worth of fixed work, per tile
  double cmax = 0.0, csum = 0.0;
  for (int c = 0; c < ctas; ++c) {
    double cost = 0.0;
    for (int32_t t = T.cta_tile[c]; t < T.cta_tile[c + 1]; ++t) cost += 6.0 + T.tile_len[t];
    cmax = std::max(cmax, cost);
    csum += cost;
  }
  printf("OK tiles=%d max_rounds=%lld max_slots=%lld stored=%lld pads=%lld directs=%lld partials=%lld carried=%lld "
         "max_runs=%lld max_windows=%lld balance=%.4f\n",
         NT, (long long)max_d, (long long)max_s, (long long)stored, (long long)pads, (long long)directs,
         (long long)partials, (long long)carried, (long long)max_runs, (long long)max_wins,
         csum > 0 ? cmax / (csum / ctas) : 1.0);
  return 0;
}
