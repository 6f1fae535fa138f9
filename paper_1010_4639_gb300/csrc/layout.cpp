// layout.cpp -- validation and host-side layout construction (see layout.h).
#include "layout.h"

#include <algorithm>
#include <cstring>
#include <cmath>
#include <cstdio>

namespace gbcg {

namespace {

constexpr int kErrInvalid = 1;

// Row lists of the operator to be sliced: row r has entries [rp[r], rp[r+1])
// of (rc, rv).
struct Rows {
  std::vector<int64_t> rp;
  std::vector<int32_t> rc;
  std::vector<double> rv;
};

int validate(int32_t format, int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx, const double* val,
             int32_t base, std::string& err) {
  char buf[256];
  if (n < 0 || nnz < 0) { err = "n and nnz must be non-negative"; return kErrInvalid; }
  if (n > 0x7fffffffLL - 64) { err = "n exceeds the int32 index range"; return kErrInvalid; }
  if (nnz > 0x7fffffffLL) { err = "nnz exceeds 2^31 - 1"; return kErrInvalid; }
  if (base != 0 && base != 1) { err = "index_base must be 0 or 1"; return kErrInvalid; }
  if (format < 0 || format > 2) { err = "unknown format"; return kErrInvalid; }
  if (!ptr || (nnz > 0 && (!idx || !val))) { err = "null array"; return kErrInvalid; }
  if (ptr[0] != base) {
    snprintf(buf, sizeof buf, "ptr[0] = %d, expected index_base %d", ptr[0], base);
    err = buf;
    return kErrInvalid;
  }
  if ((int64_t)ptr[n] - base != nnz) {
    snprintf(buf, sizeof buf, "ptr[n] - index_base = %lld does not match nnz = %lld",
             (long long)ptr[n] - base, (long long)nnz);
    err = buf;
    return kErrInvalid;
  }
  for (int64_t r = 0; r < n; ++r) {
    if (ptr[r + 1] < ptr[r]) {
      snprintf(buf, sizeof buf, "ptr decreases at %lld", (long long)r);
      err = buf;
      return kErrInvalid;
    }
    int64_t prev = -1;
    for (int64_t k = ptr[r] - base; k < ptr[r + 1] - base; ++k) {
      int64_t c = (int64_t)idx[k] - base;
      if (c < 0 || c >= n) {
        snprintf(buf, sizeof buf, "index %d out of range at position %lld", idx[k], (long long)k);
        err = buf;
        return kErrInvalid;
      }
      if (c <= prev) {
        snprintf(buf, sizeof buf, "indices not strictly increasing in line %lld at position %lld", (long long)r,
                 (long long)k);
        err = buf;
        return kErrInvalid;
      }
      if (format == 1 && c < r) {
        snprintf(buf, sizeof buf, "entry (%lld, %lld) below the diagonal in upper-triangle storage", (long long)r,
                 (long long)c);
        err = buf;
        return kErrInvalid;
      }
      if (!std::isfinite(val[k])) {
        snprintf(buf, sizeof buf, "non-finite value at position %lld", (long long)k);
        err = buf;
        return kErrInvalid;
      }
      prev = c;
    }
  }
  return 0;
}

// Slices rows into the SELL-32 layout; rows longer than `long_threshold` go
// to the warp-per-row list when `allow_long`.
void slice_rows(int64_t n, const Rows& R, bool allow_long, SellHost& S) {
  const int64_t ns = (n + 31) / 32;
  S.nslices = ns;
  int64_t maxlen = 0, total = 0;
  for (int64_t r = 0; r < n; ++r) {
    int64_t len = R.rp[r + 1] - R.rp[r];
    maxlen = std::max(maxlen, len);
    total += len;
  }
  const double mean = n > 0 ? (double)total / (double)n : 0.0;
  const int64_t long_threshold = std::max<int64_t>(64, (int64_t)std::ceil(8.0 * mean));
  std::vector<char> is_long(n, 0);
  if (allow_long)
    for (int64_t r = 0; r < n; ++r)
      if (R.rp[r + 1] - R.rp[r] > long_threshold) is_long[r] = 1;
  S.sl_ptr.assign(ns + 1, 0);
  S.long_mask.assign(ns, 0u);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t L = 0;
    for (int l = 0; l < 32; ++l) {
      int64_t r = 32 * s + l;
      if (r >= n) break;
      if (is_long[r]) {
        S.long_mask[s] |= 1u << l;
        continue;
      }
      L = std::max(L, R.rp[r + 1] - R.rp[r]);
    }
    S.sl_ptr[s + 1] = S.sl_ptr[s] + 32 * L;
  }
  const int64_t slots = S.sl_ptr[ns];
  S.col.assign(slots, 0);
  S.val.assign(slots, 0.0);
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t L = (S.sl_ptr[s + 1] - S.sl_ptr[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      int64_t r = 32 * s + l;
      int32_t pad_col = r < n ? (int32_t)r : 0;
      int64_t k = 0;
      if (r < n && !is_long[r])
        for (int64_t q = R.rp[r]; q < R.rp[r + 1]; ++q, ++k) {
          S.col[S.sl_ptr[s] + 32 * k + l] = R.rc[q];
          S.val[S.sl_ptr[s] + 32 * k + l] = R.rv[q];
        }
      for (; k < L; ++k) {
        S.col[S.sl_ptr[s] + 32 * k + l] = pad_col;
        S.val[S.sl_ptr[s] + 32 * k + l] = 0.0;
      }
    }
  }
  // 16-bit column offsets (col - row): a quarter less index traffic for the
  // product when the pattern is banded enough (finite-element matrices in
  // natural order are: offsets up to m^2 + m + 1 on an m^3 grid)
  {
    bool fits = true;
    std::vector<int16_t> c16(slots, 0);
    for (int64_t s = 0; s < ns && fits; ++s) {
      const int64_t L = (S.sl_ptr[s + 1] - S.sl_ptr[s]) / 32;
      for (int l = 0; l < 32 && fits; ++l) {
        const int64_t r = 32 * s + l;
        if (r >= n) continue;  // stays 0: the kernel reads x[0] for lanes past the last row
        for (int64_t k = 0; k < L; ++k) {
          const int64_t off = (int64_t)S.col[S.sl_ptr[s] + 32 * k + l] - r;
          if (off < -32768 || off > 32767) {
            fits = false;
            break;
          }
          c16[S.sl_ptr[s] + 32 * k + l] = (int16_t)off;
        }
      }
    }
    if (fits) S.col16.swap(c16);
    else S.col16.clear();
  }
  S.long_row.clear();
  S.long_ptr.assign(1, 0);
  S.long_col.clear();
  S.long_val.clear();
  for (int64_t r = 0; r < n; ++r) {
    if (!is_long[r]) continue;
    S.long_row.push_back((int32_t)r);
    for (int64_t q = R.rp[r]; q < R.rp[r + 1]; ++q) {
      S.long_col.push_back(R.rc[q]);
      S.long_val.push_back(R.rv[q]);
    }
    S.long_ptr.push_back((int64_t)S.long_col.size());
  }
}

}  // namespace

int check_symmetry(int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx, const double* val,
                   int32_t base, std::string& err) {
  // transpose by a counting sort: column c's entries, in increasing row order
  std::vector<int64_t> tp(n + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) ++tp[(int64_t)idx[k] - base + 1];
  for (int64_t c = 0; c < n; ++c) tp[c + 1] += tp[c];
  std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
  std::vector<int32_t> trow(nnz);
  std::vector<double> tval(nnz);
  for (int64_t r = 0; r < n; ++r)
    for (int64_t k = (int64_t)ptr[r] - base; k < (int64_t)ptr[r + 1] - base; ++k) {
      const int64_t c = (int64_t)idx[k] - base, q = fill[c]++;
      trow[q] = (int32_t)r;
      tval[q] = val[k];
    }
  // row r of the input must equal column r, entry by entry (both sorted)
  char buf[160];
  for (int64_t r = 0; r < n; ++r) {
    const int64_t k0 = (int64_t)ptr[r] - base, k1 = (int64_t)ptr[r + 1] - base;
    if (k1 - k0 != tp[r + 1] - tp[r]) {
      snprintf(buf, sizeof buf, "not symmetric: row %lld has %lld entries, column %lld has %lld", (long long)r,
               (long long)(k1 - k0), (long long)r, (long long)(tp[r + 1] - tp[r]));
      err = buf;
      return kErrInvalid;
    }
    for (int64_t k = k0, q = tp[r]; k < k1; ++k, ++q) {
      const int64_t c = (int64_t)idx[k] - base;
      if (c != trow[q] || !(val[k] == tval[q])) {
        snprintf(buf, sizeof buf, "not symmetric at entry (%lld, %lld)", (long long)r, (long long)c);
        err = buf;
        return kErrInvalid;
      }
    }
  }
  return 0;
}

int build_layout(int32_t format, int64_t n, int64_t nnz, const int32_t* ptr, const int32_t* idx,
                 const double* val, int32_t base, LayoutHost& out, std::string& err) {
  int rc = validate(format, n, nnz, ptr, idx, val, base, err);
  if (rc) return rc;
  out = LayoutHost();
  out.format = format;
  out.n = n;
  out.nnz_input = nnz;
  Rows R;
  R.rp.assign(n + 1, 0);
  if (format == 0) {  // CSR: rows as given
    for (int64_t r = 0; r <= n; ++r) R.rp[r] = (int64_t)ptr[r] - base;
    R.rc.resize(nnz);
    R.rv.assign(val, val + nnz);
    for (int64_t k = 0; k < nnz; ++k) R.rc[k] = idx[k] - base;
    out.nnz_full = nnz;
    slice_rows(n, R, true, out.A);
    return 0;
  }
  if (format == 2) {  // CSC: transpose into rows; a row's entries come in increasing column order
    for (int64_t k = 0; k < nnz; ++k) R.rp[idx[k] - base + 1]++;
    for (int64_t r = 0; r < n; ++r) R.rp[r + 1] += R.rp[r];
    R.rc.resize(nnz);
    R.rv.resize(nnz);
    std::vector<int64_t> fill(R.rp.begin(), R.rp.end() - 1);
    for (int64_t c = 0; c < n; ++c)
      for (int64_t k = ptr[c] - base; k < ptr[c + 1] - base; ++k) {
        int64_t r = idx[k] - base;
        R.rc[fill[r]] = (int32_t)c;
        R.rv[fill[r]] = val[k];
        fill[r]++;
      }
    out.nnz_full = nnz;
    slice_rows(n, R, true, out.A);
    return 0;
  }
  // symmetric upper: D to a vector, strict upper U to slices, transpose plan
  const int64_t ns = (n + 31) / 32;
  out.diag.assign(ns * 32, 0.0);
  int64_t offdiag = 0;
  for (int64_t r = 0; r < n; ++r)
    for (int64_t k = ptr[r] - base; k < ptr[r + 1] - base; ++k) {
      if (idx[k] - base == r)
        out.diag[r] = val[k];
      else
        R.rp[r + 1]++, ++offdiag;
    }
  for (int64_t r = 0; r < n; ++r) R.rp[r + 1] += R.rp[r];
  R.rc.resize(offdiag);
  R.rv.resize(offdiag);
  int64_t maxrow = 0;
  for (int64_t r = 0; r < n; ++r) {
    int64_t q = R.rp[r];
    for (int64_t k = ptr[r] - base; k < ptr[r + 1] - base; ++k)
      if (idx[k] - base != r) {
        R.rc[q] = idx[k] - base;
        R.rv[q] = val[k];
        ++q;
      }
    maxrow = std::max(maxrow, R.rp[r + 1] - R.rp[r]);
  }
  if (maxrow >= 0xFFFF) {
    err = "a row holds 65535 or more upper-triangle entries (symmetric layout limit)";
    return kErrInvalid;
  }
  int64_t ndiag = 0;
  for (int64_t r = 0; r < n; ++r) ndiag += (out.diag[r] != 0.0);
  out.nnz_full = 2 * offdiag + ndiag;
  slice_rows(n, R, false, out.A);
  out.urp = R.rp;
  out.urc = R.rc;
  out.urv = R.rv;
  // transpose plan, row j lists (i, k) for U_ij = k-th entry of row i, i increasing
  std::vector<int64_t> tp(n + 1, 0);
  for (int64_t q = 0; q < offdiag; ++q) tp[R.rc[q] + 1]++;
  for (int64_t r = 0; r < n; ++r) tp[r + 1] += tp[r];
  std::vector<int32_t> ti(offdiag);
  std::vector<uint16_t> tk(offdiag);
  std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = R.rp[i]; q < R.rp[i + 1]; ++q) {
      int64_t j = R.rc[q];
      ti[fill[j]] = (int32_t)i;
      tk[fill[j]] = (uint16_t)(q - R.rp[i]);
      fill[j]++;
    }
  PlanHost& P = out.plan;
  P.pl_ptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t L = 0;
    for (int l = 0; l < 32 && 32 * s + l < n; ++l) L = std::max(L, tp[32 * s + l + 1] - tp[32 * s + l]);
    P.pl_ptr[s + 1] = P.pl_ptr[s] + 32 * L;
  }
  P.pl_i.assign(P.pl_ptr[ns], 0);
  P.pl_k.assign(P.pl_ptr[ns], (uint16_t)0xFFFF);
  for (int64_t s = 0; s < ns; ++s)
    for (int l = 0; l < 32; ++l) {
      int64_t j = 32 * s + l;
      if (j >= n) break;
      int64_t k = 0;
      for (int64_t q = tp[j]; q < tp[j + 1]; ++q, ++k) {
        P.pl_i[P.pl_ptr[s] + 32 * k + l] = ti[q];
        P.pl_k[P.pl_ptr[s] + 32 * k + l] = tk[q];
      }
      for (; P.pl_ptr[s] + 32 * k + l < P.pl_ptr[s + 1]; ++k) P.pl_i[P.pl_ptr[s] + 32 * k + l] = (int32_t)j;
    }
  return 0;
}

namespace {

struct Window {
  int64_t start, len;
};

// Aligned windows covering the sorted targets: each starts on a multiple of
// 4 rows and ends on one (clamped to n); overlapping or adjacent windows merge.
void make_windows(const std::vector<int32_t>& tg, int64_t n, std::vector<Window>& out) {
  out.clear();
  size_t i = 0;
  while (i < tg.size()) {
    int64_t a = tg[i] & ~int64_t(3), b = ((int64_t)tg[i] + 4) & ~int64_t(3);
    size_t j = i + 1;
    while (j < tg.size() && (tg[j] & ~int64_t(3)) <= b) {
      b = std::max<int64_t>(b, ((int64_t)tg[j] + 4) & ~int64_t(3));
      ++j;
    }
    out.push_back({a, std::min<int64_t>(b, n) - a});
    i = j;
  }
}

// Colours the entries of one tile so that, in every colour (round), each
// row has at most one entry and each target slot receives at most one:
// a proper edge colouring of the bipartite graph rows x slots.  By Konig's
// theorem max(row degree, slot degree) colours suffice; edges are coloured
// in order, each taking the lowest colour free at its row, and when that
// colour is taken at its slot the alternating path of the two colours from
// the slot is flipped first (it cannot reach the row).  Returns the colour of
// each edge.
std::vector<int> colour_edges(const std::vector<int32_t>& eu, const std::vector<int32_t>& ev, int nrow, int nslot,
                              int D) {
  const int E = (int)eu.size();
  std::vector<int> col(E, -1);
  std::vector<int32_t> at_u((size_t)nrow * D, -1), at_v((size_t)nslot * D, -1);
  std::vector<int32_t> path;
  for (int e = 0; e < E; ++e) {
    const int u = eu[e], v = ev[e];
    int a = 0;
    while (at_u[(size_t)u * D + a] >= 0) ++a;
    if (at_v[(size_t)v * D + a] >= 0) {
      int b = 0;
      while (at_v[(size_t)v * D + b] >= 0) ++b;
      // the a/b path from slot v: slot -a-> row -b-> slot -a-> ...
      path.clear();
      int cur = v, c = a;
      bool on_slot = true;
      for (;;) {
        const int32_t f = on_slot ? at_v[(size_t)cur * D + c] : at_u[(size_t)cur * D + c];
        if (f < 0) break;
        path.push_back(f);
        cur = on_slot ? eu[f] : ev[f];
        on_slot = !on_slot;
        c = c == a ? b : a;
      }
      for (int32_t f : path) {
        at_u[(size_t)eu[f] * D + col[f]] = -1;
        at_v[(size_t)ev[f] * D + col[f]] = -1;
      }
      for (int32_t f : path) {
        col[f] = col[f] == a ? b : a;
        at_u[(size_t)eu[f] * D + col[f]] = f;
        at_v[(size_t)ev[f] * D + col[f]] = f;
      }
    }
    col[e] = a;
    at_u[(size_t)u * D + a] = e;
    at_v[(size_t)v * D + a] = e;
  }
  return col;
}

}  // namespace

bool build_sym_tiles(const LayoutHost& L, int ctas, int slot_cap, int ent_cap, int max_slices, SymTilesHost& Tl) {
  Tl = SymTilesHost();
  Tl.slot_cap = slot_cap;
  Tl.ent_cap = ent_cap;
  const int64_t n = L.n, ns = (n + 31) / 32;
  const std::vector<int64_t>& rp = L.urp;
  const std::vector<int32_t>& rc = L.urc;
  auto slice_len = [&](int64_t s) {
    int64_t m = 0;
    for (int64_t r = 32 * s; r < std::min<int64_t>(n, 32 * s + 32); ++r) m = std::max(m, rp[r + 1] - rp[r]);
    return m;
  };
  // 1. contiguous slice ranges per CTA, balanced by the work of the rounds:
  // a tile runs one barrier-separated round per entry of its longest row
  // (latency-bound in single precision), plus a fixed part (the stage wait,
  // the clears and the epilogue); a slice's share is its padded entries plus
  // that fixed part.  Measured per single-precision tile of 960 rows on
  // GB300: 269 cycles per round, ~1550 for the rest, i.e. about six rounds'
  // worth (double precision: 640 and ~1930, about three).  Six balances the
  // single-precision product, which the solvers iterate on, and moves the
  // double-precision one by less than 0.1%.  With three, the last CTA ran
  // 9% longer than the others at 256^3; balancing stored entries had given
  // it 1.6 times the tiles of the others.
  std::vector<int64_t> ccut(ctas + 1, ns);
  {
    int64_t total = 0;
    auto work = [&](int64_t s) { return 32 * (slice_len(s) + 6); };
    for (int64_t s = 0; s < ns; ++s) total += work(s);
    int64_t acc = 0, s = 0;
    ccut[0] = 0;
    for (int c = 1; c < ctas; ++c) {
      const long double target = (long double)total * c / ctas;
      while (s < ns && (long double)(acc + work(s)) <= target) acc += work(s++);
      ccut[c] = s;
    }
    ccut[ctas] = ns;
  }
  // targets beyond a candidate tile, its windows and slot count; the largest
  // number of entries any one column receives from the tile's rows
  std::vector<int32_t> tg;
  std::vector<Window> wins;
  std::vector<int32_t> hits(n > 0 ? n : 1, 0);
  int64_t max_hits = 0;
  auto targets = [&](int64_t sa, int64_t sb) {
    const int64_t a = 32 * sa, b = std::min<int64_t>(n, 32 * sb);
    tg.clear();
    max_hits = 0;
    for (int64_t r = a; r < b; ++r)
      for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        if (rc[q] >= b) tg.push_back(rc[q]);
        if (rc[q] != r) max_hits = std::max<int64_t>(max_hits, ++hits[rc[q]]);
      }
    for (int64_t r = a; r < b; ++r)
      for (int64_t q = rp[r]; q < rp[r + 1]; ++q) hits[rc[q]] = 0;
    std::sort(tg.begin(), tg.end());
    tg.erase(std::unique(tg.begin(), tg.end()), tg.end());
    make_windows(tg, n, wins);
    int64_t slots = ((b - a) + 3) & ~int64_t(3);
    for (const Window& w : wins) slots += w.len;
    return slots;
  };
  // rounds of a tile: its longest row or its most-hit column, whichever is more
  auto rounds = [&](int64_t sa, int64_t sb) {
    int64_t lmax = 0;
    for (int64_t s = sa; s < sb; ++s) lmax = std::max(lmax, slice_len(s));
    return std::max(lmax, max_hits);
  };
  auto fits = [&](int64_t sa, int64_t sb) {
    if (sb - sa > max_slices) return false;
    if (targets(sa, sb) > slot_cap) return false;
    return 32 * (sb - sa) * rounds(sa, sb) <= ent_cap;
  };
  // 2. tiles inside each CTA range: the longest prefix that fits
  Tl.cta_tile.assign(ctas + 1, 0);
  int32_t tile_id = 0;
  for (int c = 0; c < ctas; ++c) {
    Tl.cta_tile[c] = tile_id;
    int64_t s = ccut[c];
    while (s < ccut[c + 1]) {
      if (!fits(s, s + 1)) {
        Tl = SymTilesHost();
        return false;
      }
      int64_t e = s + 1;
      while (e < ccut[c + 1] && fits(s, e + 1)) ++e;
      Tl.tile_slice.push_back((int32_t)s);
      ++tile_id;
      s = e;
    }
  }
  Tl.cta_tile[ctas] = tile_id;
  Tl.tile_slice.push_back((int32_t)ns);
  const int32_t T = tile_id;
  // 3. per tile: windows, slot map, entries in conflict-free rounds
  Tl.tile_ns.assign(T, 0);
  Tl.tile_own.assign(T, 0);
  Tl.tile_len.assign(T, 0);
  Tl.tile_stride.assign(T, 0);
  Tl.tile_ent.assign(T + 1, 0);
  Tl.tile_meta.assign(T + 1, 0);
  Tl.tile_ext.assign(T + 1, 0);
  Tl.tile_win.assign(T + 1, 0);
  std::vector<int32_t> slot_of(n > 0 ? n : 1, -1);
  auto up8 = [](int64_t v) { return (v + 7) & ~int64_t(7); };
  std::vector<int32_t> eu, ev;
  std::vector<int64_t> eq;
  for (int32_t t = 0; t < T; ++t) {
    const int64_t s0 = Tl.tile_slice[t], s1 = Tl.tile_slice[t + 1];
    const int64_t a = 32 * s0, b = std::min<int64_t>(n, 32 * s1);
    const int64_t S = targets(s0, s1);
    const int32_t own = (int32_t)(((b - a) + 3) & ~int64_t(3));
    const int64_t D = rounds(s0, s1);
    Tl.tile_ns[t] = (int32_t)S;
    Tl.tile_own[t] = own;
    Tl.tile_len[t] = (int32_t)D;
    const int64_t R = 32 * (s1 - s0);
    Tl.tile_stride[t] = (int32_t)R;
    Tl.tile_ext[t + 1] = Tl.tile_ext[t] + (S - own);
    Tl.tile_win[t + 1] = Tl.tile_win[t] + (int32_t)wins.size();
    int32_t slot0 = own;
    for (const Window& w : wins) {
      Tl.win_start.push_back((int32_t)w.start);
      Tl.win_len.push_back((int32_t)w.len);
      for (int64_t r = w.start; r < w.start + w.len; ++r) slot_of[r] = slot0 + (int32_t)(r - w.start);
      slot0 += (int32_t)w.len;
    }
    // the strict upper entries as edges (local row, target slot), rows in
    // increasing order and each row's entries by increasing column
    eu.clear();
    ev.clear();
    eq.clear();
    for (int64_t r = a; r < b; ++r)
      for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
        const int64_t c = rc[q];
        eu.push_back((int32_t)(r - a));
        ev.push_back((int32_t)(c < b ? c - a : slot_of[c]));
        eq.push_back(q);
      }
    const std::vector<int> colour = colour_edges(eu, ev, (int)(b - a), (int)S, (int)std::max<int64_t>(D, 1));
    const int64_t E = R * D, E8 = up8(E);
    const int64_t e0 = Tl.tile_ent[t];
    Tl.tile_ent[t + 1] = e0 + E8;
    Tl.val.resize(e0 + E8, 0.0);
    // blob: slots[E8]; entry e = k * R + l holds the round-k entry of local
    // row l; a position without one is padding: value 0, slot l | kTilePad
    const int64_t m0 = Tl.tile_meta[t];
    Tl.tile_meta[t + 1] = m0 + E8;
    Tl.meta.resize(m0 + E8, 0);
    for (int64_t e = 0; e < E8; ++e) Tl.meta[m0 + e] = (uint16_t)((e % R) | kTilePad);
    for (size_t i = 0; i < eu.size(); ++i) {
      const int64_t e = (int64_t)colour[i] * R + eu[i];
      Tl.meta[m0 + e] = (uint16_t)ev[i];
      Tl.val[e0 + e] = L.urv[eq[i]];
    }
  }
  // 4. what becomes of each window slot after its tile: a row that the next
  // tile of the same CTA also covers (as an own row or in a window) is
  // carried into that tile's accumulator; the others leave as partial sums.
  // A row's first partial sum (in tile order) is written straight to the
  // row's entry of a dense array, which the pass that reads the product adds
  // ("direct" flush runs); any further one (only where the sources of a row
  // span two CTAs) goes to the compact partial-sum array and is added to its
  // row by the tile that owns it ("incoming runs")
  std::vector<int32_t> tile_of_slice(ns, 0);
  for (int32_t t = 0; t < T; ++t)
    for (int64_t s = Tl.tile_slice[t]; s < Tl.tile_slice[t + 1]; ++s) tile_of_slice[s] = t;
  std::vector<int32_t> cta_of_tile(T, 0);
  for (int c = 0; c < ctas; ++c)
    for (int32_t t = Tl.cta_tile[c]; t < Tl.cta_tile[c + 1]; ++t) cta_of_tile[t] = c;
  auto slot_in = [&](int32_t u, int64_t r) -> int64_t {  // slot of row r in tile u, or -1
    const int64_t a = 32 * (int64_t)Tl.tile_slice[u], b = std::min<int64_t>(n, 32 * (int64_t)Tl.tile_slice[u + 1]);
    if (r >= a && r < b) return r - a;
    int64_t sl = Tl.tile_own[u];
    for (int32_t w = Tl.tile_win[u]; w < Tl.tile_win[u + 1]; ++w) {
      if (r >= Tl.win_start[w] && r < (int64_t)Tl.win_start[w] + Tl.win_len[w]) return sl + r - Tl.win_start[w];
      sl += Tl.win_len[w];
    }
    return -1;
  };
  struct Run {
    int32_t tgt;
    int32_t row;
    int32_t len;
    int64_t src;
  };
  std::vector<Run> runs;
  std::vector<char> has_direct(n > 0 ? n : 1, 0);
  Tl.tile_carry.assign(T + 1, 0);
  Tl.tile_flush.assign(T + 1, 0);
  for (int32_t t = 0; t < T; ++t) {
    const int32_t next = (t + 1 < Tl.cta_tile[cta_of_tile[t] + 1]) ? t + 1 : -1;
    int64_t sl = Tl.tile_own[t];
    for (int32_t w = Tl.tile_win[t]; w < Tl.tile_win[t + 1]; ++w)
      for (int64_t r = Tl.win_start[w]; r < (int64_t)Tl.win_start[w] + Tl.win_len[w]; ++r, ++sl) {
        const int64_t dst = next >= 0 ? slot_in(next, r) : -1;
        if (dst >= 0) {
          const size_t m = Tl.carry_src.size();
          if (m > (size_t)Tl.tile_carry[t] && Tl.carry_src[m - 1] + Tl.carry_len[m - 1] == sl &&
              Tl.carry_dst[m - 1] + Tl.carry_len[m - 1] == dst)
            ++Tl.carry_len[m - 1];
          else {
            Tl.carry_src.push_back((int32_t)sl);
            Tl.carry_dst.push_back((int32_t)dst);
            Tl.carry_len.push_back(1);
          }
          continue;
        }
        const bool direct = !has_direct[r];
        has_direct[r] = 1;
        const int32_t frow = direct ? (int32_t)r : -1;
        const size_t m = Tl.flush_src.size();
        if (m > (size_t)Tl.tile_flush[t] && Tl.flush_src[m - 1] + Tl.flush_len[m - 1] == sl &&
            (direct ? Tl.flush_row[m - 1] >= 0 && Tl.flush_row[m - 1] + Tl.flush_len[m - 1] == r
                    : Tl.flush_row[m - 1] < 0))
          ++Tl.flush_len[m - 1];
        else {
          Tl.flush_src.push_back((int32_t)sl);
          Tl.flush_len.push_back(1);
          Tl.flush_row.push_back(frow);
        }
        if (direct) continue;
        // a further partial sum (index tile_ext[t] + slot - own) goes to the tile owning row r
        const int32_t tt = tile_of_slice[r / 32];
        const int64_t trow0 = 32 * (int64_t)Tl.tile_slice[tt];
        const int64_t src = Tl.tile_ext[t] + sl - Tl.tile_own[t];
        if (!runs.empty() && runs.back().tgt == tt && trow0 + runs.back().row + runs.back().len == r &&
            runs.back().src + runs.back().len == src)
          ++runs.back().len;
        else
          runs.push_back({tt, (int32_t)(r - trow0), 1, src});
      }
    Tl.tile_carry[t + 1] = (int32_t)Tl.carry_src.size();
    Tl.tile_flush[t + 1] = (int32_t)Tl.flush_src.size();
  }
  std::stable_sort(runs.begin(), runs.end(), [](const Run& x, const Run& y) { return x.tgt < y.tgt; });
  Tl.in_ptr.assign(T + 1, 0);
  for (const Run& r : runs) Tl.in_ptr[r.tgt + 1]++;
  for (int32_t t = 0; t < T; ++t) Tl.in_ptr[t + 1] += Tl.in_ptr[t];
  Tl.in_row.resize(runs.size());
  Tl.in_len.resize(runs.size());
  Tl.in_src.resize(runs.size());
  for (size_t i = 0; i < runs.size(); ++i) {
    Tl.in_row[i] = runs[i].row;
    Tl.in_len[i] = runs[i].len;
    Tl.in_src[i] = runs[i].src;
  }
  // 5. the packed descriptors
  Tl.desc.assign(T, TileDesc());
  for (int32_t t = 0; t < T; ++t) {
    TileDesc& d = Tl.desc[t];
    memset(&d, 0, sizeof d);
    const int64_t a = 32 * (int64_t)Tl.tile_slice[t], b = std::min<int64_t>(n, 32 * (int64_t)Tl.tile_slice[t + 1]);
    d.e0 = Tl.tile_ent[t];
    d.m0 = Tl.tile_meta[t];
    d.row0 = a;
    d.ext0 = Tl.tile_ext[t];
    d.rows = (int32_t)(b - a);
    d.nsl = Tl.tile_slice[t + 1] - Tl.tile_slice[t];
    d.D = Tl.tile_len[t];
    d.S = Tl.tile_ns[t];
    d.own = Tl.tile_own[t];
    d.R = Tl.tile_stride[t];
    d.E8 = (int32_t)(Tl.tile_ent[t + 1] - Tl.tile_ent[t]);
    d.nwin = Tl.tile_win[t + 1] - Tl.tile_win[t];
    d.nc = Tl.tile_carry[t + 1] - Tl.tile_carry[t];
    d.nf = Tl.tile_flush[t + 1] - Tl.tile_flush[t];
    d.win0 = Tl.tile_win[t];
    d.carry0 = Tl.tile_carry[t];
    d.flush0 = Tl.tile_flush[t];
    d.tail = (d.rows & 3) != 0;
    for (int32_t w = 0; w < d.nwin; ++w) {
      const int32_t ws = Tl.win_start[d.win0 + w], wl = Tl.win_len[d.win0 + w];
      if ((ws | wl) & 3) d.tail = 1;
      if (w < kDescWin) {
        d.ws[w] = ws;
        d.wl[w] = wl;
      }
    }
    for (int32_t u = 0; u < std::min(d.nc, kDescRun); ++u) {
      d.cs[u] = (uint16_t)Tl.carry_src[d.carry0 + u];
      d.cd[u] = (uint16_t)Tl.carry_dst[d.carry0 + u];
      d.cl[u] = (uint16_t)Tl.carry_len[d.carry0 + u];
    }
    for (int32_t u = 0; u < std::min(d.nf, kDescRun); ++u) {
      d.fs[u] = (uint16_t)Tl.flush_src[d.flush0 + u];
      d.fl[u] = (uint16_t)Tl.flush_len[d.flush0 + u];
      d.fr[u] = Tl.flush_row[d.flush0 + u];
    }
  }
  return true;
}

std::vector<int32_t> partition_slices(const LayoutHost& L, int parts) {
  const int64_t ns = L.A.nslices;
  std::vector<int32_t> cut(parts + 1, 0);
  // A slice costs its slots plus a fixed part: the warp's dependent round
  // trips to memory (stage wait, gathers, row update), measured on GB300 as
  // about 350 slots' worth; and the vector passes over its 32 rows.
  auto work = [&](int64_t s) {
    int64_t w = (L.A.sl_ptr[s + 1] - L.A.sl_ptr[s]) + 352;
    if (!L.plan.pl_ptr.empty()) w += L.plan.pl_ptr[s + 1] - L.plan.pl_ptr[s];
    return w;
  };
  int64_t total = 0;
  for (int64_t s = 0; s < ns; ++s) total += work(s);
  int64_t acc = 0, s = 0;
  for (int p = 1; p < parts; ++p) {
    const long double target = (long double)total * p / parts;
    while (s < ns && (long double)(acc + work(s)) <= target) acc += work(s++);
    cut[p] = (int32_t)s;
  }
  cut[parts] = (int32_t)ns;
  return cut;
}

std::vector<int32_t> partition_long(const LayoutHost& L, int parts) {
  const int64_t nl = (int64_t)L.A.long_row.size();
  std::vector<int32_t> cut(parts + 1);
  for (int p = 0; p <= parts; ++p) cut[p] = (int32_t)(nl * p / parts);
  return cut;
}

}  // namespace gbcg
