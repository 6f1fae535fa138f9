// layout.cpp -- validation and host-side layout construction (see layout.h).
#include "layout.h"

#include <algorithm>
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

std::vector<int32_t> partition_slices(const LayoutHost& L, int parts) {
  const int64_t ns = L.A.nslices;
  std::vector<int32_t> cut(parts + 1, 0);
  auto work = [&](int64_t s) {
    int64_t w = (L.A.sl_ptr[s + 1] - L.A.sl_ptr[s]) + 32;  // slots + vector work of 32 rows
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
