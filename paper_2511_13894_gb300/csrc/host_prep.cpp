// Host-side validation and layout of an LP (see host_prep.h).
#include "host_prep.h"

#include <algorithm>
#include <cmath>
#include <numeric>

#include "../../include/pdhgc.h"

namespace pdhgc {

namespace {

std::vector<int32_t> order_by_decreasing(const std::vector<int64_t>& len) {
  std::vector<int32_t> idx(len.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int32_t a, int32_t b) { return len[a] > len[b]; });
  return idx;
}

}  // namespace

void plan_segments(Csr& csr) {
  const int32_t R = csr.rows;
  auto len = [&](int32_t r) { return csr.row_ptr[r + 1] - csr.row_ptr[r]; };
  int32_t r = 0;
  while (r < R && len(r) > kWarpMaxLen) ++r;
  csr.cta_rows = r;
  while (r < R && len(r) > kSellMaxLen) ++r;
  csr.long_rows = r;
  const int32_t short_rows = R - csr.long_rows;
  csr.nslices = (short_rows + kSellH - 1) / kSellH;
  csr.slice_ptr.assign(csr.nslices + 1, 0);
  csr.slice_w.assign(csr.nslices, 0);
  for (int32_t s = 0; s < csr.nslices; ++s) {
    const int32_t w = len(csr.long_rows + s * kSellH);  // the first row is the longest
    csr.slice_w[s] = w;
    csr.slice_ptr[s + 1] = csr.slice_ptr[s] + w * kSellH;
  }
  // K warps per slice, then blocks of 8 / K slices of equal K
  csr.sell_blocks.clear();
  auto warps_for = [](int32_t w) {
    int32_t k = 1;
    while (k < kWarpsPerBlock && k * kColsPerWarp < w) k <<= 1;
    return k;
  };
  for (int32_t s = 0; s < csr.nslices;) {
    const int32_t k = warps_for(csr.slice_w[s]);
    const int32_t per = kWarpsPerBlock / k;
    int32_t cnt = 0;
    while (s + cnt < csr.nslices && cnt < per && warps_for(csr.slice_w[s + cnt]) == k) ++cnt;
    csr.sell_blocks.push_back(SellBlock{s, cnt, k, 0});
    s += cnt;
  }
  csr.sell_map.assign(csr.slice_ptr[csr.nslices], -1);
  for (int32_t s = 0; s < csr.nslices; ++s) {
    for (int32_t t = 0; t < kSellH; ++t) {
      const int32_t row = csr.long_rows + s * kSellH + t;
      if (row >= R) break;
      for (int32_t j = 0; j < len(row); ++j)
        csr.sell_map[csr.slice_ptr[s] + j * kSellH + t] = csr.row_ptr[row] + j;
    }
  }
}

int prepare_lp(Prepared& P, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
               const int32_t* col_idx, const double* val, const double* b, const double* c,
               const double* lb, const double* ub, const int8_t* sense, std::string& detail) {
  if (m < 1 || n < 1 || nnz < 0) {
    detail = "m and n must be >= 1 and nnz >= 0";
    return PDHGC_ERR_INVALID_ARG;
  }
  if (nnz >= (int64_t(1) << 31) - 8) {
    detail = "nnz must be < 2^31";
    return PDHGC_ERR_TOO_LARGE;
  }
  if (!row_ptr || !b || !c || (nnz > 0 && (!col_idx || !val))) {
    detail = "NULL array argument";
    return PDHGC_ERR_INVALID_ARG;
  }
  if (row_ptr[0] != 0 || row_ptr[m] != nnz) {
    detail = "row_ptr[0] must be 0 and row_ptr[m] must equal nnz";
    return PDHGC_ERR_INVALID_CSR;
  }
  for (int32_t i = 0; i < m; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) {
      detail = "row_ptr decreases at row " + std::to_string(i);
      return PDHGC_ERR_INVALID_CSR;
    }
  }
  for (int64_t e = 0; e < nnz; ++e) {
    if (col_idx[e] < 0 || col_idx[e] >= n) {
      detail = "column index out of range at nnz " + std::to_string(e);
      return PDHGC_ERR_INVALID_CSR;
    }
    if (!std::isfinite(val[e])) {
      detail = "non-finite matrix value at nnz " + std::to_string(e);
      return PDHGC_ERR_NONFINITE;
    }
  }
  for (int32_t i = 0; i < m; ++i) {
    if (!std::isfinite(b[i])) {
      detail = "non-finite b at row " + std::to_string(i);
      return PDHGC_ERR_NONFINITE;
    }
    if (sense && sense[i] != '=' && sense[i] != '<' && sense[i] != '>') {
      detail = "sense must be '=', '<' or '>' at row " + std::to_string(i);
      return PDHGC_ERR_INVALID_ARG;
    }
  }
  for (int32_t j = 0; j < n; ++j) {
    if (!std::isfinite(c[j])) {
      detail = "non-finite c at column " + std::to_string(j);
      return PDHGC_ERR_NONFINITE;
    }
    const double lj = lb ? lb[j] : 0.0;
    const double uj = ub ? ub[j] : INFINITY;
    if (std::isnan(lj) || std::isnan(uj) || lj == INFINITY || uj == -INFINITY) {
      detail = "bad bound (NaN, l = +inf or u = -inf) at column " + std::to_string(j);
      return PDHGC_ERR_NONFINITE;
    }
    if (lj > uj) {
      detail = "l > u at column " + std::to_string(j);
      return PDHGC_ERR_BOUNDS;
    }
  }

  P.m = m;
  P.n = n;
  P.nnz = nnz;
  std::vector<int64_t> rlen(m), clen(n, 0);
  for (int32_t i = 0; i < m; ++i) rlen[i] = row_ptr[i + 1] - row_ptr[i];
  for (int64_t e = 0; e < nnz; ++e) clen[col_idx[e]]++;
  P.row_perm = order_by_decreasing(rlen);
  P.col_perm = order_by_decreasing(clen);
  P.row_inv.assign(m, 0);
  P.col_inv.assign(n, 0);
  for (int32_t r = 0; r < m; ++r) P.row_inv[P.row_perm[r]] = r;
  for (int32_t j = 0; j < n; ++j) P.col_inv[P.col_perm[j]] = j;

  // internal A: rows in internal order, entries in the user's order within a row
  Csr& A = P.A;
  A.rows = m;
  A.cols = n;
  A.nnz = nnz;
  A.row_ptr.assign(m + 1, 0);
  A.col.resize(nnz);
  A.val.resize(nnz);
  P.sign.assign(m, 1.0);
  P.ge.assign(m, 0);
  P.b_int.assign(m, 0.0);
  double bn = 0.0;
  for (int32_t i = 0; i < m; ++i) bn += b[i] * b[i];
  P.b_norm = std::sqrt(bn);
  int64_t pos = 0;
  for (int32_t r = 0; r < m; ++r) {
    const int32_t i = P.row_perm[r];
    const char s = sense ? char(sense[i]) : '=';
    const double sg = (s == '<') ? -1.0 : 1.0;
    P.sign[r] = sg;
    P.ge[r] = (s != '=') ? 1 : 0;
    P.b_int[r] = sg * b[i];
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      A.col[pos] = P.col_inv[col_idx[e]];
      A.val[pos] = sg * val[e];
      ++pos;
    }
    A.row_ptr[r + 1] = int32_t(pos);
  }

  // internal A': stable counting sort of A's entries by internal column
  Csr& T = P.AT;
  T.rows = n;
  T.cols = m;
  T.nnz = nnz;
  T.row_ptr.assign(n + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) T.row_ptr[A.col[e] + 1]++;
  for (int32_t j = 0; j < n; ++j) T.row_ptr[j + 1] += T.row_ptr[j];
  std::vector<int32_t> next(T.row_ptr.begin(), T.row_ptr.end() - 1);
  T.col.resize(nnz);
  T.val.resize(nnz);
  for (int32_t r = 0; r < m; ++r) {
    for (int32_t e = A.row_ptr[r]; e < A.row_ptr[r + 1]; ++e) {
      const int32_t j = A.col[e];
      const int32_t q = next[j]++;
      T.col[q] = r;
      T.val[q] = A.val[e];
    }
  }

  P.c.resize(n);
  P.l.resize(n);
  P.u.resize(n);
  double cn = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    const int32_t uj = P.col_perm[j];
    P.c[j] = c[uj];
    P.l[j] = lb ? lb[uj] : 0.0;
    P.u[j] = ub ? ub[uj] : INFINITY;
    cn += c[uj] * c[uj];
  }
  P.c_norm = std::sqrt(cn);
  plan_segments(P.A);
  plan_segments(P.AT);
  return PDHGC_OK;
}

}  // namespace pdhgc
