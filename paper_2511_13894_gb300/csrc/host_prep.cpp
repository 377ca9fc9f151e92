// Host-side validation and layout of an LP (see host_prep.h).
#include "host_prep.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>

#include "../../include/pdhgc.h"

namespace pdhgc {

namespace {

// Runs body(t) for t in [0, parts) on up to `parts` threads (the calling
// thread takes part 0 and any part whose thread could not start).  Each part
// writes only its own outputs, so the result does not depend on the threads.
template <class F>
void run_parts(int parts, const F& body) {
  std::vector<std::thread> th;
  int started = 1;
  try {
    for (; started < parts; ++started) th.emplace_back([&body, started] { body(started); });
  } catch (...) {
  }
  for (int t = started; t < parts; ++t) body(t);
  body(0);
  for (auto& x : th) x.join();
}

// threads for a pass over nnz entries: one per 64k entries, at most 16 and at
// most the machine's
int parts_for(int64_t nnz) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t cap = std::min<int64_t>(16, hw == 0 ? 1 : (int64_t)hw);
  return (int)std::max<int64_t>(1, std::min<int64_t>(cap, nnz / 65536));
}

// splits [0, rows) into `parts` ranges of about equal entry counts (row_ptr
// prefix sums); bounds has parts + 1 entries
template <class RP>
std::vector<int32_t> split_rows(const RP& row_ptr, int32_t rows, int parts) {
  std::vector<int32_t> bounds(parts + 1, rows);
  bounds[0] = 0;
  const int64_t total = (int64_t)row_ptr[rows];
  int32_t r = 0;
  for (int t = 1; t < parts; ++t) {
    const int64_t target = total * t / parts;
    while (r < rows && (int64_t)row_ptr[r] < target) ++r;
    bounds[t] = r;
  }
  return bounds;
}

std::vector<int32_t> order_by_decreasing(const std::vector<int64_t>& len) {
  std::vector<int32_t> idx(len.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int32_t a, int32_t b) { return len[a] > len[b]; });
  return idx;
}

// columns by decreasing length, then by decreasing chunk counts q[.][0..2]
std::vector<int32_t> order_columns(const std::vector<int64_t>& len, const std::vector<int32_t>& q) {
  const size_t n = len.size();
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  // when every length and chunk count fits in 16 bits, the order is that of
  // the 64-bit key (len, q0, q1, q2) descending, stable: a 4-pass LSD radix
  // sort of the indices on the complemented key gives it in linear time
  bool small = true;
  for (size_t j = 0; j < n && small; ++j)
    small = len[j] < 65536 && q[3 * j] < 65536 && q[3 * j + 1] < 65536 && q[3 * j + 2] < 65536;
  if (small) {
    std::vector<uint64_t> key(n);
    for (size_t j = 0; j < n; ++j)
      key[j] = ~(((uint64_t)len[j] << 48) | ((uint64_t)q[3 * j] << 32) | ((uint64_t)q[3 * j + 1] << 16) |
                 (uint64_t)q[3 * j + 2]);
    std::vector<int32_t> tmp(n);
    std::vector<size_t> cnt(65537);
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 16 * pass;
      std::fill(cnt.begin(), cnt.end(), 0);
      for (size_t t = 0; t < n; ++t) cnt[((key[idx[t]] >> shift) & 0xffff) + 1]++;
      for (size_t d = 0; d < 65536; ++d) cnt[d + 1] += cnt[d];
      for (size_t t = 0; t < n; ++t) tmp[cnt[(key[idx[t]] >> shift) & 0xffff]++] = idx[t];
      idx.swap(tmp);
    }
    return idx;
  }
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
    if (len[a] != len[b]) return len[a] > len[b];
    for (int k = 0; k < 3; ++k)
      if (q[3 * (size_t)a + k] != q[3 * (size_t)b + k]) return q[3 * (size_t)a + k] > q[3 * (size_t)b + k];
    return false;
  });
  return idx;
}

}  // namespace

void plan_chunks(const Csr& T, int32_t chunk, int32_t sms, ChunkPlan& P) {
  const int32_t R = T.rows;
  const int32_t G = T.cols;  // gathered length
  P = ChunkPlan{};
  P.chunk = chunk;
  P.nch = G > 0 ? (G + chunk - 1) / chunk : 1;
  const int32_t nch = P.nch;
  auto len = [&](int32_t r) { return T.row_ptr[r + 1] - T.row_ptr[r]; };
  // units: long rows one by one, then slices of 32 rows
  int32_t r = 0;
  while (r < R && len(r) > kChunkLongLen) {
    P.units.push_back(ChunkUnit{r, 1, 1, 0});
    ++r;
  }
  for (; r < R; r += 32) P.units.push_back(ChunkUnit{r, std::min<int32_t>(32, R - r), 0, 0});
  P.nunits = (int32_t)P.units.size();
  P.uc_off.assign((size_t)P.nunits * nch, 0);
  P.uc_cnt.assign((size_t)P.nunits * nch, 0);
  std::vector<int64_t> steps(P.nunits, 0);
  // slot counts per unit and chunk
  std::vector<int32_t> cnt(nch), wid(nch);
  int64_t off = 0;
  for (int32_t u = 0; u < P.nunits; ++u) {
    const ChunkUnit& U = P.units[u];
    std::fill(wid.begin(), wid.end(), 0);
    for (int32_t t = 0; t < U.nrows; ++t) {  // widest row of the unit in each chunk
      std::fill(cnt.begin(), cnt.end(), 0);
      const int32_t row = U.row0 + t;
      for (int32_t e = T.row_ptr[row]; e < T.row_ptr[row + 1]; ++e) cnt[T.col[e] / chunk]++;
      for (int32_t c = 0; c < nch; ++c) wid[c] = std::max(wid[c], cnt[c]);
    }
    for (int32_t c = 0; c < nch; ++c) {
      const int32_t w = wid[c];
      P.uc_off[(size_t)u * nch + c] = (int32_t)off;
      P.uc_cnt[(size_t)u * nch + c] = w;
      off += U.is_long ? w : (int64_t)w * 32;
      steps[u] += U.is_long ? (w + 31) / 32 : w;
    }
    steps[u] += 1;  // the epilogue
  }
  P.nslots = off;
  P.slot_map.assign((size_t)off, -1);
  P.slot_idx.assign((size_t)off, kChunkPadIdx);
  std::vector<int32_t> fill(nch);
  for (int32_t u = 0; u < P.nunits; ++u) {
    const ChunkUnit& U = P.units[u];
    for (int32_t t = 0; t < U.nrows; ++t) {
      std::fill(fill.begin(), fill.end(), 0);
      const int32_t row = U.row0 + t;
      for (int32_t e = T.row_ptr[row]; e < T.row_ptr[row + 1]; ++e) {
        const int32_t c = T.col[e] / chunk;
        const int64_t base = P.uc_off[(size_t)u * nch + c];
        const int64_t s = U.is_long ? base + fill[c] : base + (int64_t)fill[c] * 32 + t;
        fill[c]++;
        P.slot_map[(size_t)s] = e;
        P.slot_idx[(size_t)s] = (uint16_t)(T.col[e] - c * chunk);
      }
    }
  }
  // warps: longest-processing-time first, at most kChunkMaxUnits units per warp
  std::vector<int32_t> order(P.nunits);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return steps[a] > steps[b]; });
  const int32_t per_wave = std::max(1, sms) * kChunkWarps * kChunkMaxUnits;
  int32_t waves = std::max(1, (P.nunits + per_wave - 1) / per_wave);
  while (true) {
    const int32_t blocks = std::max(1, sms) * waves;
    const int32_t W = blocks * kChunkWarps;
    std::vector<int64_t> load(W, 0);
    std::vector<int32_t> nu(W, 0);
    std::vector<int32_t> wu((size_t)W * kChunkMaxUnits, -1);
    // a min-heap of (load, warp) over the warps that still have room
    std::vector<std::pair<int64_t, int32_t>> heap;
    heap.reserve(W);
    for (int32_t w = 0; w < W; ++w) heap.push_back({0, w});
    auto cmp = [](const std::pair<int64_t, int32_t>& a, const std::pair<int64_t, int32_t>& b) {
      return a.first != b.first ? a.first > b.first : a.second > b.second;
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    bool ok = true;
    for (int32_t u : order) {
      if (heap.empty()) {
        ok = false;
        break;
      }
      std::pop_heap(heap.begin(), heap.end(), cmp);
      auto top = heap.back();
      heap.pop_back();
      const int32_t w = top.second;
      wu[(size_t)w * kChunkMaxUnits + nu[w]] = u;
      nu[w]++;
      load[w] += steps[u];
      if (nu[w] < kChunkMaxUnits) {
        heap.push_back({load[w], w});
        std::push_heap(heap.begin(), heap.end(), cmp);
      }
    }
    if (ok) {
      P.blocks = blocks;
      P.warp_units.swap(wu);
      return;
    }
    ++waves;
  }
}

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
  P.row_inv.assign(m, 0);
  for (int32_t r = 0; r < m; ++r) P.row_inv[P.row_perm[r]] = r;
  // per column: entries whose internal row lies in chunk 0, 1, 2 of kChunkElems64 rows
  std::vector<int32_t> q(3 * (size_t)n, 0);
  for (int32_t i = 0; i < m; ++i) {
    const int32_t k = P.row_inv[i] / kChunkElems64;
    if (k >= 3) continue;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) q[3 * (size_t)col_idx[e] + k]++;
  }
  P.col_perm = order_columns(clen, q);
  P.col_inv.assign(n, 0);
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
  // row pointers first (a prefix sum of the internal rows' lengths), then the
  // rows' entries in parallel: each part fills its own rows' slots
  for (int32_t r = 0; r < m; ++r) {
    const int32_t i = P.row_perm[r];
    A.row_ptr[r + 1] = A.row_ptr[r] + int32_t(row_ptr[i + 1] - row_ptr[i]);
  }
  const int parts = parts_for(nnz);
  const std::vector<int32_t> rb = split_rows(A.row_ptr, m, parts);
  run_parts(parts, [&](int t) {
    for (int32_t r = rb[t]; r < rb[t + 1]; ++r) {
      const int32_t i = P.row_perm[r];
      const char s = sense ? char(sense[i]) : '=';
      const double sg = (s == '<') ? -1.0 : 1.0;
      P.sign[r] = sg;
      P.ge[r] = (s != '=') ? 1 : 0;
      P.b_int[r] = sg * b[i];
      int64_t pos = A.row_ptr[r];
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        A.col[pos] = P.col_inv[col_idx[e]];
        A.val[pos] = sg * val[e];
        ++pos;
      }
    }
  });

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
  // each part owns a range of columns (of about equal entry counts) and scans
  // all of A in row order, placing only its columns' entries: every column's
  // entries land in increasing row order, as one sequential pass places them
  const std::vector<int32_t> cb = split_rows(T.row_ptr, n, parts);
  run_parts(parts, [&](int t) {
    const int32_t j0 = cb[t], j1 = cb[t + 1];
    if (j0 >= j1) return;
    for (int32_t r = 0; r < m; ++r) {
      for (int32_t e = A.row_ptr[r]; e < A.row_ptr[r + 1]; ++e) {
        const int32_t j = A.col[e];
        if (j < j0 || j >= j1) continue;
        const int32_t q = next[j]++;
        T.col[q] = r;
        T.val[q] = A.val[e];
      }
    }
  });

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
