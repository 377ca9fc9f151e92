// Test driver for the host-side layout (paper_2511_13894_gb300/csrc/host_prep.cpp):
// reads an LP written by tests/test_host_prep.py, runs prepare_lp, and writes
// its return code and every array of the layout in a tagged binary format.
//
// input (little endian): int64 m, n, nnz, flags (1: lb, 2: ub, 4: sense);
//   int64 row_ptr[m+1]; int32 col[nnz]; f64 val[nnz]; f64 b[m]; f64 c[n];
//   then f64 lb[n], f64 ub[n], int8 sense[m] when flagged
// output: int64 rc; int64 detail length; detail bytes; then records
//   int32 name length, name, int32 type (0 int32, 1 f64, 2 int8), int64 count, data
// With two more arguments (chunk size, SM count) it also writes the chunked
// pass's plan of A' (plan_chunks).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "host_prep.h"

namespace {

template <class T>
bool read_vec(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return n == 0 || std::fread(v.data(), sizeof(T), n, f) == n;
}

template <class T>
void put(FILE* f, const char* name, int type, const T* data, int64_t count) {
  const int32_t len = (int32_t)std::strlen(name);
  std::fwrite(&len, 4, 1, f);
  std::fwrite(name, 1, len, f);
  std::fwrite(&type, 4, 1, f);
  std::fwrite(&count, 8, 1, f);
  if (count > 0) std::fwrite(data, sizeof(T), (size_t)count, f);
}

void put_csr(FILE* f, const std::string& p, const pdhgc::Csr& c) {
  put(f, (p + ".row_ptr").c_str(), 0, c.row_ptr.data(), (int64_t)c.row_ptr.size());
  put(f, (p + ".col").c_str(), 0, c.col.data(), (int64_t)c.col.size());
  put(f, (p + ".val").c_str(), 1, c.val.data(), (int64_t)c.val.size());
  const int32_t seg[3] = {c.cta_rows, c.long_rows, c.nslices};
  put(f, (p + ".seg").c_str(), 0, seg, 3);
  put(f, (p + ".slice_ptr").c_str(), 0, c.slice_ptr.data(), (int64_t)c.slice_ptr.size());
  put(f, (p + ".slice_w").c_str(), 0, c.slice_w.data(), (int64_t)c.slice_w.size());
  put(f, (p + ".sell_map").c_str(), 0, c.sell_map.data(), (int64_t)c.sell_map.size());
  std::vector<int32_t> blocks;
  for (const pdhgc::SellBlock& b : c.sell_blocks) {
    blocks.push_back(b.first);
    blocks.push_back(b.count);
    blocks.push_back(b.k);
    blocks.push_back(b.pad);
  }
  put(f, (p + ".sell_blocks").c_str(), 0, blocks.data(), (int64_t)blocks.size());
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3 && argc != 5) return 2;
  FILE* in = std::fopen(argv[1], "rb");
  if (!in) return 3;
  int64_t hdr[4];
  if (std::fread(hdr, 8, 4, in) != 4) return 4;
  const int64_t m = hdr[0], n = hdr[1], nnz = hdr[2], flags = hdr[3];
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<double> val, b, c, lb, ub;
  std::vector<int8_t> sense;
  bool ok = read_vec(in, row_ptr, (size_t)m + 1) && read_vec(in, col, (size_t)nnz) &&
            read_vec(in, val, (size_t)nnz) && read_vec(in, b, (size_t)m) && read_vec(in, c, (size_t)n);
  if (ok && (flags & 1)) ok = read_vec(in, lb, (size_t)n);
  if (ok && (flags & 2)) ok = read_vec(in, ub, (size_t)n);
  if (ok && (flags & 4)) ok = read_vec(in, sense, (size_t)m);
  std::fclose(in);
  if (!ok) return 5;

  pdhgc::Prepared P;
  std::string detail;
  const int64_t rc = pdhgc::prepare_lp(P, (int32_t)m, (int32_t)n, nnz, row_ptr.data(), col.data(), val.data(),
                                       b.data(), c.data(), (flags & 1) ? lb.data() : nullptr,
                                       (flags & 2) ? ub.data() : nullptr, (flags & 4) ? sense.data() : nullptr,
                                       detail);
  FILE* out = std::fopen(argv[2], "wb");
  if (!out) return 6;
  std::fwrite(&rc, 8, 1, out);
  const int64_t dl = (int64_t)detail.size();
  std::fwrite(&dl, 8, 1, out);
  std::fwrite(detail.data(), 1, detail.size(), out);
  if (rc == 0) {
    put(out, "row_perm", 0, P.row_perm.data(), (int64_t)P.row_perm.size());
    put(out, "col_perm", 0, P.col_perm.data(), (int64_t)P.col_perm.size());
    put(out, "row_inv", 0, P.row_inv.data(), (int64_t)P.row_inv.size());
    put(out, "col_inv", 0, P.col_inv.data(), (int64_t)P.col_inv.size());
    put(out, "b_int", 1, P.b_int.data(), (int64_t)P.b_int.size());
    put(out, "sign", 1, P.sign.data(), (int64_t)P.sign.size());
    put(out, "ge", 2, P.ge.data(), (int64_t)P.ge.size());
    put(out, "c", 1, P.c.data(), (int64_t)P.c.size());
    put(out, "l", 1, P.l.data(), (int64_t)P.l.size());
    put(out, "u", 1, P.u.data(), (int64_t)P.u.size());
    const double norms[2] = {P.b_norm, P.c_norm};
    put(out, "norms", 1, norms, 2);
    put_csr(out, "A", P.A);
    put_csr(out, "AT", P.AT);
    if (argc == 5) {
      pdhgc::ChunkPlan C;
      pdhgc::plan_chunks(P.AT, std::atoi(argv[3]), std::atoi(argv[4]), C);
      const int32_t hdr2[4] = {C.chunk, C.nch, C.blocks, C.nunits};
      put(out, "ch.hdr", 0, hdr2, 4);
      std::vector<int32_t> units;
      for (const pdhgc::ChunkUnit& u : C.units) {
        units.push_back(u.row0);
        units.push_back(u.nrows);
        units.push_back(u.is_long);
      }
      put(out, "ch.units", 0, units.data(), (int64_t)units.size());
      put(out, "ch.uc_off", 0, C.uc_off.data(), (int64_t)C.uc_off.size());
      put(out, "ch.uc_cnt", 0, C.uc_cnt.data(), (int64_t)C.uc_cnt.size());
      put(out, "ch.slot_map", 0, C.slot_map.data(), (int64_t)C.slot_map.size());
      std::vector<int32_t> idx(C.slot_idx.begin(), C.slot_idx.end());
      put(out, "ch.slot_idx", 0, idx.data(), (int64_t)idx.size());
      put(out, "ch.warp_units", 0, C.warp_units.data(), (int64_t)C.warp_units.size());
    }
  }
  std::fclose(out);
  return 0;
}
