// Host-side layout of an LP for the GPU kernels (plain C++, no CUDA).
//
// Rows and columns are renumbered internally by decreasing nnz (stable), so
// that the 32 rows of a warp have nearly equal lengths; '<' rows are negated
// into '>' rows (Section 2: inequalities handled implicitly); an explicit CSR
// of A' is built by a stable counting sort; and each CSR gets its row
// segments and SELL-32 slots planned.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pdhgc {

// Row segments of a CSR whose rows are sorted by decreasing length:
//   rows [0, cta_rows)           longer than kWarpMaxLen: one CTA per row
//   rows [cta_rows, long_rows)   longer than kSellMaxLen: one warp per row
//   rows [long_rows, rows)       SELL-32: slices of 32 consecutive rows stored
//                                column-major (element j of the slice's 32 rows
//                                contiguous), each slice as wide as its first
//                                (longest) row; a lane owns one row, and the
//                                slice's columns are split over K warps
//                                (K = 1, 2, 4 or 8, at most kColsPerWarp
//                                columns each) whose partial row sums are
//                                added in shared memory in warp order
constexpr int kBlock = 256;          // threads per CTA of the SpMV kernel
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kSellH = 32;           // rows per slice (one warp)
constexpr int kColsPerWarp = 16;     // SELL columns one warp takes
constexpr int kSellMaxLen = kColsPerWarp * kWarpsPerBlock;  // longest row kept in SELL (128)
constexpr int kWarpMaxLen = 4096;    // longest row given to a single warp
constexpr int kPad = 8;              // trailing padding elements of every device array

// one CTA of SELL work: slices [first, first + count), K warps per slice
struct SellBlock {
  int32_t first;
  int32_t count;
  int32_t k;
  int32_t pad;
};

struct Csr {
  int32_t rows = 0, cols = 0;
  int64_t nnz = 0;
  std::vector<int32_t> row_ptr;  // rows + 1
  std::vector<int32_t> col;      // nnz
  std::vector<double> val;       // nnz
  // segments
  int32_t cta_rows = 0, long_rows = 0, nslices = 0;
  std::vector<int32_t> slice_ptr;  // nslices + 1 element offsets (multiples of 32)
  std::vector<int32_t> slice_w;    // nslices
  std::vector<int32_t> sell_map;   // slice_ptr[nslices]: CSR index of each slot, -1 = padding
  std::vector<SellBlock> sell_blocks;
  int32_t nb_cta() const { return cta_rows; }
  int32_t nb_warp() const { return (long_rows - cta_rows + kWarpsPerBlock - 1) / kWarpsPerBlock; }
  int32_t nb_sell() const { return (int32_t)sell_blocks.size(); }
  int32_t nblocks() const { return nb_cta() + nb_warp() + nb_sell(); }
};

struct Prepared {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  std::vector<int32_t> row_perm, row_inv;  // internal -> user, user -> internal
  std::vector<int32_t> col_perm, col_inv;
  Csr A, AT;                               // internal numbering, '<' rows negated
  std::vector<double> b_int;               // sign * b, internal row order
  std::vector<double> sign;                // -1 for user '<' rows, internal order
  std::vector<int8_t> ge;                  // 1 for an inequality row, internal order
  std::vector<double> c, l, u;             // internal column order
  double b_norm = 0.0;                     // ||b||_2 of the user's b
  double c_norm = 0.0;                     // ||c||_2 of the user's c
};

// Validates and lays out host arrays.  Returns 0 or a negative PDHGC_ERR_*
// code and sets `detail`.
int prepare_lp(Prepared& out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
               const int32_t* col_idx, const double* val, const double* b, const double* c,
               const double* lb, const double* ub, const int8_t* sense, std::string& detail);

// Plans the row segments and the SELL-32 slots of a CSR whose rows are
// sorted by decreasing length.
void plan_segments(Csr& csr);

}  // namespace pdhgc
