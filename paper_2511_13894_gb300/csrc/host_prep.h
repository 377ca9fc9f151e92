// Host-side layout of an LP for the GPU kernels (plain C++, no CUDA).
//
// Rows and columns are renumbered internally by decreasing nnz (stable), so
// that consecutive rows handled by one warp have nearly equal lengths; '<'
// rows are negated into '>' rows (Section 2: inequalities handled
// implicitly); an explicit CSR of A' is built by a stable counting sort; and
// each CSR is cut into row tiles for the SpMV kernels.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pdhgc {

// Tile kinds, chosen per tile from the longest row in it:
//   lanes = 0      one whole CTA per row (row longer than kLongRow)
//   lanes = g > 0  g lanes per row (g a power of two <= 32), the tile's
//                  values and column indices staged in shared memory
constexpr int kBlock = 256;          // threads per CTA of every tile kernel
constexpr int kTileNnz = 2048;       // nnz staged per tile
constexpr int kLongRow = 1024;       // rows longer than this get a CTA each
constexpr int kLaneWork = 32;        // target nnz per lane in a staged tile

struct Tile {
  int32_t row0;    // first (internal) row
  int32_t nrows;   // rows in the tile
  int32_t lanes;   // lanes per row; 0 = CTA per row
  int32_t pad;
};

struct Csr {
  int32_t rows = 0, cols = 0;
  int64_t nnz = 0;
  std::vector<int32_t> row_ptr;  // rows + 1
  std::vector<int32_t> col;      // nnz
  std::vector<double> val;       // nnz
  std::vector<Tile> tiles;
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

// Cuts a CSR (rows sorted by decreasing length) into tiles.
void plan_tiles(Csr& csr);

}  // namespace pdhgc
