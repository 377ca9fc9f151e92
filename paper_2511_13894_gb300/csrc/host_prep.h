// Host-side layout of an LP for the GPU kernels (plain C++, no CUDA).
//
// Rows are renumbered internally by decreasing nnz (stable).  Columns are
// renumbered by decreasing nnz, then (stable, among columns of equal length)
// by decreasing counts of entries in the row-index ranges [0, C), [C, 2C),
// [2C, 3C) with C = kChunkElems64, so that the 32 columns of a slice have
// nearly equal lengths both in total and within each staged chunk of the
// gathered vector (ChunkPlan).  '<' rows are negated into '>' rows (Section
// 2: inequalities handled implicitly); an explicit CSR of A' is built by a
// stable counting sort; and each CSR gets its row segments and SELL-32 slots
// planned.
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
constexpr int kColsPerWarp = 32;     // SELL columns one warp takes (16 measured 1.5-2 us slower per pass)
constexpr int kSellMaxLen = kColsPerWarp * kWarpsPerBlock;  // longest row kept in SELL (256)
constexpr int kWarpMaxLen = 4096;    // longest row given to a single warp
constexpr int kPad = 8;              // trailing padding elements of every device array

// Chunked primal pass (ChunkPlan): the gathered vector is staged in shared
// memory kChunkBytes at a time; one CTA of kChunkThreads threads per SM
constexpr int kChunkBytes = 200 * 1024;
constexpr int kChunkElems32 = kChunkBytes / 4;  // 51,200 FP32 entries per chunk
constexpr int kChunkElems64 = kChunkBytes / 8;  // 25,600 FP64 entries per chunk
constexpr int kChunkThreads = 1024;
constexpr int kChunkWarps = kChunkThreads / 32;
constexpr int kChunkMaxUnits = 8;   // work units one warp owns
constexpr int kChunkLongLen = 128;  // rows longer than this are a unit of their own
constexpr uint16_t kChunkPadIdx = 0xFFFF;  // index of a padding slot

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

// The primal pass over A' (rows = columns j of A, gathered vector of length
// A'.cols = m) with the gathered vector staged in shared memory `chunk`
// entries at a time (nch chunks).  Work units: a row longer than
// kChunkLongLen (its 32 lanes stride over the row's entries in the chunk),
// or a slice of up to 32 consecutive shorter rows (a lane per row; the
// slice's entries in the chunk stored column-major, as wide as its widest
// row there).  Per unit and chunk: the offset and the count (long row) or
// width (slice) of its slots; a slot holds the CSR index of its entry
// (slot_map, -1 for padding) and the entry's index within the chunk
// (slot_idx, kChunkPadIdx for padding).  Units go to the warps of `blocks`
// CTAs (a multiple of the SM count) longest-processing-time first on their
// steps, at most kChunkMaxUnits per warp; warp_units lists them (-1: none).
struct ChunkUnit {
  int32_t row0;
  int32_t nrows;
  int32_t is_long;
  int32_t pad;
};
struct ChunkPlan {
  int32_t chunk = 0, nch = 0, blocks = 0, nunits = 0;
  int64_t nslots = 0;
  std::vector<ChunkUnit> units;
  std::vector<int32_t> uc_off, uc_cnt;  // nunits * nch
  std::vector<int32_t> slot_map;
  std::vector<uint16_t> slot_idx;
  std::vector<int32_t> warp_units;      // blocks * kChunkWarps * kChunkMaxUnits
};

// Plans the chunked pass over `T` (A', rows sorted by decreasing length) for
// chunks of `chunk` (<= 65535) gathered entries on a GPU with `sms` SMs.
void plan_chunks(const struct Csr& T, int32_t chunk, int32_t sms, ChunkPlan& out);

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
