// Stateless KKT evaluation of a user point (see kkt_eval.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/pdhgc.h"

namespace pdhgc {

constexpr int kEvBlocks = 1024;  // fixed grid: the reduction order does not depend on the GPU
constexpr int kEvThreads = 256;
constexpr int kEvRowQ = 6;       // partial quantities per block from the rows
constexpr int kEvColQ = 7;       // partial quantities per block from the columns
constexpr int kEvOut = 16;       // doubles of assembled results

struct EvalInput {
  int m, n;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  const double* b;
  const double* c;
  const double* lb;
  const double* ub;
  const int8_t* sense;
  const double* x;
  const double* y;
};

// doubles of scratch one evaluation needs: A'y (n), partials, results
size_t kkt_eval_scratch_doubles(int32_t n);
int kkt_eval_check(int32_t m, int32_t n, int64_t nnz, const void* row_ptr, const void* col_idx, const void* val,
                   const void* b, const void* c, const void* x, const void* y, const pdhgc_report* out,
                   std::string& detail);
// runs the evaluation with `scratch` (kkt_eval_scratch_doubles(n) doubles, device)
int kkt_eval_run(const EvalInput& in, double* scratch, cudaStream_t st, pdhgc_report* out, std::string& detail);

// records the detail string returned by pdhgc_last_error_detail(); returns code
int set_error_detail(int code, const std::string& detail);

}  // namespace pdhgc
