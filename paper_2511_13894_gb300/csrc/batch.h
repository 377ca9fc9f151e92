// Batched solve (see batch.cu): the per-LP result record the device writes.
#pragma once
#include <stdint.h>

namespace pdhgc {

struct BatchReport {
  int32_t status, chosen;
  int64_t iters, restarts;
  double rP2, rD2, rPinf, rDinf, pobj, dobj;
  double p, dd, cand;  // metric counts (off bound, zero reduced cost, candidates)
  double omega, eta, sigma_max, seconds;
};

}  // namespace pdhgc
