// Descriptors shared by the batched solver's host code (batch.cu) and its
// persistent kernel (batch_kernel.cuh, instantiated in batch_k_*.cu): the
// per-LP device view, the phase parameters, and the launch entry points of
// the four kernel instantiations (value type x threads per CTA), each
// compiled in a translation unit of its own so that they build in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "batch.h"

namespace pdhgc {

// ---------------------------------------------------------------------------
// Per-LP device view (all pointers are device addresses of this LP's slices
// of the batch's packed arrays; internal row / column order)
// ---------------------------------------------------------------------------
struct LpDesc {
  int m, n, nnz;
  int gA, gT;         // lanes per row of the A and A' passes in the CSR layout (autotuned)
  int sell;           // 1: passes read the SELL-32 copies; 0: CSR rows with gA / gT lanes
  int smem;           // 1: x_bar and y live in shared memory
  double b_norm, c_norm;
  const int *A_rp, *A_col, *T_rp, *T_col;
  const double *A_val, *T_val;
  double *A_hat, *T_hat;
  float *A_hat32, *T_hat32;
  // SELL-32 copies of the rows with <= kSellMaxLen nonzeros (rows [long, rows))
  int A_long, A_ns, A_slots, T_long, T_ns, T_slots;
  const int *A_sptr, *A_sw, *A_scol, *A_smap, *T_sptr, *T_sw, *T_scol, *T_smap;
  const double *A_sval, *T_sval;
  double *A_shat, *T_shat;
  float *A_shat32, *T_shat32;
  const double *b_int, *c, *l, *u;
  const int8_t* ge;
  int8_t* ge_c;
  double *Dr, *Dc, *rfac, *cfac, *bhat, *chat, *lhat, *uhat;
  double *chat_c, *lhat_c, *uhat_c;
  float *bhat32, *chat32, *lhat32, *uhat32, *chat_c32, *lhat_c32, *uhat_c32;
  double *x, *xbar, *sum_x, *x_r, *y, *sum_y, *y_r;  // FP64 iterates (x_bar, y: global fallback)
  float *x32, *xbar32, *y32;                          // FP32 iterates (global fallback)
  float *x32lo, *y32lo;                               // low parts of the float-float FP32 iterates
  float2 *sx32, *sy32;                                // float-float FP32 running sums
  double *x1, *y1, *xc;
  double *pi_v, *pi_w, *pi_u;
  double* keep;  // eta, sigma_max, ||b_hat||, ||c_hat|| from phase 1 (read by the corner phase)
  const int *row_perm, *col_perm;
  // Halpern loop: T(z) and z - T(z) of a check step (FP64), the chunk's
  // anchoring weights (FP64 and FP32 complements), the float-float anchors
  double *hxp, *hyp, *hdx, *hdy, *hw;
  float* hs;
  float2 *xa32, *ya32;
  // FP32-bulk Halpern loop: the iterate's y (high part; the gathered vector
  // is fl(y - y_0)) and c_hat - A_hat' y_0, b_hat - A_hat x_0 at the anchor
  float* yh32;
  float2 *q32, *r032;
};

struct BatchParams {
  double eps_rel, beta_suff, beta_nec, beta_art, theta, eta_factor, time_limit_s;
  long long max_iters;
  int check_period, ruiz_iters, power_iters;
  // corner
  double eps_abs, c_eps_rel, obj_scale, c_time_limit_s;
  long long c_min_iters, c_max_iters;
  unsigned long long obj_seed;
  int stop_rule;
  int row_rule;
  // inner loop (PDHGC_ALG_*) and the Halpern loop's reflection and PID gains
  int algorithm;
  double rho, pid_kp, pid_ki, pid_kd;
  // tail handoff: once the queue is empty and at most handoff_running LPs are
  // still running, an LP past handoff_min_iters iterations of its phase stops
  // at its next check and is finished on the single-LP path (0: never)
  int handoff_running;
  long long handoff_min_iters;
};

// BatchReport.status of an LP handed to the single-LP path
constexpr int kStatusHandoff = 100;

// cudaFuncSetAttribute (dynamic shared memory) and the resident CTAs per SM
// of k_batch<VT, BT> for `smem` bytes of dynamic shared memory
template <class VT, int BT>
cudaError_t batch_kernel_prepare(size_t smem, int* per_sm);

// launches k_batch<VT, BT> (grid CTAs, BT threads) on stream `st`; phase 0:
// phase 1 (reports in reps), 1: the corner phase (reps), 2: both per LP
// (phase-1 reports in reps, corner reports in reps2)
template <class VT, int BT>
cudaError_t batch_kernel_launch(int grid, size_t smem, cudaStream_t st, const LpDesc* descs, const int* order,
                                int count, int* queue, const BatchParams& bp, int phase, BatchReport* reps,
                                BatchReport* reps2);

}  // namespace pdhgc
