// Device code of the PDHG + corner-push path (sm_103a).
//
// Every matrix pass is one SpMV launch over the row segments of host_prep.h
// (SELL-32 slices for short rows, a warp or a CTA per long row) with a fused
// epilogue (projection, extrapolation, running sums, residuals) and per-block
// partial sums for the KKT reductions, which a single CTA later folds in a
// fixed order: every reduction is deterministic run to run.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/pdhgc.h"
#include "host_prep.h"

namespace pdhgc {

// ---------------------------------------------------------------------------
// Device scalar state of one phase.  Written only by the single-thread
// control kernels (init / pre-check / decide) between matrix passes.
// ---------------------------------------------------------------------------
struct Scalars {
  double eta, omega, tau, sigma, sigma_max;
  double kkt_r, kkt_prev, inv_t;
  double eps_rel, beta_suff, beta_nec, beta_art, theta, time_limit_s;
  double nb, nc;           // ||b||_2 of the user's b; ||c||_2 of the phase's (unscaled) objective
  double nb_hat, nc_hat;   // ||b_hat||, ||c_hat|| (initial primal weight)
  long long k, t, restarts, chunks, max_chunks, max_iters, min_iters;
  unsigned long long t0_ns, t1_ns;
  int check_period, phase, stop_rule, done, status, chosen, restart_to;
  int at_check, at_limit, pi_zero, error;
  // last evaluation of the current (0) and average (1) point
  double kkt[2], rel_p[2], rel_d[2], rel_gap[2], rel_kkt[2], rP2[2], rD2[2];
  // Halpern loop (algorithm == PDHGC_ALG_HALPERN): reflection, PID gains,
  // fixed-point residual of the last check, of the anchor and of the
  // previous check in this epoch, PID integral and last error
  int algorithm;
  double rho, pid_kp, pid_ki, pid_kd;
  double fpr, fpr0, fpr_prev, pid_int, pid_eprev;
};


// DevModel::ge: 0 for an '=' row, 1 for a '>' row (y >= 0), kRowDualZero for
// a row whose dual is fixed at 0 (the dual corner push's inactive rows: the
// projection returns y = 0 and the row's primal residual counts as 0)
constexpr int8_t kRowDualZero = 2;

struct DevModel {
  const double* chat;
  const double* lhat;
  const double* uhat;
  const double* bhat;
  const double* Dr;
  const double* Dc;
  const int8_t* ge;
};

struct DevIter {
  double* x;
  double* y;
  double* xbar;
  double* sum_x;
  double* sum_y;
  double* x_r;
  double* y_r;
};

// Halpern loop buffers: the PDHG output T(z) = (xp, yp) of a check step and
// z - T(z) = (dx, dy); hw[i] = (t + i + 1) / (t + i + 2), the anchoring
// weight of step i of the next chunk (t = steps since the anchor), and
// hs[i] = 1 - hw[i] = 1 / (t + i + 2) in FP32 for the FP32-bulk steps.  The
// anchor is DevIter::x_r / y_r (FP64) and DevIter32::xa / ya (FP32 bulk).
struct DevHalpern {
  double* xp;
  double* yp;
  double* dx;
  double* dy;
  double* hw;
  float* hs;
};


// ---------------------------------------------------------------------------
// Accumulators
// ---------------------------------------------------------------------------
template <int NV>
struct SumD {
  double v[NV];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0.0;
  }
  __device__ __forceinline__ void add(const SumD& o) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += o.v[i];
  }
  __device__ __forceinline__ SumD shfl_xor(unsigned mask, int off) const {
    SumD r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = __shfl_xor_sync(mask, v[i], off);
    return r;
  }
};

struct MaxD {
  double v[1];
  __device__ __forceinline__ void zero() { v[0] = 0.0; }
  __device__ __forceinline__ void add(const MaxD& o) { v[0] = fmax(v[0], o.v[0]); }
  __device__ __forceinline__ MaxD shfl_xor(unsigned mask, int off) const {
    MaxD r;
    r.v[0] = __shfl_xor_sync(mask, v[0], off);
    return r;
  }
};

// Ordering key of a (non-NaN) double as a signed 64-bit integer: clamps of
// the iteration epilogues are done on the integer pipe, sparing the FP64 unit
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffll;
}
__device__ __forceinline__ double clamp_i(double x, double lo, double hi) {
  const long long k = dkey(x);
  if (k < dkey(lo)) return lo;
  if (k > dkey(hi)) return hi;
  return x;
}

// z = projection of lam onto the cone the finite bounds allow (Section 2)
__device__ __forceinline__ double proj_dual(double lam, double l, double u) {
  const bool lf = l != -INFINITY, uf = u != INFINITY;
  if (lf && uf) return lam;
  if (lf) return fmax(lam, 0.0);
  if (uf) return fmin(lam, 0.0);
  return 0.0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The decision made at a check, from the 22 folded KKT quantities q
// (rows: 5 per point, cur then avg; columns: 6 per point): the Section 2
// ratios and the omega-weighted KKT of both points, then termination (the
// Section 2 test in phase 1, the Section 3.1 rule in the corner phase),
// limits, and the adaptive restart with its primal-weight update.
// mode 0 only records KKT_omega of the start point as the restart reference.
// Runs on one thread; shared by the graph-driven and the batched solvers.
__device__ inline void decide_step(Scalars* S, const double* q, int mode) {

  double nrp2[2], nrd2[2], gap[2], dx2[2], dy2[2];
  const double om = S->omega;
  for (int w = 0; w < 2; ++w) {
    nrp2[w] = q[5 * w + 0];
    const double rP2 = sqrt(q[5 * w + 1]);
    const double by = q[5 * w + 3];
    dy2[w] = q[5 * w + 4];
    nrd2[w] = q[10 + 6 * w + 0];
    const double rD2 = sqrt(q[10 + 6 * w + 1]);
    const double cx = q[10 + 6 * w + 3];
    const double bnd = q[10 + 6 * w + 4];
    dx2[w] = q[10 + 6 * w + 5];
    const double pobj = cx, dobj = by + bnd;
    gap[w] = pobj - dobj;
    S->kkt[w] = sqrt(om * nrp2[w] + nrd2[w] / om + gap[w] * gap[w]);
    S->rP2[w] = rP2;
    S->rD2[w] = rD2;
    S->rel_p[w] = rP2 / (1.0 + S->nb);
    S->rel_d[w] = rD2 / (1.0 + S->nc);
    S->rel_gap[w] = fabs(gap[w]) / (1.0 + fabs(pobj) + fabs(dobj));
    S->rel_kkt[w] = fmax(S->rel_p[w], fmax(S->rel_d[w], S->rel_gap[w]));
  }
  if (mode == 0) {
    S->kkt_r = S->kkt[0];
    S->kkt_prev = INFINITY;
    return;
  }
  S->restart_to = 0;
  const int pick = S->rel_kkt[1] <= S->rel_kkt[0] ? 1 : 0;
  const double elapsed = (double)(global_ns() - S->t0_ns) * 1e-9;
  const bool finite = isfinite(S->kkt[0]) && isfinite(S->kkt[1]);
  if (S->phase == 0) {
    if (!finite) {
      S->done = 1; S->status = PDHGC_STATUS_NUMERICAL; S->chosen = 0;
    } else if (S->at_check && fmin(S->rel_kkt[0], S->rel_kkt[1]) <= S->eps_rel) {
      S->done = 1; S->status = PDHGC_STATUS_OPTIMAL; S->chosen = pick;
    } else if (S->at_limit) {
      S->done = 1; S->status = PDHGC_STATUS_ITER_LIMIT; S->chosen = pick;
    } else if (elapsed > S->time_limit_s) {
      S->done = 1; S->status = PDHGC_STATUS_TIME_LIMIT; S->chosen = pick;
    }
  } else {
    if (!finite) {
      S->done = 1; S->status = PDHGC_STATUS_CORNER_LIMIT; S->chosen = 0;
    } else if (S->at_check && S->k >= S->min_iters) {
      const double tol = S->eps_rel * (1.0 + S->nb);
      const double tol_d = S->eps_rel * (1.0 + S->nc);
      if (S->stop_rule == 1) {
        if (fmin(S->rel_kkt[0], S->rel_kkt[1]) <= S->eps_rel) {
          S->done = 1; S->status = PDHGC_STATUS_CORNER_DONE; S->chosen = pick;
        }
      } else if (S->stop_rule == 2) {  // the dual corner push: the dual residual regained
        if (S->rD2[0] <= tol_d) {
          S->done = 1; S->status = PDHGC_STATUS_CORNER_DONE; S->chosen = 0;
        } else if (S->rD2[1] <= tol_d) {
          S->done = 1; S->status = PDHGC_STATUS_CORNER_DONE; S->chosen = 1;
        }
      } else if (S->rP2[0] <= tol) {
        S->done = 1; S->status = PDHGC_STATUS_CORNER_DONE; S->chosen = 0;
      } else if (S->rP2[1] <= tol) {
        S->done = 1; S->status = PDHGC_STATUS_CORNER_DONE; S->chosen = 1;
      }
    }
    if (!S->done && (S->at_limit || elapsed > S->time_limit_s)) {
      S->done = 1; S->status = PDHGC_STATUS_CORNER_LIMIT; S->chosen = 0;
    }
  }
  if (!S->done) {
    const int c = S->kkt[1] <= S->kkt[0] ? 1 : 0;
    const double kc = S->kkt[c];
    const bool restart = kc <= S->beta_suff * S->kkt_r ||
                         (kc <= S->beta_nec * S->kkt_r && kc > S->kkt_prev) ||
                         (double)S->t >= S->beta_art * (double)S->k;
    if (!restart) {
      S->kkt_prev = kc;
    } else {
      const double dx = sqrt(dx2[c]), dy = sqrt(dy2[c]);
      double omega = S->omega;
      if (dx > 1e-10 && dy > 1e-10)
        omega = exp(S->theta * log(dy / dx) + (1.0 - S->theta) * log(omega));
      S->omega = omega;
      S->kkt_r = sqrt(omega * nrp2[c] + nrd2[c] / omega + gap[c] * gap[c]);
      S->kkt_prev = INFINITY;
      S->t = 0;
      S->restarts += 1;
      S->restart_to = c ? 2 : 1;
      S->tau = S->eta / omega;
      S->sigma = S->eta * omega;
    }
  }
  S->t1_ns = global_ns();
}

// The Halpern loop's decision at a check, from the 14 folded quantities q of
// EvalRowsH (0..6) and EvalColsH (7..13): the Section 2 ratios of T(z) (slot
// 0; slot 1 repeats it), the fixed-point residual
//   r = sqrt(|dx|^2 / tau + |dy|^2 / sigma + 2 dy' A_hat dx),
// termination as in decide_step (the returned point is always T(z):
// chosen = 2), then the restart test on r against the anchor's residual
// fpr0 and the previous check's fpr_prev, with the PID primal-weight update
// on a restart.  mode 0 (the start point's probe) only records fpr0.
__device__ inline void decide_halpern(Scalars* S, const double* q, int mode) {
  const double om = S->omega;
  const double nrp2 = q[0], rP2 = sqrt(q[1]), by = q[3], dy0 = q[4], dy2 = q[5], cross = q[6];
  const double nrd2 = q[7], rD2 = sqrt(q[8]), cx = q[10], bnd = q[11], dx0 = q[12], dx2 = q[13];
  const double pobj = cx, dobj = by + bnd, gap = pobj - dobj;
  S->kkt[0] = sqrt(om * nrp2 + nrd2 / om + gap * gap);
  S->rP2[0] = rP2;
  S->rD2[0] = rD2;
  S->rD2[1] = rD2;
  S->rel_p[0] = rP2 / (1.0 + S->nb);
  S->rel_d[0] = rD2 / (1.0 + S->nc);
  S->rel_gap[0] = fabs(gap) / (1.0 + fabs(pobj) + fabs(dobj));
  S->rel_kkt[0] = fmax(S->rel_p[0], fmax(S->rel_d[0], S->rel_gap[0]));
  S->kkt[1] = S->kkt[0];
  S->rP2[1] = S->rP2[0];
  S->rel_p[1] = S->rel_p[0];
  S->rel_d[1] = S->rel_d[0];
  S->rel_gap[1] = S->rel_gap[0];
  S->rel_kkt[1] = S->rel_kkt[0];
  const double r = sqrt(fmax(dx2 / S->tau + dy2 / S->sigma + 2.0 * cross, 0.0));
  S->fpr = r;
  if (mode == 0) {
    S->fpr0 = r;
    S->fpr_prev = INFINITY;
    return;
  }
  S->restart_to = 0;
  const double elapsed = (double)(global_ns() - S->t0_ns) * 1e-9;
  const bool finite = isfinite(S->kkt[0]) && isfinite(r);
  if (S->phase == 0) {
    if (!finite) {
      S->done = 1; S->status = PDHGC_STATUS_NUMERICAL; S->chosen = 2;
    } else if (S->at_check && S->rel_kkt[0] <= S->eps_rel) {
      S->done = 1; S->status = PDHGC_STATUS_OPTIMAL; S->chosen = 2;
    } else if (S->at_limit) {
      S->done = 1; S->status = PDHGC_STATUS_ITER_LIMIT; S->chosen = 2;
    } else if (elapsed > S->time_limit_s) {
      S->done = 1; S->status = PDHGC_STATUS_TIME_LIMIT; S->chosen = 2;
    }
  } else {
    if (!finite) {
      S->done = 1; S->status = PDHGC_STATUS_CORNER_LIMIT; S->chosen = 2;
    } else if (S->at_check && S->k >= S->min_iters) {
      const bool met = S->stop_rule == 1   ? S->rel_kkt[0] <= S->eps_rel
                       : S->stop_rule == 2 ? rD2 <= S->eps_rel * (1.0 + S->nc)
                                           : rP2 <= S->eps_rel * (1.0 + S->nb);
      if (met) {
        S->done = 1; S->status = PDHGC_STATUS_CORNER_DONE; S->chosen = 2;
      }
    }
    if (!S->done && (S->at_limit || elapsed > S->time_limit_s)) {
      S->done = 1; S->status = PDHGC_STATUS_CORNER_LIMIT; S->chosen = 2;
    }
  }
  if (!S->done) {
    const bool restart = r <= S->beta_suff * S->fpr0 || (r <= S->beta_nec * S->fpr0 && r > S->fpr_prev) ||
                         (double)S->t >= S->beta_art * (double)S->k;
    if (!restart) {
      S->fpr_prev = r;
    } else {
      const double dx = sqrt(dx0), dy = sqrt(dy0);
      if (dx > 1e-10 && dy > 1e-10) {
        const double e = log(om) - log(dy / dx);
        S->pid_int += e;
        const double lo = log(om) - (S->pid_kp * e + S->pid_ki * S->pid_int + S->pid_kd * (e - S->pid_eprev));
        S->pid_eprev = e;
        S->omega = exp(lo);
      }
      S->fpr0 = r;
      S->fpr_prev = INFINITY;
      S->t = 0;
      S->restarts += 1;
      S->restart_to = 3;
      S->tau = S->eta / S->omega;
      S->sigma = S->eta * S->omega;
    }
  }
  S->t1_ns = global_ns();
}

// ---------------------------------------------------------------------------
// The SpMV kernel
//
// One launch covers a whole matrix pass.  Blocks are split over the three
// row segments planned on the host (host_prep.h):
//   CTA rows   the whole CTA strides over the row
//   warp rows  a warp strides over the row, then a shuffle reduction
//   SELL-32    a lane owns one row of a 32-row slice; element j of the
//              slice's rows is contiguous, so every value / index load of a
//              warp is one coalesced 256 + 128-byte access, there is no
//              shared memory and no barrier, and a row costs exactly one FMA
//              per nonzero; PDHGC_GATHER_BATCH gathers are kept in flight per lane
// The row sum goes straight into the operator's fused epilogue, and the
// epilogue's partial sums are folded per block in a fixed order.
//
// kPdl: launched with programmatic dependent launch.  The matrix is never
// written by an iteration kernel, so row lengths and the first batch of
// values and indices are read before `griddepcontrol.wait`; every gather of
// an iterate, every read of the scalar state and every write come after it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Loads of the streamed matrix (values and indices, read once per pass) skip
// L1 allocation so that L1 keeps the gathered vector entries; the L2 policy
// is untouched (the matrix is reused from L2 by the next iteration).
#ifndef PDHGC_STREAM_NO_L1
#define PDHGC_STREAM_NO_L1 1
#endif
__device__ __forceinline__ double ld_stream(const double* p) {
#if PDHGC_STREAM_NO_L1
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}
__device__ __forceinline__ float ld_stream(const float* p) {
#if PDHGC_STREAM_NO_L1
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}
__device__ __forceinline__ int ld_stream(const int* p) {
#if PDHGC_STREAM_NO_L1
  int v;
  asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}

// Gathers of the iterate vector (random entries, reused across the pass):
// read-only path, L1 allocation as usual; PDHGC_GATHER_HINT = 1 asks L1 to
// keep them over other lines (evict_last)
#ifndef PDHGC_GATHER_HINT
#define PDHGC_GATHER_HINT 0
#endif
__device__ __forceinline__ double ld_gather(const double* p) {
#if PDHGC_GATHER_HINT
  double v;
  asm("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}
__device__ __forceinline__ float ld_gather(const float* p) {
#if PDHGC_GATHER_HINT
  float v;
  asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
#else
  return __ldg(p);
#endif
}

template <class T, int NG>
struct GV {
  T v[NG];
};

// VT: value type of the matrix copy a pass reads (double, or float for the
// FP32-bulk iteration)
template <class VT>
struct SpmvMatT {
  const int* __restrict__ row_ptr;
  const int* __restrict__ col;
  const VT* __restrict__ val;            // CSR values (CTA and warp rows)
  const int* __restrict__ slice_ptr;
  const int* __restrict__ slice_w;
  const int* __restrict__ scol;          // SELL-32 indices
  const VT* __restrict__ sval;           // SELL-32 values
  const SellBlock* __restrict__ sell_blocks;
  int rows, cta_rows, long_rows, nslices;
  int nb_cta, nb_warp, nb_sell;
};
using SpmvMat = SpmvMatT<double>;

// gathers in flight per lane, and the minimum resident blocks per SM the
// register allocation must allow (tuning knobs, overridable at build time)
#ifndef PDHGC_GATHER_BATCH
#define PDHGC_GATHER_BATCH 4
#endif
#ifndef PDHGC_MIN_BLOCKS
#define PDHGC_MIN_BLOCKS 4
#endif
// 1: the SELL-32 loop requests the next batch's matrix entries before it
// consumes the current batch's gathers
#ifndef PDHGC_SELL_PIPE
#define PDHGC_SELL_PIPE 0
#endif
constexpr int kBatch = PDHGC_GATHER_BATCH;

// acc += sum over k = k0, k0+step, ... < k1 of val[k] * gathered(col[k]), in
// that order, with kBatch gathers in flight per lane (CSR rows)
template <class Op>
__device__ __forceinline__ void row_dot_global(const Op& op, typename Op::Acc& acc, double rc,
                                               const typename Op::VT* __restrict__ val,
                                               const int* __restrict__ col, int k0, int k1, int step) {
  constexpr int NG = Op::NG;
  using VT = typename Op::VT;
  using GT = typename Op::GT;
  int k = k0;
  for (; k + (kBatch - 1) * step < k1; k += kBatch * step) {
    VT v[kBatch];
    int c[kBatch];
    GV<GT, NG> g[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      v[u] = ld_stream(val + k + u * step);
      c[u] = ld_stream(col + k + u * step);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
#pragma unroll
      for (int i = 0; i < NG; ++i) g[u].v[i] = ld_gather(op.gsrc(i) + c[u]);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) op.accum(acc, rc, v[u], g[u]);
  }
  // the ragged tail (fewer than kBatch entries left) as one predicated batch:
  // its loads and gathers are in flight together, in the same summation order
  if (k < k1) {
    VT v[kBatch];
    int c[kBatch];
    GV<GT, NG> g[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (k + u * step < k1) {
        v[u] = ld_stream(val + k + u * step);
        c[u] = ld_stream(col + k + u * step);
      }
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
      if (k + u * step < k1)
#pragma unroll
        for (int i = 0; i < NG; ++i) g[u].v[i] = ld_gather(op.gsrc(i) + c[u]);
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
      if (k + u * step < k1) op.accum(acc, rc, v[u], g[u]);
  }
}

// Operators whose epilogue reads per-row inputs can declare `Pre`,
// `prefetch(row)` and `epilogue_pre(row, acc, pre, part)`: the kernel then
// loads those inputs right after the grid-dependency wait, so that their
// latency overlaps the gathers instead of following them.
template <class Op, class = void>
struct Prefetcher {
  struct Pre {};
  __device__ static Pre get(const Op&, int) { return Pre{}; }
  __device__ static void epilogue(const Op& op, int r, const typename Op::Acc& a, const Pre&, double* part) {
    op.epilogue(r, a, part);
  }
};
#ifndef PDHGC_PREFETCH
#define PDHGC_PREFETCH 1
#endif
template <class Op>
struct Prefetcher<Op, std::void_t<typename Op::Pre>> {
#if PDHGC_PREFETCH
  using Pre = typename Op::Pre;
  __device__ static Pre get(const Op& op, int r) { return op.prefetch(r); }
  __device__ static void epilogue(const Op& op, int r, const typename Op::Acc& a, const Pre& p, double* part) {
    op.epilogue_pre(r, a, p, part);
  }
#else  // the same inputs, loaded when the epilogue runs
  struct Pre {};
  __device__ static Pre get(const Op&, int) { return Pre{}; }
  __device__ static void epilogue(const Op& op, int r, const typename Op::Acc& a, const Pre&, double* part) {
    op.epilogue_pre(r, a, op.prefetch(r), part);
  }
#endif
};

template <class Op, bool kPdl>
__global__ void __launch_bounds__(kBlock, PDHGC_MIN_BLOCKS)
    spmv(SpmvMatT<typename Op::VT> M, Op op, double* __restrict__ partials) {
  using VT = typename Op::VT;
  using GT = typename Op::GT;
  using PF = Prefetcher<Op>;
  constexpr int NG = Op::NG;
  constexpr int NQ = Op::NQ;
  constexpr int NQS = NQ > 0 ? NQ : 1;
  __shared__ typename Op::Acc s_acc[kWarpsPerBlock];
  __shared__ double s_red[NQS][kWarpsPerBlock];
  if constexpr (!kPdl) {
    if (op.skip()) return;
  }
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int blk = blockIdx.x;
  double part[NQS];
#pragma unroll
  for (int q = 0; q < NQS; ++q) part[q] = 0.0;

  if (blk < M.nb_cta) {
    const int r = blk;
    const int e0 = M.row_ptr[r], e1 = M.row_ptr[r + 1];
    if constexpr (kPdl) {
      grid_dep_wait();
      if (op.skip()) return;
    }
    const double rc = op.row_ctx(r);
    typename PF::Pre pre{};
    if (tid == 0) pre = PF::get(op, r);
    typename Op::Acc acc;
    acc.zero();
    row_dot_global(op, acc, rc, M.val, M.col, e0 + tid, e1, kBlock);
    if constexpr (kPdl) grid_dep_launch();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc.add(acc.shfl_xor(0xffffffffu, off));
    if (lane == 0) s_acc[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      typename Op::Acc tot = s_acc[0];
#pragma unroll
      for (int w = 1; w < kWarpsPerBlock; ++w) tot.add(s_acc[w]);
      PF::epilogue(op, r, tot, pre, part);
    }
  } else if (blk < M.nb_cta + M.nb_warp) {
    const int r = M.cta_rows + (blk - M.nb_cta) * kWarpsPerBlock + warp;
    const bool has = r < M.long_rows;  // uniform within the warp
    int e0 = 0, e1 = 0;
    if (has) {
      e0 = M.row_ptr[r];
      e1 = M.row_ptr[r + 1];
    }
    if constexpr (kPdl) {
      grid_dep_wait();
      if (op.skip()) return;
    }
    if (has) {
      const double rc = op.row_ctx(r);
      typename PF::Pre pre{};
      if (lane == 0) pre = PF::get(op, r);
      typename Op::Acc acc;
      acc.zero();
      row_dot_global(op, acc, rc, M.val, M.col, e0 + lane, e1, 32);
      if constexpr (kPdl) grid_dep_launch();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc.add(acc.shfl_xor(0xffffffffu, off));
      if (lane == 0) PF::epilogue(op, r, acc, pre, part);
    } else {
      if constexpr (kPdl) grid_dep_launch();
    }
  } else {
    // SELL-32: this warp sums columns [jb, je) of its slice's 32 rows
    const SellBlock sb = M.sell_blocks[blk - M.nb_cta - M.nb_warp];
    const int K = sb.k;
    const int ls = warp / K, kw = warp - ls * K;
    int r = -1, len = 0, base = 0, jb = 0, je = 0;
    if (ls < sb.count) {
      const int s = sb.first + ls;
      base = M.slice_ptr[s];
      const int w = M.slice_w[s];
      const int cw = (w + K - 1) / K;
      jb = kw * cw;
      je = min(w, jb + cw);
      const int rr = M.long_rows + s * kSellH + lane;
      if (rr < M.rows) {
        r = rr;
        len = M.row_ptr[rr + 1] - M.row_ptr[rr];
      }
    }
    const int jend = min(je, len);  // this lane's last column + 1
    VT v[kBatch];
    int c[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (jb + u < jend) {
        v[u] = ld_stream(M.sval + base + (jb + u) * kSellH + lane);
        c[u] = ld_stream(M.scol + base + (jb + u) * kSellH + lane);
      }
    }
    if constexpr (kPdl) {
      grid_dep_wait();
      if (op.skip()) return;
    }
    typename PF::Pre pre{};
    if (kw == 0 && r >= 0) pre = PF::get(op, r);
    typename Op::Acc acc;
    acc.zero();
    const double rc = r >= 0 ? op.row_ctx(r) : 0.0;
#if PDHGC_SELL_PIPE
    // software-pipelined: the next batch's values and indices are requested
    // while this batch's gathers are in flight, so that a step waits for the
    // slower of the two loads instead of their sum
    for (int j = jb; j < je; j += kBatch) {
      GV<GT, NG> g[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (j + u < jend)
#pragma unroll
          for (int i = 0; i < NG; ++i) g[u].v[i] = ld_gather(op.gsrc(i) + c[u]);
      VT vn[kBatch];
      int cn[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (j + kBatch + u < jend) {
          vn[u] = ld_stream(M.sval + base + (j + kBatch + u) * kSellH + lane);
          cn[u] = ld_stream(M.scol + base + (j + kBatch + u) * kSellH + lane);
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (j + u < jend) op.accum(acc, rc, v[u], g[u]);
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        v[u] = vn[u];
        c[u] = cn[u];
      }
    }
#else
    for (int j = jb; j < je; j += kBatch) {
      if (j > jb) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          if (j + u < jend) {
            v[u] = ld_stream(M.sval + base + (j + u) * kSellH + lane);
            c[u] = ld_stream(M.scol + base + (j + u) * kSellH + lane);
          }
        }
      }
      GV<GT, NG> g[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (j + u < jend)
#pragma unroll
          for (int i = 0; i < NG; ++i) g[u].v[i] = ld_gather(op.gsrc(i) + c[u]);
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (j + u < jend) op.accum(acc, rc, v[u], g[u]);
    }
#endif
    if constexpr (kPdl) grid_dep_launch();
    if (K > 1) {  // uniform over the block
      __shared__ typename Op::Acc s_part[kWarpsPerBlock][kSellH];
      s_part[warp][lane] = acc;
      __syncthreads();
      if (kw == 0) {
        for (int q = 1; q < K; ++q) acc.add(s_part[warp + q][lane]);
      }
    }
    if (kw == 0 && r >= 0) PF::epilogue(op, r, acc, pre, part);
  }

  if constexpr (NQ > 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = part[q];
      const bool is_max = (Op::kMaxMask >> q) & 1u;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_xor_sync(0xffffffffu, x, off);
        x = is_max ? fmax(x, o) : x + o;
      }
      if (lane == 0) s_red[q][warp] = x;
    }
    __syncthreads();
    if (tid < NQ) {
      const bool is_max = (Op::kMaxMask >> tid) & 1u;
      double x = s_red[tid][0];
#pragma unroll
      for (int w2 = 1; w2 < kWarpsPerBlock; ++w2) x = is_max ? fmax(x, s_red[tid][w2]) : x + s_red[tid][w2];
      partials[(size_t)tid * gridDim.x + blk] = x;
    }
  }
}

// ---------------------------------------------------------------------------
// The chunked pass (ChunkPlan in host_prep.h): one CTA of kChunkThreads per
// SM.  For each chunk of the gathered vector the CTA copies the chunk into
// shared memory with coalesced 16-byte loads, then every warp runs its work
// units' entries in that chunk, gathering from shared memory; the row sums
// stay in registers across chunks and the operator's epilogue runs once at
// the end.  A slice unit (up to 32 rows) gives a lane a row and reads the
// chunk's slots column-major; a long-row unit lets its 32 lanes stride over
// the row's slots and reduces them by shuffles.  Padding slots carry
// kChunkPadIdx and are skipped.
// ---------------------------------------------------------------------------
template <class VT>
struct ChunkMatT {
  const VT* __restrict__ val;          // slots
  const uint16_t* __restrict__ idx;    // slots: index within the chunk
  const ChunkUnit* __restrict__ units;
  const int* __restrict__ uc_off;      // nunits * nch
  const int* __restrict__ uc_cnt;
  const int* __restrict__ warp_units;  // blocks * kChunkWarps * kChunkMaxUnits
  int nch, chunk, glen;
};

template <class GT>
__device__ __forceinline__ void stage_chunk(GT* __restrict__ s, const GT* __restrict__ src, int len) {
  // 16-byte vector loads (src is 16-byte aligned: the chunk starts at a
  // multiple of kChunkBytes / sizeof(GT) entries of a cudaMalloc'd array)
  constexpr int V = 16 / sizeof(GT);
  const int nv = len / V;
  const float4* __restrict__ s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(s);
  for (int t = threadIdx.x; t < nv; t += kChunkThreads) d4[t] = __ldcg(s4 + t);
  for (int t = nv * V + threadIdx.x; t < len; t += kChunkThreads) s[t] = src[t];
}

template <class Op, bool kPdl>
__global__ void __launch_bounds__(kChunkThreads, 1)
    spmv_chunked(ChunkMatT<typename Op::VT> M, Op op) {
  using VT = typename Op::VT;
  using GT = typename Op::GT;
  using PF = Prefetcher<Op>;
  static_assert(Op::NG == 1, "one gathered vector");
  extern __shared__ __align__(16) unsigned char s_raw[];
  GT* s_g = reinterpret_cast<GT*>(s_raw);
  if constexpr (!kPdl) {
    if (op.skip()) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int* wl = M.warp_units + ((size_t)blockIdx.x * kChunkWarps + warp) * kChunkMaxUnits;
  int u[kChunkMaxUnits];
#pragma unroll
  for (int k = 0; k < kChunkMaxUnits; ++k) u[k] = wl[k];
  typename Op::Acc acc[kChunkMaxUnits];
#pragma unroll
  for (int k = 0; k < kChunkMaxUnits; ++k) acc[k].zero();
  if constexpr (kPdl) {
    grid_dep_wait();
    if (op.skip()) return;  // uniform over the grid
  }
  const GT* src = op.gsrc(0);
  for (int c = 0; c < M.nch; ++c) {
    const int base = c * M.chunk;
    __syncthreads();  // every warp is done with the previous chunk
    stage_chunk(s_g, src + base, min(M.chunk, M.glen - base));
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kChunkMaxUnits; ++k) {
      if (u[k] < 0) continue;  // uniform within the warp
      const size_t uc = (size_t)u[k] * M.nch + c;
      const int off = M.uc_off[uc], cnt = M.uc_cnt[uc];
      // this lane's slots are off + lane + 32 j: column j of a slice (width
      // cnt), or entry lane + 32 j of a long row's cnt slots
      const bool is_long = M.units[u[k]].is_long != 0;
      const int n_lane = is_long ? (cnt - lane + 31) / 32 : cnt;
      const VT* vp = M.val + off + lane;
      const uint16_t* ip = M.idx + off + lane;
      constexpr int stride = 32;
      int j = 0;
      for (; j + 4 <= n_lane; j += 4) {
        VT v[4];
        int ii[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] = ld_stream(vp + (size_t)(j + q) * stride);
          ii[q] = __ldg(ip + (size_t)(j + q) * stride);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (ii[q] != kChunkPadIdx) {
            GV<GT, 1> g;
            g.v[0] = s_g[ii[q]];
            op.accum(acc[k], 0.0, v[q], g);
          }
      }
      for (; j < n_lane; ++j) {
        const int i = __ldg(ip + (size_t)j * stride);
        if (i != kChunkPadIdx) {
          GV<GT, 1> g;
          g.v[0] = s_g[i];
          op.accum(acc[k], 0.0, ld_stream(vp + (size_t)j * stride), g);
        }
      }
    }
  }
  if constexpr (kPdl) grid_dep_launch();
#pragma unroll
  for (int k = 0; k < kChunkMaxUnits; ++k) {
    if (u[k] < 0) continue;
    const ChunkUnit U = M.units[u[k]];
    if (U.is_long) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[k].add(acc[k].shfl_xor(0xffffffffu, off));
      if (lane == 0) PF::epilogue(op, U.row0, acc[k], PF::get(op, U.row0), nullptr);
    } else if (lane < U.nrows) {
      const int r = U.row0 + lane;
      PF::epilogue(op, r, acc[k], PF::get(op, r), nullptr);
    }
  }
}

// ---------------------------------------------------------------------------
// Epilogue operators
// ---------------------------------------------------------------------------

// x' = proj_[l,u](x - tau (c - A'y)),  x_bar = 2x' - x,  sum_x += x'
struct PrimalOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const Scalars* S;
  int it;
  const double* __restrict__ y;
  DevModel md;
  DevIter w;
  __device__ bool skip() const { return S->done || S->k + it >= S->max_iters; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return y; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  struct Pre {
    double c, l, u, x, sx, tau;
  };
  __device__ Pre prefetch(int j) const { return Pre{md.chat[j], md.lhat[j], md.uhat[j], w.x[j], w.sum_x[j], S->tau}; }
  __device__ void epilogue_pre(int j, const Acc& a, const Pre& p, double*) const {
    const double g = p.c - a.v[0];
    const double xn = clamp_i(p.x - p.tau * g, p.l, p.u);
    w.xbar[j] = 2.0 * xn - p.x;
    w.sum_x[j] = p.sx + xn;
    w.x[j] = xn;
  }
};

// y' = y + sigma (b - A x_bar), y' >= 0 on '>' rows,  sum_y += y'
struct DualOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const Scalars* S;
  int it;
  const double* __restrict__ xbar;
  DevModel md;
  DevIter w;
  __device__ bool skip() const { return S->done || S->k + it >= S->max_iters; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return xbar; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  struct Pre {
    double b, y, sy, sigma;
    int8_t ge;
  };
  __device__ Pre prefetch(int i) const { return Pre{md.bhat[i], w.y[i], w.sum_y[i], S->sigma, md.ge[i]}; }
  __device__ void epilogue_pre(int i, const Acc& a, const Pre& p, double*) const {
    double yn = p.y + p.sigma * (p.b - a.v[0]);
    // y >= 0 on '>' rows (sign bit test); y = 0 on a row whose dual is fixed
    if (p.ge && (p.ge == kRowDualZero || __double_as_longlong(yn) < 0)) yn = 0.0;
    w.sum_y[i] = p.sy + yn;
    w.y[i] = yn;
  }
};

// KKT pieces from the rows: for w in {current, average}
//   r_hat = b_hat - A_hat x_w (max(.,0) on '>' rows), r_hat^2, (r_hat/D_r)^2,
//   max |r_hat/D_r|, b_hat y_w, (y_w - y_r)^2
struct EvalRowsOp {
  using Acc = SumD<2>;
  static constexpr int NQ = 10;
  static constexpr unsigned kMaxMask = (1u << 2) | (1u << 7);
  const Scalars* S;
  const double* __restrict__ x;
  const double* __restrict__ sum_x;
  const double* __restrict__ y;
  const double* __restrict__ sum_y;
  const double* __restrict__ y_r;
  DevModel md;
  __device__ bool skip() const { return S->done; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 2;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int i) const { return i == 0 ? x : sum_x; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 2>& g) const {
    a.v[0] = fma(v, g.v[0], a.v[0]);
    a.v[1] = fma(v, g.v[1], a.v[1]);
  }
  __device__ void epilogue(int i, const Acc& a, double* part) const {
    const double inv_t = S->inv_t;
    const double b = md.bhat[i], dr = md.Dr[i];
    const int8_t ge = md.ge[i];
#pragma unroll
    for (int wv = 0; wv < 2; ++wv) {
      const double ax = wv == 0 ? a.v[0] : a.v[1] * inv_t;
      double r = b - ax;
      if (ge) r = ge == kRowDualZero ? 0.0 : fmax(r, 0.0);
      const double ru = r / dr;
      const double yw = wv == 0 ? y[i] : sum_y[i] * inv_t;
      const double d = yw - y_r[i];
      part[5 * wv + 0] += r * r;
      part[5 * wv + 1] += ru * ru;
      part[5 * wv + 2] = fmax(part[5 * wv + 2], fabs(ru));
      part[5 * wv + 3] += b * yw;
      part[5 * wv + 4] += d * d;
    }
  }
};

// KKT pieces from the columns: lam = c_hat - A_hat' y_w, z = proj(lam),
//   r_D = lam - z, r_D^2, (r_D/D_c)^2, max |r_D/D_c|, c_hat x_w,
//   l z^+ - u z^- (finite bounds), (x_w - x_r)^2
struct EvalColsOp {
  using Acc = SumD<2>;
  static constexpr int NQ = 12;
  static constexpr unsigned kMaxMask = (1u << 2) | (1u << 8);
  const Scalars* S;
  const double* __restrict__ y;
  const double* __restrict__ sum_y;
  const double* __restrict__ x;
  const double* __restrict__ sum_x;
  const double* __restrict__ x_r;
  DevModel md;
  // optional: z_hat of the current (z_out0) and average (z_out1) point, for
  // the restart history of the guidance features (phase 1 only)
  double* __restrict__ z_out0;
  double* __restrict__ z_out1;
  __device__ bool skip() const { return S->done; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 2;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int i) const { return i == 0 ? y : sum_y; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 2>& g) const {
    a.v[0] = fma(v, g.v[0], a.v[0]);
    a.v[1] = fma(v, g.v[1], a.v[1]);
  }
  __device__ void epilogue(int j, const Acc& a, double* part) const {
    const double inv_t = S->inv_t;
    const double c = md.chat[j], l = md.lhat[j], u = md.uhat[j], dc = md.Dc[j];
#pragma unroll
    for (int wv = 0; wv < 2; ++wv) {
      const double aty = wv == 0 ? a.v[0] : a.v[1] * inv_t;
      const double lam = c - aty;
      const double z = proj_dual(lam, l, u);
      if (z_out0) (wv == 0 ? z_out0 : z_out1)[j] = z;
      const double rd = lam - z;
      const double rdu = rd / dc;
      const double xw = wv == 0 ? x[j] : sum_x[j] * inv_t;
      const double bnd = (l != -INFINITY ? l * fmax(z, 0.0) : 0.0) - (u != INFINITY ? u * fmax(-z, 0.0) : 0.0);
      const double d = xw - x_r[j];
      part[6 * wv + 0] += rd * rd;
      part[6 * wv + 1] += rdu * rdu;
      part[6 * wv + 2] = fmax(part[6 * wv + 2], fabs(rdu));
      part[6 * wv + 3] += c * xw;
      part[6 * wv + 4] += bnd;
      part[6 * wv + 5] += d * d;
    }
  }
};

// ---------------------------------------------------------------------------
// The Halpern loop (PDHGC_ALG_HALPERN): one step from z = (x, y) forms the
// PDHG output T(z) = (x+, y+) exactly as PrimalOp / DualOp do, then moves z
// to the anchored combination
//   z <- w ((1 + rho) T(z) - rho z) + (1 - w) z_0,  w = hw[it],
// evaluated as z_0 + w (r - z_0) with r = T(z) + rho (T(z) - z).  A check
// step (the last of a chunk, or of the phase) also stores T(z) and z - T(z)
// for the evaluation; `probe` forms T(z) of the start point only, leaving z.
// ---------------------------------------------------------------------------
// kUnitRho: the reflection is known to be 1 when the kernel is launched, so
// the reflected point is x_bar with no run-time test (the general operator
// makes the same choice from S->rho; both give the same bits at rho = 1)
template <bool kUnitRho>
struct PrimalOpHT {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const Scalars* S;
  int it, last_it, probe;
  const double* __restrict__ y;
  DevModel md;
  DevIter w;
  DevHalpern h;
  __device__ bool skip() const { return S->done || (!probe && S->k + it >= S->max_iters); }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return y; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  struct Pre {
    double c, l, u, x, x0, tau, wt, rho;
    bool last;
  };
  __device__ Pre prefetch(int j) const {
    const bool last = probe || it == last_it || S->k + it + 1 == S->max_iters;
    return Pre{md.chat[j], md.lhat[j], md.uhat[j], w.x[j], w.x_r[j], S->tau, h.hw[it], kUnitRho ? 1.0 : S->rho, last};
  }
  __device__ void epilogue_pre(int j, const Acc& a, const Pre& p, double*) const {
    const double g = p.c - a.v[0];
    const double xn = clamp_i(p.x - p.tau * g, p.l, p.u);
    const double xb = 2.0 * xn - p.x;
    w.xbar[j] = xb;
    if (!probe) {
      // the reflected point x+ + rho (x+ - x); with rho = 1 it is x_bar itself
      const double r = (kUnitRho || p.rho == 1.0) ? xb : fma(p.rho, xn - p.x, xn);
      w.x[j] = fma(p.wt, r - p.x0, p.x0);
    }
    if (p.last) {
      h.xp[j] = xn;
      h.dx[j] = p.x - xn;
    }
  }
};
using PrimalOpH = PrimalOpHT<false>;

template <bool kUnitRho>
struct DualOpHT {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const Scalars* S;
  int it, last_it, probe;
  const double* __restrict__ xbar;
  DevModel md;
  DevIter w;
  DevHalpern h;
  __device__ bool skip() const { return S->done || (!probe && S->k + it >= S->max_iters); }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return xbar; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  struct Pre {
    double b, y, y0, sigma, wt, rho;
    int8_t ge;
    bool last;
  };
  __device__ Pre prefetch(int i) const {
    const bool last = probe || it == last_it || S->k + it + 1 == S->max_iters;
    return Pre{md.bhat[i], w.y[i], w.y_r[i], S->sigma, h.hw[it], kUnitRho ? 1.0 : S->rho, md.ge[i], last};
  }
  __device__ void epilogue_pre(int i, const Acc& a, const Pre& p, double*) const {
    double yn = p.y + p.sigma * (p.b - a.v[0]);
    if (p.ge && (p.ge == kRowDualZero || __double_as_longlong(yn) < 0)) yn = 0.0;
    if (!probe) {
      const double r = (kUnitRho || p.rho == 1.0) ? fma(2.0, yn, -p.y) : fma(p.rho, yn - p.y, yn);
      w.y[i] = fma(p.wt, r - p.y0, p.y0);
    }
    if (p.last) {
      h.yp[i] = yn;
      h.dy[i] = p.y - yn;
    }
  }
};
using DualOpH = DualOpHT<false>;

// Halpern check, rows: r_hat = b_hat - A_hat x+ (max(., 0) on '>' rows),
//   r_hat^2, (r_hat/D_r)^2, max |r_hat/D_r|, b_hat y+, (y+ - y_0)^2,
//   dy^2 and dy (A_hat dx) for the metric residual
struct EvalRowsH {
  using Acc = SumD<2>;
  static constexpr int NQ = 7;
  static constexpr unsigned kMaxMask = 1u << 2;
  const Scalars* S;
  DevHalpern h;
  const double* __restrict__ y_r;
  DevModel md;
  __device__ bool skip() const { return S->done; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 2;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int i) const { return i == 0 ? h.xp : h.dx; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 2>& g) const {
    a.v[0] = fma(v, g.v[0], a.v[0]);
    a.v[1] = fma(v, g.v[1], a.v[1]);
  }
  __device__ void epilogue(int i, const Acc& a, double* part) const {
    const double b = md.bhat[i], dr = md.Dr[i];
    double r = b - a.v[0];
    if (md.ge[i]) r = md.ge[i] == kRowDualZero ? 0.0 : fmax(r, 0.0);
    const double ru = r / dr;
    const double yp = h.yp[i], dy = h.dy[i];
    const double d = yp - y_r[i];
    part[0] += r * r;
    part[1] += ru * ru;
    part[2] = fmax(part[2], fabs(ru));
    part[3] += b * yp;
    part[4] += d * d;
    part[5] += dy * dy;
    part[6] += dy * a.v[1];
  }
};

// Halpern check, columns: lam = c_hat - A_hat' y+, z = proj(lam), r_D = lam - z,
//   r_D^2, (r_D/D_c)^2, max |r_D/D_c|, c_hat x+, l z^+ - u z^- (finite
//   bounds), (x+ - x_0)^2, dx^2; optionally z of T(z) for the restart history
struct EvalColsH {
  using Acc = SumD<1>;
  static constexpr int NQ = 7;
  static constexpr unsigned kMaxMask = 1u << 2;
  const Scalars* S;
  DevHalpern h;
  const double* __restrict__ x_r;
  DevModel md;
  double* __restrict__ z_out;
  __device__ bool skip() const { return S->done; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return h.yp; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int j, const Acc& a, double* part) const {
    const double c = md.chat[j], l = md.lhat[j], u = md.uhat[j], dc = md.Dc[j];
    const double lam = c - a.v[0];
    const double z = proj_dual(lam, l, u);
    if (z_out) z_out[j] = z;
    const double rd = lam - z;
    const double rdu = rd / dc;
    const double xp = h.xp[j], dx = h.dx[j];
    const double bnd = (l != -INFINITY ? l * fmax(z, 0.0) : 0.0) - (u != INFINITY ? u * fmax(-z, 0.0) : 0.0);
    const double d = xp - x_r[j];
    part[0] += rd * rd;
    part[1] += rdu * rdu;
    part[2] = fmax(part[2], fabs(rdu));
    part[3] += c * xp;
    part[4] += bnd;
    part[5] += d * d;
    part[6] += dx * dx;
  }
};

// Ruiz / Pock-Chambolle factor passes on the entries (D_r |a|) D_c of the
// current scaled matrix, in the order the products are formed on the host
// reference.  ScaleMaxOp: 1/sqrt(row or column maximum); ScaleSumOp:
// 1/sqrt(row or column sum); 1 for an empty row or column.  kTransposed: the
// CSR is A' (its row is column j of A, its col is row i of A).
template <bool kTransposed>
struct ScaleMaxOp {
  using Acc = MaxD;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const double* __restrict__ d_own;    // D_r for A rows, D_c for A' rows
  const double* __restrict__ d_other;  // D_c for A rows, D_r for A' rows
  double* __restrict__ fac;
  __device__ bool skip() const { return false; }
  __device__ double row_ctx(int r) const { return d_own[r]; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return d_other; }
  __device__ void accum(Acc& a, double rc, double v, const GV<double, 1>& g) const {
    const double d = g.v[0];
    const double e = kTransposed ? (d * fabs(v)) * rc : (rc * fabs(v)) * d;
    a.v[0] = fmax(a.v[0], e);
  }
  __device__ void epilogue(int r, const Acc& a, double*) const {
    fac[r] = a.v[0] > 0.0 ? 1.0 / sqrt(a.v[0]) : 1.0;
  }
};

template <bool kTransposed>
struct ScaleSumOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const double* __restrict__ d_own;
  const double* __restrict__ d_other;
  double* __restrict__ fac;
  __device__ bool skip() const { return false; }
  __device__ double row_ctx(int r) const { return d_own[r]; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return d_other; }
  __device__ void accum(Acc& a, double rc, double v, const GV<double, 1>& g) const {
    const double d = g.v[0];
    const double e = kTransposed ? (d * fabs(v)) * rc : (rc * fabs(v)) * d;
    a.v[0] += e;
  }
  __device__ void epilogue(int r, const Acc& a, double*) const {
    fac[r] = a.v[0] > 0.0 ? 1.0 / sqrt(a.v[0]) : 1.0;
  }
};

// out = A_hat v (or A_hat' v); optional partial sum of out^2
template <bool kNorm>
struct SpmvOp {
  using Acc = SumD<1>;
  static constexpr int NQ = kNorm ? 1 : 0;
  static constexpr unsigned kMaxMask = 0;
  const Scalars* S;
  const double* __restrict__ v;
  double* __restrict__ out;
  __device__ bool skip() const { return S->pi_zero != 0; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return v; }
  __device__ void accum(Acc& a, double, double val, const GV<double, 1>& g) const { a.v[0] = fma(val, g.v[0], a.v[0]); }
  __device__ void epilogue(int r, const Acc& a, double* part) const {
    out[r] = a.v[0];
    if constexpr (kNorm) part[0] += a.v[0] * a.v[0];
  }
};

// Report on the ORIGINAL model for a given scaled point (x_hat, y_hat):
// residual pieces plus the Section 2.1 / 4.2 slack metrics per row.
struct ReportRowsOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 7;
  static constexpr unsigned kMaxMask = 1u << 2;
  const double* __restrict__ x;
  const double* __restrict__ y;
  DevModel md;
  double tol;
  __device__ bool skip() const { return false; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return x; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int i, const Acc& a, double* part) const {
    const double b = md.bhat[i], dr = md.Dr[i];
    const bool ge = md.ge[i];
    double r = b - a.v[0];
    if (ge) r = fmax(r, 0.0);
    const double ru = r / dr;
    part[0] += r * r;
    part[1] += ru * ru;
    part[2] = fmax(part[2], fabs(ru));
    part[3] += b * y[i];
    if (ge) {
      const double slack = (a.v[0] - b) / dr;
      const bool off = slack > tol;
      const bool zero = fabs(dr * y[i]) <= tol;
      part[4] += off ? 1.0 : 0.0;
      part[5] += zero ? 1.0 : 0.0;
      part[6] += (off && zero) ? 1.0 : 0.0;
    }
  }
};

struct ReportColsOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 8;
  static constexpr unsigned kMaxMask = 1u << 2;
  const double* __restrict__ y;
  const double* __restrict__ x;
  const double* __restrict__ l_user;
  const double* __restrict__ u_user;
  DevModel md;
  double tol;
  __device__ bool skip() const { return false; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return y; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int j, const Acc& a, double* part) const {
    const double c = md.chat[j], l = md.lhat[j], u = md.uhat[j], dc = md.Dc[j];
    const double lam = c - a.v[0];
    const double z = proj_dual(lam, l, u);
    const double rd = lam - z;
    const double rdu = rd / dc;
    part[0] += rd * rd;
    part[1] += rdu * rdu;
    part[2] = fmax(part[2], fabs(rdu));
    part[3] += c * x[j];
    part[4] += (l != -INFINITY ? l * fmax(z, 0.0) : 0.0) - (u != INFINITY ? u * fmax(-z, 0.0) : 0.0);
    const double xu = dc * x[j];
    const double zu = z / dc;
    const bool off = fmin(xu - l_user[j], u_user[j] - xu) > tol;
    const bool zero = fabs(zu) <= tol;
    part[5] += off ? 1.0 : 0.0;
    part[6] += zero ? 1.0 : 0.0;
    part[7] += (off && zero) ? 1.0 : 0.0;
  }
};

// SplitMix64 (Steele, Lea and Flood 2014): output number (j+1) of the stream
// started at `seed`, i.e. the finaliser applied to seed + (j+1) * gamma.
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long j) {
  unsigned long long z = seed + (j + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53;
}

// Algorithm 1 on the columns: z = proj(c_hat - A_hat' y1) / D_c (unscaled),
// ub <- x where z > eps_abs, lb <- x where z < -eps_abs (scaled space),
// c' = obj_scale * U(seed, user column) scaled by D_c; partial sums of
// c_hat'^2 and c'^2 for the new primal weight and ||c'||.
struct CornerColsOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 2;
  static constexpr unsigned kMaxMask = 0;
  const double* __restrict__ y1;
  const double* __restrict__ x1;
  const int* __restrict__ col_perm;
  DevModel md;  // original model
  double* __restrict__ lc;
  double* __restrict__ uc;
  double* __restrict__ cc;
  double eps_abs, obj_scale;
  unsigned long long seed;
  int8_t* __restrict__ fixed;  // optional: 1 where the reduced-cost rule fixed a bound
  __device__ bool skip() const { return false; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return y1; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int j, const Acc& a, double* part) const {
    const double dc = md.Dc[j];
    const double lam = md.chat[j] - a.v[0];
    const double z = proj_dual(lam, md.lhat[j], md.uhat[j]) / dc;
    lc[j] = z < -eps_abs ? x1[j] : md.lhat[j];
    uc[j] = z > eps_abs ? x1[j] : md.uhat[j];
    if (fixed) fixed[j] = (z > eps_abs || z < -eps_abs) ? 1 : 0;
    const double cu = obj_scale * splitmix_uniform(seed, (unsigned long long)col_perm[j]);
    const double ch = dc * cu;
    cc[j] = ch;
    part[0] += ch * ch;
    part[1] += cu * cu;
  }
};

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------

// deterministic sum (or max) of partials[q * ntiles + 0 .. ntiles-1] by one CTA
__device__ inline double block_fold(const double* __restrict__ p, int ntiles, bool is_max, double* s_tmp) {
  double v = 0.0;
  for (int k = threadIdx.x; k < ntiles; k += blockDim.x) v = is_max ? fmax(v, p[k]) : v + p[k];
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, v, off);
    v = is_max ? fmax(v, o) : v + o;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
  __syncthreads();
  double tot = s_tmp[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tot = is_max ? fmax(tot, s_tmp[w]) : tot + s_tmp[w];
  return tot;  // same value in every thread
}


// ---------------------------------------------------------------------------
// FP32-bulk iteration (precision PDHGC_FP32_BULK)
//
// Matrix values, x, x_bar, y and the model vectors are FP32; each product
// v * g is formed exactly as a float pair (p, fma(v, g, -p)) and the row sum
// is kept as an unevaluated float pair (hi, lo) with Knuth's TwoSum, so the
// only error of a row sum is that of its FP32 inputs.  The running sums of
// the averages stay FP64.  Every KKT, gap, restart and step-size quantity is
// computed in FP64 by the evaluation operators above, from FP64 copies.
// ---------------------------------------------------------------------------
struct SumFF {
  float hi[1], lo[1];
  __device__ __forceinline__ void zero() {
    hi[0] = 0.f;
    lo[0] = 0.f;
  }
  // (hi, lo) += (a, b): TwoSum of the high parts, low parts added
  __device__ __forceinline__ void add_pair(float a, float b) {
    const float s = hi[0] + a;
    const float bb = s - hi[0];
    const float err = (hi[0] - (s - bb)) + (a - bb);
    hi[0] = s;
    lo[0] += err + b;
  }
  __device__ __forceinline__ void add(const SumFF& o) { add_pair(o.hi[0], o.lo[0]); }
  __device__ __forceinline__ SumFF shfl_xor(unsigned mask, int off) const {
    SumFF r;
    r.hi[0] = __shfl_xor_sync(mask, hi[0], off);
    r.lo[0] = __shfl_xor_sync(mask, lo[0], off);
    return r;
  }
  __device__ __forceinline__ double value() const { return (double)hi[0] + (double)lo[0]; }
};

__device__ __forceinline__ void ff_fma(SumFF& a, float v, float g) {
  const float p = v * g;
  const float e = fmaf(v, g, -p);  // exact: v * g = p + e
  a.add_pair(p, e);
}

// float clamp on the integer pipe (same ordering key as dkey)
__device__ __forceinline__ int fkey(float x) {
  const int b = __float_as_int(x);
  return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float clamp_f(float x, float lo, float hi) {
  const int k = fkey(x);
  if (k < fkey(lo)) return lo;
  if (k > fkey(hi)) return hi;
  return x;
}

struct DevModel32 {
  const float* chat;
  const float* lhat;
  const float* uhat;
  const float* bhat;
  const int8_t* ge;
};

// FP32-bulk iterates.  x and y are carried as float-float pairs (x + xlo):
// the gathers and the matrix products read the high parts only, while the
// updates x - tau g and y + sigma r are added exactly into the pair, so that
// steps far below an FP32 unit of the iterate (tiny tau or sigma) still move
// it.  xbar is FP32 (it is only gathered).  The running sums are float-float
// pairs too (8 bytes, like a double), so the iteration does no FP64 work;
// they are widened to FP64 at each check.
struct DevIter32 {
  float* x;
  float* y;
  float* xbar;
  float2* sum_x;
  float2* sum_y;
  float* xlo;
  float* ylo;
  float2* xa;  // Halpern loop: the anchor z_0 as float-float pairs (hi, lo)
  float2* ya;
};

// (hi, lo) += (a, b) for float-float pairs, TwoSum of the high parts
__device__ __forceinline__ void ff_add(float2& s, float a, float b) {
  const float t = s.x + a;
  const float bb = t - s.x;
  const float err = (s.x - (t - bb)) + (a - bb);
  const float l = s.y + (err + b);
  const float h = t + l;
  s.y = l - (h - t);
  s.x = h;
}

// (hi, lo) + a * b, with a * b formed exactly (fma) and both sums TwoSum:
// the pair keeps about 48 bits
__device__ __forceinline__ void ff_axpy(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  const float l = lo + (err + e);
  const float h2 = s + l;
  const float b2 = h2 - s;
  lo = (s - (h2 - b2)) + (l - b2);
  hi = h2;
}

// x' = proj_[l,u](x - tau (c - A'y)),  x_bar = 2x' - x,  sum_x += x'  (FP32 bulk)
struct PrimalOp32 {
  using Acc = SumFF;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  static constexpr int NG = 1;
  using VT = float;
  using GT = float;
  const Scalars* S;
  int it;
  const float* __restrict__ y;
  DevModel32 md;
  DevIter32 w;
  __device__ bool skip() const { return S->done || S->k + it >= S->max_iters; }
  __device__ double row_ctx(int) const { return 0.0; }
  __device__ const float* gsrc(int) const { return y; }
  __device__ void accum(Acc& a, double, float v, const GV<float, 1>& g) const { ff_fma(a, v, g.v[0]); }
  struct Pre {
    float c, l, u, x, xl, tau;
    float2 sx;
  };
  __device__ Pre prefetch(int j) const {
    return Pre{md.chat[j], md.lhat[j], md.uhat[j], w.x[j], w.xlo[j], (float)S->tau, w.sum_x[j]};
  }
  __device__ void epilogue_pre(int j, const Acc& a, const Pre& p, double*) const {
    // g = c - (A'y) from the float-float row sum: c - hi is exact when the two
    // are close (Sterbenz), so g keeps its relative precision near optimality
    const float g = (p.c - a.hi[0]) - a.lo[0];
    float xh = p.x, xl = p.xl;
    ff_axpy(xh, xl, -p.tau, g);
    // projection onto [l, u] of the pair (a clamped value carries no low part)
    const float xc = clamp_f(xh, p.l, p.u);
    if (xc != xh || (xh == p.l && xl < 0.0f) || (xh == p.u && xl > 0.0f)) {
      xh = xc;
      xl = 0.0f;
    }
    w.xbar[j] = 2.0f * xh - p.x;
    float2 sx = p.sx;
    ff_add(sx, xh, xl);
    w.sum_x[j] = sx;
    w.x[j] = xh;
    w.xlo[j] = xl;
  }
};

// y' = y + sigma (b - A x_bar), y' >= 0 on '>' rows,  sum_y += y'  (FP32 bulk)
struct DualOp32 {
  using Acc = SumFF;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  static constexpr int NG = 1;
  using VT = float;
  using GT = float;
  const Scalars* S;
  int it;
  const float* __restrict__ xbar;
  DevModel32 md;
  DevIter32 w;
  __device__ bool skip() const { return S->done || S->k + it >= S->max_iters; }
  __device__ double row_ctx(int) const { return 0.0; }
  __device__ const float* gsrc(int) const { return xbar; }
  __device__ void accum(Acc& a, double, float v, const GV<float, 1>& g) const { ff_fma(a, v, g.v[0]); }
  struct Pre {
    float b, y, yl, sigma;
    int8_t ge;
    float2 sy;
  };
  __device__ Pre prefetch(int i) const {
    return Pre{md.bhat[i], w.y[i], w.ylo[i], (float)S->sigma, md.ge[i], w.sum_y[i]};
  }
  __device__ void epilogue_pre(int i, const Acc& a, const Pre& p, double*) const {
    const float r = (p.b - a.hi[0]) - a.lo[0];
    float yh = p.y, yl = p.yl;
    ff_axpy(yh, yl, p.sigma, r);
    // y >= 0 on '>' rows: a negative pair projects to (0, 0); y = 0 where fixed
    if (p.ge && (p.ge == kRowDualZero || yh < 0.0f || (yh == 0.0f && yl < 0.0f))) {
      yh = 0.0f;
      yl = 0.0f;
    }
    float2 sy = p.sy;
    ff_add(sy, yh, yl);
    w.sum_y[i] = sy;
    w.y[i] = yh;
    w.ylo[i] = yl;
  }
};


// ---------------------------------------------------------------------------
// The Halpern loop in FP32 bulk: the PDHG output T(z) is formed as in
// PrimalOp32 / DualOp32 (FP32 values and gathers, float-float row sums and
// iterates), and the anchored combination is taken on float-float pairs,
//   r = T(z) + rho (T(z) - z),   z <- r + s (z_0 - r),   s = 1 - w = hs[it],
// which is the Halpern step w r + (1 - w) z_0 of the FP64 operators.  No
// FP64 arithmetic runs except on a check step, which widens T(z) and
// z - T(z) to the FP64 buffers the FP64 evaluation reads.
// ---------------------------------------------------------------------------

// (ah, al) - (bh, bl) as a normalised pair: TwoSum of the high parts, the low
// parts added to its error
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl, float& h, float& l) {
  const float s = ah - bh;
  const float bb = s - ah;
  const float err = (ah - (s - bb)) + (-bh - bb);
  const float t = err + (al - bl);
  const float h2 = s + t;
  const float b2 = h2 - s;
  l = (s - (h2 - b2)) + (t - b2);
  h = h2;
}

// (hi, lo) += a * (bh, bl): a * bh exact (fma), a * bl rounded into the low
// part, both sums TwoSum
__device__ __forceinline__ void ff_axpy_ff(float& hi, float& lo, float a, float bh, float bl) {
  const float p = a * bh;
  const float e = fmaf(a, bl, fmaf(a, bh, -p));
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  const float l = lo + (err + e);
  const float h2 = s + l;
  const float b2 = h2 - s;
  lo = (s - (h2 - b2)) + (l - b2);
  hi = h2;
}

// z <- r + s (z_0 - r) with r = T(z) + rho (T(z) - z), all pairs
__device__ __forceinline__ void ff_halpern(float th, float tl, float zh, float zl, float2 z0, float rho, float s,
                                           float& oh, float& ol) {
  float dh, dl;
  ff_sub(th, tl, zh, zl, dh, dl);
  float rh = th, rl = tl;
  ff_axpy_ff(rh, rl, rho, dh, dl);
  float eh, el;
  ff_sub(z0.x, z0.y, rh, rl, eh, el);
  ff_axpy_ff(rh, rl, s, eh, el);
  oh = rh;
  ol = rl;
}

// FP32-bulk Halpern iterate.  z = (x, y) and the anchor z_0 = (xa, ya) are
// float-float pairs.  The gathered vectors are differences from the anchor,
// gx = fl(x_bar - x_0) (gathered by the dual pass) and gy = fl(y - y_0)
// (gathered by the primal pass), and q = c_hat - A_hat' y_0, r0 = b_hat -
// A_hat x_0 are formed in FP64 at every anchor (AnchorColsOp, AnchorRowsOp)
// and kept as float-float pairs, so that the steps use
//   c_hat - A_hat' y = q - A_hat' gy,   b_hat - A_hat x_bar = r0 - A_hat gx.
// The FP32 rounding of the matrix values and of the gathered vectors then
// scales with the distance from the anchor instead of with the iterate, and
// the FP32 map's fixed point is that of the FP64 LP (up to that rounding of
// a vanishing correction).
struct DevH32 {
  float* x;
  float* xlo;
  float* y;
  float* ylo;
  float2* xa;
  float2* ya;
  float* gx;
  float* gy;
  float2* q;
  float2* r0;
};

// a double as a float-float pair
__device__ __forceinline__ float2 to_ff(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// q = c_hat - A_hat' y_0 at the anchor (pass over A', FP64 matrix and anchor)
struct AnchorColsOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  const Scalars* S;
  int force;  // 1: at the start of a phase; 0: only after a restart to T(z)
  const double* __restrict__ y0;
  const double* __restrict__ chat;
  float2* __restrict__ q;
  __device__ bool skip() const { return !force && (S->done || S->restart_to != 3); }
  __device__ double row_ctx(int) const { return 0.0; }
  __device__ const double* gsrc(int) const { return y0; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int j, const Acc& a, double*) const { q[j] = to_ff(chat[j] - a.v[0]); }
};

// r0 = b_hat - A_hat x_0 at the anchor (pass over A)
struct AnchorRowsOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  const Scalars* S;
  int force;
  const double* __restrict__ x0;
  const double* __restrict__ bhat;
  float2* __restrict__ r0;
  __device__ bool skip() const { return !force && (S->done || S->restart_to != 3); }
  __device__ double row_ctx(int) const { return 0.0; }
  __device__ const double* gsrc(int) const { return x0; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int i, const Acc& a, double*) const { r0[i] = to_ff(bhat[i] - a.v[0]); }
};

// (h, l) + (a, b) as a normalised pair
__device__ __forceinline__ void ff_sum(float ah, float al, float bh, float bl, float& h, float& l) {
  ff_sub(ah, al, -bh, -bl, h, l);
}

// kUnitRho: the reflection is 1, so the reflected point T + (T - z) is the
// x_bar pair the epilogue already forms (the general operator recomputes it)
template <bool kUnitRho>
struct PrimalOpH32T {
  using Acc = SumFF;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  static constexpr int NG = 1;
  using VT = float;
  using GT = float;
  const Scalars* S;
  int it, last_it, probe;
  DevModel32 md;  // lhat, uhat (c_hat enters through w.q)
  DevH32 w;
  DevHalpern h;
  __device__ bool skip() const { return S->done || (!probe && S->k + it >= S->max_iters); }
  __device__ double row_ctx(int) const { return 0.0; }
  __device__ const float* gsrc(int) const { return w.gy; }
  __device__ void accum(Acc& a, double, float v, const GV<float, 1>& g) const { ff_fma(a, v, g.v[0]); }
  struct Pre {
    float l, u, x, xl, tau, s, rho;
    float2 q, x0;
    bool last;
  };
  __device__ Pre prefetch(int j) const {
    const bool last = probe || it == last_it || S->k + it + 1 == S->max_iters;
    return Pre{md.lhat[j], md.uhat[j], w.x[j], w.xlo[j], (float)S->tau, h.hs[it], (float)S->rho, w.q[j],
               w.xa[j], last};
  }
  __device__ void epilogue_pre(int j, const Acc& a, const Pre& p, double*) const {
    // g = c_hat - A_hat' y = q - A_hat' gy
    const float g = (p.q.x - a.hi[0]) + (p.q.y - a.lo[0]);
    float th = p.x, tl = p.xl;
    ff_axpy(th, tl, -p.tau, g);
    const float xc = clamp_f(th, p.l, p.u);
    if (xc != th || (th == p.l && tl < 0.0f) || (th == p.u && tl > 0.0f)) {
      th = xc;
      tl = 0.0f;
    }
    // x_bar = T - z + T, gathered as its difference from the anchor
    float dh, dl;
    ff_sub(th, tl, p.x, p.xl, dh, dl);
    float bh, bl;
    ff_sum(th, tl, dh, dl, bh, bl);
    float eh, el;
    ff_sub(bh, bl, p.x0.x, p.x0.y, eh, el);
    w.gx[j] = eh + el;
    if (!probe) {
      float oh, ol;
      if constexpr (kUnitRho) {
        // z <- r + s (z_0 - r) with r = x_bar = (bh, bl), and z_0 - r =
        // -(eh, el) exactly (TwoSum differences are odd in their arguments)
        float rh = bh, rl = bl;
        ff_axpy_ff(rh, rl, p.s, -eh, -el);
        oh = rh;
        ol = rl;
      } else {
        ff_halpern(th, tl, p.x, p.xl, p.x0, p.rho, p.s, oh, ol);
      }
      w.x[j] = oh;
      w.xlo[j] = ol;
    }
    if (p.last) {
      h.xp[j] = (double)th + (double)tl;
      h.dx[j] = -((double)dh + (double)dl);
    }
  }
};
using PrimalOpH32 = PrimalOpH32T<false>;

struct DualOpH32 {
  using Acc = SumFF;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  static constexpr int NG = 1;
  using VT = float;
  using GT = float;
  const Scalars* S;
  int it, last_it, probe;
  DevModel32 md;  // ge (b_hat enters through w.r0)
  DevH32 w;
  DevHalpern h;
  __device__ bool skip() const { return S->done || (!probe && S->k + it >= S->max_iters); }
  __device__ double row_ctx(int) const { return 0.0; }
  __device__ const float* gsrc(int) const { return w.gx; }
  __device__ void accum(Acc& a, double, float v, const GV<float, 1>& g) const { ff_fma(a, v, g.v[0]); }
  struct Pre {
    float y, yl, sigma, s, rho;
    float2 r0, y0;
    int8_t ge;
    bool last;
  };
  __device__ Pre prefetch(int i) const {
    const bool last = probe || it == last_it || S->k + it + 1 == S->max_iters;
    return Pre{w.y[i], w.ylo[i], (float)S->sigma, h.hs[it], (float)S->rho, w.r0[i], w.ya[i], md.ge[i], last};
  }
  __device__ void epilogue_pre(int i, const Acc& a, const Pre& p, double*) const {
    // r = b_hat - A_hat x_bar = r0 - A_hat gx
    const float r = (p.r0.x - a.hi[0]) + (p.r0.y - a.lo[0]);
    float th = p.y, tl = p.yl;
    ff_axpy(th, tl, p.sigma, r);
    // y >= 0 on '>' rows; y = 0 on a row whose dual is fixed
    if (p.ge && (p.ge == kRowDualZero || th < 0.0f || (th == 0.0f && tl < 0.0f))) {
      th = 0.0f;
      tl = 0.0f;
    }
    float yh = p.y, yl = p.yl;
    if (!probe) {
      ff_halpern(th, tl, p.y, p.yl, p.y0, p.rho, p.s, yh, yl);
      w.y[i] = yh;
      w.ylo[i] = yl;
    }
    // the next primal pass gathers the new y as its difference from the anchor
    float eh, el;
    ff_sub(yh, yl, p.y0.x, p.y0.y, eh, el);
    w.gy[i] = eh + el;
    if (p.last) {
      float dh, dl;
      ff_sub(p.y, p.yl, th, tl, dh, dl);
      h.yp[i] = (double)th + (double)tl;
      h.dy[i] = (double)dh + (double)dl;
    }
  }
};

}  // namespace pdhgc
