// The batched solver's persistent kernel: one CTA runs the whole method on
// one LP at a time (see batch.cu for the design).  Included only by the
// instantiation units batch_k_*.cu.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/pdhgc.h"
#include "batch_desc.h"
#include "kernels.cuh"

namespace pdhgc {

// ---- CTA-level building blocks --------------------------------------------

// one pass over the rows of a CSR: G lanes per row, rows round-robin over the
// CTA's groups; gathers by plain loads (shared or global memory)
template <int BT, class Op>
__device__ void cta_rows(const int* __restrict__ rp, const int* __restrict__ col,
                         const typename Op::VT* __restrict__ val, int rows, int G, const Op& op, double* part) {
  using PF = Prefetcher<Op>;
  using GT = typename Op::GT;
  constexpr int NG = Op::NG;
  const int tid = threadIdx.x;
  const int lane = tid & (G - 1);
  const int gid = tid / G;
  const int ngroups = BT / G;
  for (int r0 = 0; r0 < rows; r0 += ngroups) {
    const int r = r0 + gid;
    const bool has = r < rows;
    typename Op::Acc acc;
    acc.zero();
    typename PF::Pre pre{};
    if (has) {
      if (lane == 0) pre = PF::get(op, r);
      const double rc = op.row_ctx(r);
      const int e0 = rp[r], e1 = rp[r + 1];
      for (int e = e0 + lane; e < e1; e += G) {
        const int cc = col[e];
        GV<GT, NG> g;
#pragma unroll
        for (int i = 0; i < NG; ++i) g.v[i] = op.gsrc(i)[cc];
        op.accum(acc, rc, val[e], g);
      }
    }
    for (int off = G >> 1; off > 0; off >>= 1) acc.add(acc.shfl_xor(0xffffffffu, off));
    if (has && lane == 0) PF::epilogue(op, r, acc, pre, part);
  }
}

// one matrix of an LP as a pass reads it: CSR for the long rows, SELL-32
// slices for the rest
template <class VT>
struct BMat {
  const int* rp;
  const int* col;
  const VT* val;
  int rows, long_rows, nslices;
  const int* sptr;
  const int* sw;
  const int* scol;
  const VT* sval;
};

// asks L2 to fetch [p, p + bytes) from DRAM ahead of its use (a hint: no
// data moves into the SM and nothing waits on it); p 16-byte aligned, bytes a
// multiple of 16
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  if (bytes != 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (bytes & 15) == 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// matrix entries in flight per lane in the batched SELL pass, and how many of
// its own slices ahead a warp asks L2 for (tuning knobs)
#ifndef PDHGC_BATCH_KBATCH
#define PDHGC_BATCH_KBATCH 4
#endif
#ifndef PDHGC_BATCH_AHEAD
#define PDHGC_BATCH_AHEAD 1
#endif
constexpr int kBatchB = PDHGC_BATCH_KBATCH;

// lane 0 of the warp prefetches slice s's values and indices into L2
template <class VT>
__device__ __forceinline__ void prefetch_slice(const BMat<VT>& M, int s) {
  const int base = M.sptr[s], w = M.sw[s];
  prefetch_l2(M.sval + base, (unsigned)(w * kSellH * sizeof(VT)));
  prefetch_l2(M.scol + base, (unsigned)(w * kSellH * sizeof(int)));
}

// one pass: long rows with a warp each (CSR), then SELL-32 slices with a lane
// per row and kBatch coalesced loads in flight, slices round-robin over warps.
// Each warp asks L2 for its next slice's values and indices while it works on
// the current one: one CTA streams its LP's matrix alone, and without the
// look-ahead every batch of loads waits a full DRAM latency.
template <int BT, class Op>
__device__ void cta_pass(const BMat<typename Op::VT>& M, const Op& op, double* part) {
  using PF = Prefetcher<Op>;
  using VT = typename Op::VT;
  using GT = typename Op::GT;
  constexpr int NG = Op::NG;
  constexpr int W = BT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0 && warp < M.nslices) prefetch_slice(M, warp);
  if (M.long_rows > 0) cta_rows<BT>(M.rp, M.col, M.val, M.long_rows, 32, op, part);
  for (int s = warp; s < M.nslices; s += W) {
    if (lane == 0 && s + PDHGC_BATCH_AHEAD * W < M.nslices) prefetch_slice(M, s + PDHGC_BATCH_AHEAD * W);
    const int base = M.sptr[s], w = M.sw[s];
    const int r = M.long_rows + s * kSellH + lane;
    const bool has = r < M.rows;
    const int len = has ? M.rp[r + 1] - M.rp[r] : 0;
    typename PF::Pre pre{};
    if (has) pre = PF::get(op, r);
    const double rc = has ? op.row_ctx(r) : 0.0;
    typename Op::Acc acc;
    acc.zero();
    for (int j = 0; j < w; j += kBatchB) {
      VT v[kBatchB];
      int c[kBatchB];
#pragma unroll
      for (int u = 0; u < kBatchB; ++u)
        if (j + u < len) {
          v[u] = ld_stream(M.sval + base + (j + u) * kSellH + lane);
          c[u] = ld_stream(M.scol + base + (j + u) * kSellH + lane);
        }
      GV<GT, NG> g[kBatchB];
#pragma unroll
      for (int u = 0; u < kBatchB; ++u)
        if (j + u < len)
#pragma unroll
          for (int i = 0; i < NG; ++i) g[u].v[i] = op.gsrc(i)[c[u]];
#pragma unroll
      for (int u = 0; u < kBatchB; ++u)
        if (j + u < len) op.accum(acc, rc, v[u], g[u]);
    }
    if (has) PF::epilogue(op, r, acc, pre, part);
  }
}

// deterministic CTA fold of part[0..nq) (sum, or max where mask bit set) into out[]
template <int BT>
__device__ void cta_fold(const double* part, int nq, unsigned max_mask, double* out, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = BT / 32;
  for (int q = 0; q < nq; ++q) {
    const bool is_max = (max_mask >> q) & 1u;
    double v = part[q];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = is_max ? fmax(v, o) : v + o;
    }
    if (lane == 0) red[q * W + warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    const int q = threadIdx.x;
    const bool is_max = (max_mask >> q) & 1u;
    double v = red[q * W];
    for (int w = 1; w < W; ++w) v = is_max ? fmax(v, red[q * W + w]) : v + red[q * W + w];
    out[q] = v;
  }
  __syncthreads();
}

template <int BT>
__device__ double cta_sum(double v, double* red) {
  double part[1] = {v};
  double out[1];
  __shared__ double s_out[1];
  cta_fold<BT>(part, 1, 0u, s_out, red);
  out[0] = s_out[0];
  __syncthreads();
  return out[0];
}

// ---- one LP, one CTA ------------------------------------------------------

template <class VT, int BT>
struct LpSolver {
  static constexpr bool kF32 = std::is_same<VT, float>::value;
  const LpDesc& d;
  const BatchParams& bp;
  Scalars* S;
  double* red;  // [32 * BT / 32] reduction scratch
  double* q;    // [32] folded quantities
  VT* s_y;      // gathered y (shared or global)
  VT* s_xbar;   // gathered x_bar (shared or global)
  const int* queue;  // [0] next LP of the queue, [1] LPs running
  int count;

  __device__ void fill(double* a, int n, double v) const {
    for (int i = threadIdx.x; i < n; i += BT) a[i] = v;
  }
  // one pass over A (or A') in the layout the tuner chose
  template <class Op>
  __device__ void passA(const BMat<typename Op::VT>& M, const Op& op, double* part) const {
    if (d.sell) cta_pass<BT>(M, op, part);
    else cta_rows<BT>(M.rp, M.col, M.val, M.rows, d.gA, op, part);
  }
  template <class Op>
  __device__ void passT(const BMat<typename Op::VT>& M, const Op& op, double* part) const {
    if (d.sell) cta_pass<BT>(M, op, part);
    else cta_rows<BT>(M.rp, M.col, M.val, M.rows, d.gT, op, part);
  }
  // kind 0: original values, 1: scaled FP64
  __device__ BMat<double> matA(int kind) const {
    return BMat<double>{d.A_rp, d.A_col, kind ? d.A_hat : d.A_val, d.m, d.A_long, d.A_ns,
                        d.A_sptr, d.A_sw, d.A_scol, kind ? d.A_shat : d.A_sval};
  }
  __device__ BMat<double> matT(int kind) const {
    return BMat<double>{d.T_rp, d.T_col, kind ? d.T_hat : d.T_val, d.n, d.T_long, d.T_ns,
                        d.T_sptr, d.T_sw, d.T_scol, kind ? d.T_shat : d.T_sval};
  }
  __device__ BMat<float> matA32() const {
    return BMat<float>{d.A_rp, d.A_col, d.A_hat32, d.m, d.A_long, d.A_ns, d.A_sptr, d.A_sw, d.A_scol, d.A_shat32};
  }
  __device__ BMat<float> matT32() const {
    return BMat<float>{d.T_rp, d.T_col, d.T_hat32, d.n, d.T_long, d.T_ns, d.T_sptr, d.T_sw, d.T_scol, d.T_shat32};
  }

  __device__ DevModel model(bool corner) const {
    return corner ? DevModel{d.chat_c, d.lhat_c, d.uhat_c, d.bhat, d.Dr, d.Dc, d.ge_c}
                  : DevModel{d.chat, d.lhat, d.uhat, d.bhat, d.Dr, d.Dc, d.ge};
  }
  __device__ DevModel32 model32(bool corner) const {
    return corner ? DevModel32{d.chat_c32, d.lhat_c32, d.uhat_c32, d.bhat32, d.ge_c}
                  : DevModel32{d.chat32, d.lhat32, d.uhat32, d.bhat32, d.ge};
  }
  // FP64 view of the current iterates for the evaluation operators
  __device__ DevIter iter64() const {
    double* y = kF32 ? d.y : (double*)s_y;
    double* xbar = kF32 ? d.xbar : (double*)s_xbar;
    return DevIter{d.x, y, xbar, d.sum_x, d.sum_y, d.x_r, d.y_r};
  }

  // a0: Ruiz + Pock-Chambolle, scaled copies, power iteration
  __device__ void setup() {
    const int m = d.m, n = d.n;
    fill(d.Dr, m, 1.0);
    fill(d.Dc, n, 1.0);
    __syncthreads();
    double part[1] = {0.0};
    for (int pass = 0; pass < bp.ruiz_iters; ++pass) {
      passA(matA(0), ScaleMaxOp<false>{d.Dr, d.Dc, d.rfac}, part);
      passT(matT(0), ScaleMaxOp<true>{d.Dc, d.Dr, d.cfac}, part);
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += BT) d.Dr[i] *= d.rfac[i];
      for (int j = threadIdx.x; j < n; j += BT) d.Dc[j] *= d.cfac[j];
      __syncthreads();
    }
    passA(matA(0), ScaleSumOp<false>{d.Dr, d.Dc, d.rfac}, part);
    passT(matT(0), ScaleSumOp<true>{d.Dc, d.Dr, d.cfac}, part);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += BT) d.Dr[i] *= d.rfac[i];
    for (int j = threadIdx.x; j < n; j += BT) d.Dc[j] *= d.cfac[j];
    __syncthreads();
    // scaled matrix and vectors: (D_r a) D_c, D_r b, D_c c, l / D_c, u / D_c
    for (int r = threadIdx.x; r < m; r += BT)
      for (int e = d.A_rp[r]; e < d.A_rp[r + 1]; ++e) {
        const double v = (d.Dr[r] * d.A_val[e]) * d.Dc[d.A_col[e]];
        d.A_hat[e] = v;
        if (kF32) d.A_hat32[e] = (float)v;
      }
    for (int j = threadIdx.x; j < n; j += BT)
      for (int e = d.T_rp[j]; e < d.T_rp[j + 1]; ++e) {
        const double v = (d.Dr[d.T_col[e]] * d.T_val[e]) * d.Dc[j];
        d.T_hat[e] = v;
        if (kF32) d.T_hat32[e] = (float)v;
      }
    __syncthreads();
    for (int k = threadIdx.x; k < d.A_slots; k += BT) {
      const int e = d.A_smap[k];
      const double v = e >= 0 ? d.A_hat[e] : 0.0;
      d.A_shat[k] = v;
      if (kF32) d.A_shat32[k] = (float)v;
    }
    for (int k = threadIdx.x; k < d.T_slots; k += BT) {
      const int e = d.T_smap[k];
      const double v = e >= 0 ? d.T_hat[e] : 0.0;
      d.T_shat[k] = v;
      if (kF32) d.T_shat32[k] = (float)v;
    }
    double nb2 = 0.0, nc2 = 0.0;
    for (int i = threadIdx.x; i < m; i += BT) {
      const double bh = d.Dr[i] * d.b_int[i];
      d.bhat[i] = bh;
      nb2 += bh * bh;
      if (kF32) d.bhat32[i] = (float)bh;
    }
    for (int j = threadIdx.x; j < n; j += BT) {
      const double ch = d.Dc[j] * d.c[j];
      d.chat[j] = ch;
      d.lhat[j] = d.l[j] / d.Dc[j];
      d.uhat[j] = d.u[j] / d.Dc[j];
      nc2 += ch * ch;
      if (kF32) {
        d.chat32[j] = (float)ch;
        d.lhat32[j] = (float)d.lhat[j];
        d.uhat32[j] = (float)d.uhat[j];
      }
    }
    nb2 = cta_sum<BT>(nb2, red);
    nc2 = cta_sum<BT>(nc2, red);
    // power iteration on A_hat' A_hat from v = 1/sqrt(n)
    fill(d.pi_v, n, 1.0 / sqrt((double)n));
    __syncthreads();
    bool zero = false;
    for (int k = 0; k < bp.power_iters && !zero; ++k) {
      passA(matA(1), SpmvOp<false>{S, d.pi_v, d.pi_u}, part);
      __syncthreads();
      double pw[1] = {0.0};
      passT(matT(1), SpmvOp<true>{S, d.pi_u, d.pi_w}, pw);
      const double nw = sqrt(cta_sum<BT>(pw[0], red));
      if (nw == 0.0) {
        zero = true;
        break;
      }
      for (int j = threadIdx.x; j < n; j += BT) d.pi_v[j] = d.pi_w[j] / nw;
      __syncthreads();
    }
    double sigma_max = 0.0;
    if (!zero) {
      double pu[1] = {0.0};
      passA(matA(1), SpmvOp<true>{S, d.pi_v, d.pi_u}, pu);
      sigma_max = sqrt(cta_sum<BT>(pu[0], red));
    }
    if (threadIdx.x == 0) {
      S->sigma_max = sigma_max;
      S->eta = sigma_max > 0.0 ? bp.eta_factor / sigma_max : 1.0;
      S->nb_hat = sqrt(nb2);
      S->nc_hat = sqrt(nc2);
      d.keep[0] = S->eta;
      d.keep[1] = S->sigma_max;
      d.keep[2] = S->nb_hat;
      d.keep[3] = S->nc_hat;
    }
    __syncthreads();
  }

  // start of a phase (mirrors k_init_scalars / k_init_iterates)
  __device__ void init_phase(int phase, const double* x_start, double nch, double nc_user) {
    const int m = d.m, n = d.n;
    const DevModel md = model(phase == 1);
    for (int j = threadIdx.x; j < n; j += BT) {
      const double x0 = x_start ? x_start[j] : fmin(fmax(0.0, md.lhat[j]), md.uhat[j]);
      d.x[j] = x0;
      d.x_r[j] = x0;
      d.sum_x[j] = 0.0;
      if (kF32) {
        const float h = (float)x0;
        d.x32[j] = h;
        d.x32lo[j] = (float)(x0 - (double)h);
        d.sx32[j] = make_float2(0.f, 0.f);
        d.xa32[j] = make_float2(h, d.x32lo[j]);
        s_xbar[j] = (VT)h;
      } else {
        ((double*)s_xbar)[j] = x0;
      }
    }
    for (int i = threadIdx.x; i < m; i += BT) {
      s_y[i] = (VT)0;
      if (kF32) {
        d.y[i] = 0.0;
        d.y32lo[i] = 0.0f;
        d.yh32[i] = 0.0f;
        d.sy32[i] = make_float2(0.f, 0.f);
        d.ya32[i] = make_float2(0.f, 0.f);
      }
      d.y_r[i] = 0.0;
      d.sum_y[i] = 0.0;
    }
    if (threadIdx.x == 0) {
      S->eps_rel = phase ? bp.c_eps_rel : bp.eps_rel;
      S->beta_suff = bp.beta_suff;
      S->beta_nec = bp.beta_nec;
      S->beta_art = bp.beta_art;
      S->theta = bp.theta;
      S->time_limit_s = phase ? bp.c_time_limit_s : bp.time_limit_s;
      S->nb = d.b_norm;
      S->nc = nc_user;
      S->max_iters = phase ? bp.c_max_iters : bp.max_iters;
      S->min_iters = phase ? bp.c_min_iters : 0;
      S->check_period = bp.check_period;
      S->phase = phase;
      S->stop_rule = phase ? bp.stop_rule : 0;
      S->omega = (nch > 1e-10 && S->nb_hat > 1e-10) ? nch / S->nb_hat : 1.0;
      S->tau = S->eta / S->omega;
      S->sigma = S->eta * S->omega;
      S->k = 0;
      S->t = 0;
      S->restarts = 0;
      S->chunks = 0;
      S->max_chunks = S->max_iters / S->check_period + 2;
      S->done = 0;
      S->status = PDHGC_STATUS_NONE;
      S->chosen = 0;
      S->restart_to = 0;
      S->inv_t = 0.0;
      S->at_check = 0;
      S->at_limit = 0;
      S->kkt_prev = INFINITY;
      S->algorithm = bp.algorithm;
      S->rho = bp.rho;
      S->pid_kp = bp.pid_kp;
      S->pid_ki = bp.pid_ki;
      S->pid_kd = bp.pid_kd;
      S->fpr = S->fpr0 = 0.0;
      S->fpr_prev = INFINITY;
      S->pid_int = 0.0;
      S->pid_eprev = 0.0;
      S->error = 0;
      S->t0_ns = global_ns();
    }
    __syncthreads();
  }

  // the 22 KKT quantities of the current and average points, folded
  __device__ void evaluate(bool corner) {
    const DevModel md = model(corner);
    const DevIter w = iter64();
    double pr[10];
    for (int i = 0; i < 10; ++i) pr[i] = 0.0;
    passA(matA(1), EvalRowsOp{S, w.x, w.sum_x, w.y, w.sum_y, w.y_r, md}, pr);
    cta_fold<BT>(pr, 10, EvalRowsOp::kMaxMask, q, red);
    double pc[12];
    for (int i = 0; i < 12; ++i) pc[i] = 0.0;
    passT(matT(1), EvalColsOp{S, w.y, w.sum_y, w.x, w.sum_x, w.x_r, md}, pc);
    cta_fold<BT>(pc, 12, EvalColsOp::kMaxMask, q + 10, red);
  }

  __device__ void iterate(bool corner, int it) {
    double part[1] = {0.0};
    if constexpr (kF32) {
      const DevModel32 md = model32(corner);
      const DevIter32 w{d.x32, (float*)s_y, (float*)s_xbar, d.sx32, d.sy32, d.x32lo, d.y32lo};
      passT(matT32(), PrimalOp32{S, it, (float*)s_y, md, w}, part);
      __syncthreads();
      passA(matA32(), DualOp32{S, it, (float*)s_xbar, md, w}, part);
      __syncthreads();
    } else {
      const DevModel md = model(corner);
      const DevIter w{d.x, (double*)s_y, (double*)s_xbar, d.sum_x, d.sum_y, d.x_r, d.y_r};
      passT(matT(1), PrimalOp{S, it, (double*)s_y, md, w}, part);
      __syncthreads();
      passA(matA(1), DualOp{S, it, (double*)s_xbar, md, w}, part);
      __syncthreads();
    }
  }

  // the restarted loop of one phase (mirrors the graph body of run_phase)
  __device__ void loop(bool corner) {
    const int m = d.m, n = d.n;
    const DevModel md = model(corner);
    if (kF32) {
      for (int i = threadIdx.x; i < m; i += BT) d.y[i] = (double)((float*)s_y)[i] + (double)d.y32lo[i];
    }
    __syncthreads();
    evaluate(corner);
    if (threadIdx.x == 0) decide_step(S, q, 0);
    __syncthreads();
    while (true) {
      const long long k0 = S->k, kmax = S->max_iters;
      const int P = S->check_period;
      for (int i = 0; i < P && k0 + i < kmax; ++i) iterate(corner, i);
      if (threadIdx.x == 0) {
        long long run = kmax - k0;
        if (run > P) run = P;
        if (run < 0) run = 0;
        S->k += run;
        S->t += run;
        S->inv_t = S->t > 0 ? 1.0 / (double)S->t : 0.0;
        S->at_check = (S->k % P) == 0;
        S->at_limit = S->k >= kmax;
        S->chunks += 1;
        if (S->chunks > S->max_chunks) S->at_limit = 1;
      }
      if (kF32) {
        for (int j = threadIdx.x; j < n; j += BT) {
          d.x[j] = fmin(fmax((double)d.x32[j] + (double)d.x32lo[j], md.lhat[j]), md.uhat[j]);
          d.sum_x[j] = (double)d.sx32[j].x + (double)d.sx32[j].y;
        }
        for (int i = threadIdx.x; i < m; i += BT) {
          d.y[i] = (double)((float*)s_y)[i] + (double)d.y32lo[i];
          d.sum_y[i] = (double)d.sy32[i].x + (double)d.sy32[i].y;
        }
      }
      __syncthreads();
      evaluate(corner);
      if (threadIdx.x == 0) {
        decide_step(S, q, 1);
        // tail handoff (reads of the queue counters, no wait)
        if (!S->done && bp.handoff_running > 0 && S->k >= bp.handoff_min_iters &&
            *(volatile const int*)&queue[0] >= count && *(volatile const int*)&queue[1] <= bp.handoff_running) {
          S->done = 1;
          S->status = kStatusHandoff;
        }
      }
      __syncthreads();
      if (S->done) break;
      const int rt = S->restart_to;
      if (rt != 0) {
        const double inv_t = S->inv_t;
        const DevIter w = iter64();
        for (int j = threadIdx.x; j < n; j += BT) {
          const double xn = rt == 2 ? w.sum_x[j] * inv_t : w.x[j];
          w.x[j] = xn;
          w.x_r[j] = xn;
          w.sum_x[j] = 0.0;
          if (kF32) {
            d.sx32[j] = make_float2(0.f, 0.f);
            if (rt == 2) {
              const float h = (float)xn;
              d.x32[j] = h;
              d.x32lo[j] = (float)(xn - (double)h);
            }
          }
        }
        for (int i = threadIdx.x; i < m; i += BT) {
          const double yn = rt == 2 ? w.sum_y[i] * inv_t : w.y[i];
          w.y[i] = yn;
          w.y_r[i] = yn;
          w.sum_y[i] = 0.0;
          if (kF32) {
            d.sy32[i] = make_float2(0.f, 0.f);
            if (rt == 2) {
              const float h = (float)yn;
              ((float*)s_y)[i] = h;
              d.y32lo[i] = (float)(yn - (double)h);
            }
          }
        }
      }
      __syncthreads();
    }
  }

  // ---- the Halpern loop (mirrors the Halpern branch of run_phase) ----------
  __device__ DevHalpern hz() const { return DevHalpern{d.hxp, d.hyp, d.hdx, d.hdy, d.hw, d.hs}; }

  // the anchoring weights of the next chunk (k_halpern_weights)
  __device__ void weights_h() {
    const long long t = S->t;
    const int P = S->check_period;
    for (int i = threadIdx.x; i < P; i += BT) {
      d.hw[i] = (double)(t + i + 1) / (double)(t + i + 2);
      d.hs[i] = (float)(1.0 / (double)(t + i + 2));
    }
    __syncthreads();
  }

  // the 7 + 7 check quantities of T(z) against the anchor, folded into q
  __device__ void evaluate_h(bool corner) {
    const DevModel md = model(corner);
    double pr[7];
    for (int i = 0; i < 7; ++i) pr[i] = 0.0;
    passA(matA(1), EvalRowsH{S, hz(), d.y_r, md}, pr);
    cta_fold<BT>(pr, 7, EvalRowsH::kMaxMask, q, red);
    double pc[7];
    for (int i = 0; i < 7; ++i) pc[i] = 0.0;
    passT(matT(1), EvalColsH{S, hz(), d.x_r, md, nullptr}, pc);
    cta_fold<BT>(pc, 7, EvalColsH::kMaxMask, q + 7, red);
  }

  // the FP32-bulk Halpern iterate: gathered differences from the anchor in
  // s_xbar / s_y (shared or global memory)
  __device__ DevH32 h32() const {
    return DevH32{d.x32, d.x32lo, d.yh32, d.y32lo, d.xa32, d.ya32, (float*)s_xbar, (float*)s_y, d.q32, d.r032};
  }

  // q = c_hat - A_hat' y_0, r0 = b_hat - A_hat x_0 at the anchor (FP64)
  __device__ void anchor_h(bool corner) {
    const DevModel md = model(corner);
    double part[1] = {0.0};
    passT(matT(1), AnchorColsOp{S, 1, d.y_r, md.chat, d.q32}, part);
    passA(matA(1), AnchorRowsOp{S, 1, d.x_r, md.bhat, d.r032}, part);
    __syncthreads();
  }

  // one Halpern step (probe: T of the start point only)
  __device__ void iterate_h(bool corner, int it, int last, int probe) {
    double part[1] = {0.0};
    if constexpr (kF32) {
      const DevModel32 md = model32(corner);
      passT(matT32(), PrimalOpH32{S, it, last, probe, md, h32(), hz()}, part);
      __syncthreads();
      passA(matA32(), DualOpH32{S, it, last, probe, md, h32(), hz()}, part);
      __syncthreads();
      return;
    }
    const DevModel md = model(corner);
    const DevIter w = iter64();
    passT(matT(1), PrimalOpH{S, it, last, probe, w.y, md, w, hz()}, part);
    __syncthreads();
    passA(matA(1), DualOpH{S, it, last, probe, w.xbar, md, w, hz()}, part);
    __syncthreads();
  }

  // a restart: the iterate and the anchor become T(z)
  __device__ void restart_h(bool corner) {
    const DevIter w = iter64();
    for (int j = threadIdx.x; j < d.n; j += BT) {
      const double xn = d.hxp[j];
      d.x[j] = xn;
      d.x_r[j] = xn;
      if (kF32) {
        const float h = (float)xn, lo = (float)(xn - (double)h);
        d.x32[j] = h;
        d.x32lo[j] = lo;
        d.xa32[j] = make_float2(h, lo);
      }
    }
    for (int i = threadIdx.x; i < d.m; i += BT) {
      const double yn = d.hyp[i];
      w.y[i] = yn;
      d.y_r[i] = yn;
      if (kF32) {
        const float h = (float)yn, lo = (float)(yn - (double)h);
        d.yh32[i] = h;
        d.y32lo[i] = lo;
        d.ya32[i] = make_float2(h, lo);
        ((float*)s_y)[i] = 0.0f;  // y is the anchor now
      }
    }
    __syncthreads();
    if (kF32) anchor_h(corner);
  }

  __device__ void loop_h(bool corner) {
    if (kF32) {
      for (int i = threadIdx.x; i < d.m; i += BT) ((float*)s_y)[i] = 0.0f;  // gy: y = y_0 = 0
      __syncthreads();
      anchor_h(corner);
    }
    // the anchor's fixed-point residual: T of the start point (not an iteration)
    iterate_h(corner, 0, 0, 1);
    evaluate_h(corner);
    if (threadIdx.x == 0) decide_halpern(S, q, 0);
    __syncthreads();
    weights_h();
    while (true) {
      const long long k0 = S->k, kmax = S->max_iters;
      const int P = S->check_period;
      for (int i = 0; i < P && k0 + i < kmax; ++i) iterate_h(corner, i, P - 1, 0);
      if (threadIdx.x == 0) {
        long long run = kmax - k0;
        if (run > P) run = P;
        if (run < 0) run = 0;
        S->k += run;
        S->t += run;
        S->at_check = (S->k % P) == 0;
        S->at_limit = S->k >= kmax;
        S->chunks += 1;
        if (S->chunks > S->max_chunks) S->at_limit = 1;
      }
      __syncthreads();
      evaluate_h(corner);
      if (threadIdx.x == 0) {
        decide_halpern(S, q, 1);
        if (!S->done && bp.handoff_running > 0 && S->k >= bp.handoff_min_iters &&
            *(volatile const int*)&queue[0] >= count && *(volatile const int*)&queue[1] <= bp.handoff_running) {
          S->done = 1;
          S->status = kStatusHandoff;
        }
      }
      __syncthreads();
      if (S->done) break;
      if (S->restart_to == 3) restart_h(corner);
      weights_h();
    }
  }

  // the returned point (mirrors k_finalize)
  __device__ void finalize(double* xo, double* yo, const double* x_fallback, bool corner) {
    const DevModel md = model(corner);
    const DevIter w = iter64();
    const bool out = S->chosen == 2;  // the Halpern loop returns T(z) of its last check
    const bool avg = S->chosen == 1 && S->t > 0;
    const double inv_t = S->inv_t;
    const bool fallback = x_fallback && S->status == PDHGC_STATUS_CORNER_LIMIT;
    for (int j = threadIdx.x; j < d.n; j += BT) {
      const double xv = out ? d.hxp[j] : (avg ? w.sum_x[j] * inv_t : w.x[j]);
      xo[j] = fallback ? x_fallback[j] : fmin(fmax(xv, md.lhat[j]), md.uhat[j]);
    }
    if (yo)
      for (int i = threadIdx.x; i < d.m; i += BT) yo[i] = out ? d.hyp[i] : (avg ? w.sum_y[i] * inv_t : w.y[i]);
    __syncthreads();
  }

  // KKT numbers and metrics of (x, y) on the original model (mirrors run_report)
  __device__ void report(const double* x, const double* y, BatchReport* out) {
    const DevModel md = model(false);
    double pr[7];
    for (int i = 0; i < 7; ++i) pr[i] = 0.0;
    passA(matA(1), ReportRowsOp{x, y, md, 1e-6}, pr);
    cta_fold<BT>(pr, 7, ReportRowsOp::kMaxMask, q, red);
    double pc[8];
    for (int i = 0; i < 8; ++i) pc[i] = 0.0;
    passT(matT(1), ReportColsOp{y, x, d.l, d.u, md, 1e-6}, pc);
    cta_fold<BT>(pc, 8, ReportColsOp::kMaxMask, q + 7, red);
    if (threadIdx.x == 0) {
      BatchReport r;
      r.status = S->status;
      r.chosen = S->chosen;
      r.iters = S->k;
      r.restarts = S->restarts;
      r.rP2 = sqrt(q[1]);
      r.rPinf = q[2];
      r.rD2 = sqrt(q[8]);
      r.rDinf = q[9];
      r.pobj = q[10];
      r.dobj = q[3] + q[11];
      r.p = q[4] + q[12];
      r.dd = q[5] + q[13];
      r.cand = q[6] + q[14];
      r.omega = S->omega;
      r.eta = S->eta;
      r.sigma_max = S->sigma_max;
      r.seconds = (double)(global_ns() - S->t0_ns) * 1e-9;
      *out = r;
    }
    __syncthreads();
  }

  // the host watches the reports while the kernel runs and starts a handed-off
  // LP on the single-LP path as soon as its status shows: every earlier write
  // of the CTA is made visible before the status is
  __device__ bool handed_off(BatchReport* out) {
    if (S->status != kStatusHandoff) return false;
    if (threadIdx.x == 0) {
      BatchReport r{};
      r.status = kStatusHandoff;
      r.iters = S->k;
      __threadfence_system();
      *out = r;
    }
    __syncthreads();
    return true;
  }

  // returns false when the LP was handed to the single-LP path
  __device__ bool phase1(BatchReport* out) {
    setup();
    init_phase(0, nullptr, S->nc_hat, d.c_norm);
    if (bp.algorithm == PDHGC_ALG_HALPERN) loop_h(false);
    else loop(false);
    if (handed_off(out)) return false;
    finalize(d.x1, d.y1, nullptr, false);
    report(d.x1, d.y1, out);
    return true;
  }

  // Algorithm 1 (mirrors pdhgc_corner_phase)
  __device__ void corner(BatchReport* out) {
    if (threadIdx.x == 0) {
      S->eta = d.keep[0];
      S->sigma_max = d.keep[1];
      S->nb_hat = d.keep[2];
      S->nc_hat = d.keep[3];
    }
    __syncthreads();
    double pc[2] = {0.0, 0.0};
    passT(matT(1),
                 CornerColsOp{d.y1, d.x1, d.col_perm, model(false), d.lhat_c, d.uhat_c, d.chat_c, bp.eps_abs,
                              bp.obj_scale, bp.obj_seed},
                 pc);
    cta_fold<BT>(pc, 2, 0u, q, red);
    const double cc2 = q[0], cu2 = q[1];
    if (bp.row_rule == 1) {  // the option: A_hat x1 for the row slacks
      if (threadIdx.x == 0) S->pi_zero = 0;
      fill(d.pi_u, d.m, 0.0);
      __syncthreads();
      double pu[1] = {0.0};
      passA(matA(1), SpmvOp<false>{S, d.x1, d.pi_u}, pu);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < d.m; i += BT) {
      const double yu = fabs(d.Dr[i] * d.y1[i]);
      bool to_eq = d.ge[i] && yu > bp.eps_abs;
      if (to_eq && bp.row_rule == 1) to_eq = d.pi_u[i] / d.Dr[i] - d.b_int[i] <= yu;
      d.ge_c[i] = (d.ge[i] && !to_eq) ? 1 : 0;
    }
    if (kF32)
      for (int j = threadIdx.x; j < d.n; j += BT) {
        d.chat_c32[j] = (float)d.chat_c[j];
        d.lhat_c32[j] = (float)d.lhat_c[j];
        d.uhat_c32[j] = (float)d.uhat_c[j];
      }
    __syncthreads();
    init_phase(1, d.x1, sqrt(cc2), sqrt(cu2));
    if (bp.algorithm == PDHGC_ALG_HALPERN) loop_h(true);
    else loop(true);
    if (handed_off(out)) return;
    finalize(d.xc, nullptr, d.x1, true);
    report(d.xc, d.y1, out);
  }
};

// resident CTAs per SM the register allocation of k_batch must allow (0: the
// compiler's choice under the thread count alone).  1: the compiler may give
// a thread 65536 / BT registers; with the thread count alone it held the
// 1024-thread kernel to 32 registers and spilled 34 KB of state, and the
// batch_512 step took 13.5 s against 9.2 s with one CTA per SM and 64
// registers.
#ifndef PDHGC_BATCH_MIN_BLOCKS
#define PDHGC_BATCH_MIN_BLOCKS 1
#endif
#if PDHGC_BATCH_MIN_BLOCKS > 0
#define PDHGC_BATCH_BOUNDS(bt) __launch_bounds__(bt, PDHGC_BATCH_MIN_BLOCKS)
#else
#define PDHGC_BATCH_BOUNDS(bt) __launch_bounds__(bt)
#endif

template <class VT, int BT>
__global__ void PDHGC_BATCH_BOUNDS(BT) k_batch(const LpDesc* __restrict__ descs, const int* __restrict__ order,
                                              int count, int* queue, BatchParams bp, int phase,
                                              BatchReport* reps, BatchReport* reps2) {
  extern __shared__ __align__(16) unsigned char s_vec[];
  __shared__ Scalars S;
  __shared__ double red[32 * (BT / 32)];
  __shared__ double q[32];
  __shared__ int job;
  while (true) {
    if (threadIdx.x == 0) {
      job = atomicAdd(&queue[0], 1);
      if (job < count) atomicAdd(&queue[1], 1);
    }
    __syncthreads();
    const int jj = job;
    __syncthreads();
    if (jj >= count) break;
    const int lp = order[jj];
    const LpDesc& d = descs[lp];
    VT* sy = d.smem ? reinterpret_cast<VT*>(s_vec) : (std::is_same<VT, float>::value ? (VT*)d.y32 : (VT*)d.y);
    VT* sxb = d.smem ? reinterpret_cast<VT*>(s_vec) + d.m
                     : (std::is_same<VT, float>::value ? (VT*)d.xbar32 : (VT*)d.xbar);
    LpSolver<VT, BT> sol{d, bp, &S, red, q, sy, sxb, queue, count};
    if (phase == 0) {
      sol.phase1(&reps[lp]);
    } else if (phase == 1) {
      sol.corner(&reps[lp]);
    } else {  // 2: phase 1, then at once Algorithm 1 on the same LP (no batch-wide barrier between)
      if (sol.phase1(&reps[lp])) {
        sol.corner(&reps2[lp]);
      } else if (threadIdx.x == 0) {
        BatchReport r{};
        r.status = kStatusHandoff;
        reps2[lp] = r;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicSub(&queue[1], 1);
  }
}

template <class VT, int BT>
cudaError_t batch_kernel_prepare(size_t smem, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_batch<VT, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<VT, BT>, BT, smem);
}

template <class VT, int BT>
cudaError_t batch_kernel_launch(int grid, size_t smem, cudaStream_t st, const LpDesc* descs, const int* order,
                                int count, int* queue, const BatchParams& bp, int phase, BatchReport* reps,
                                BatchReport* reps2) {
  k_batch<VT, BT><<<grid, BT, smem, st>>>(descs, order, count, queue, bp, phase, reps, reps2);
  return cudaGetLastError();
}

}  // namespace pdhgc
