// C-ABI of the PDHG + corner-push library (include/pdhgc.h): handle,
// device memory, setup kernels, the graph-driven restarted PDHG loop in its
// two forms (averaged, and the reflected restarted Halpern loop of cuPDLP+
// that Section 4.1 names), Algorithm 1 with its corner primal-weight rule,
// reports and accessors; the phase-1 restart history, features, labels and
// held corner phase of the learned guidance; checkpoint/restore; the
// random-gather probe.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/pdhgc.h"
#include "host_prep.h"
#include "kernels.cuh"
#include "guide.h"
#include "kkt_eval.h"

using namespace pdhgc;

namespace {
thread_local std::string g_detail;
}  // namespace

namespace pdhgc {
int set_error_detail(int code, const std::string& d) {
  g_detail = d;
  return code;
}
}  // namespace pdhgc

namespace {

int set_err(int code, const std::string& d) { return set_error_detail(code, d); }

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return set_err(e_ == cudaErrorMemoryAllocation ? PDHGC_ERR_OOM : PDHGC_ERR_CUDA,    \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    }                                                                                     \
  } while (0)

#define CKL()                                                                             \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      return set_err(PDHGC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// ---- report as computed on the device ------------------------------------
struct DevReport {
  double rP2, rD2, rPinf, rDinf, pobj, dobj, gap, rel_p, rel_d, rel_gap, rel_kkt;
  double p, d, cand;
};

// ---- small kernels ---------------------------------------------------------

__global__ void k_fill(double* v, int n, double a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = a;
}

__global__ void k_mul_inplace(double* v, const double* f, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = v[i] * f[i];
}

// A_hat values: (D_r a) D_c for A, the same product for A'
__global__ void k_scale_values(const int* __restrict__ row_ptr, const int* __restrict__ col,
                               const double* __restrict__ val, double* __restrict__ out, int rows,
                               const double* __restrict__ Dr, const double* __restrict__ Dc,
                               int transposed) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows) return;
  for (int e = row_ptr[warp] + lane; e < row_ptr[warp + 1]; e += 32) {
    const int c = col[e];
    out[e] = transposed ? (Dr[c] * val[e]) * Dc[warp] : (Dr[warp] * val[e]) * Dc[c];
  }
}

// SELL-32 copy of a CSR array: dst[k] = src[map[k]], 0 on padding slots
template <class T>
__global__ void k_sell_fill(const int* __restrict__ map, const T* __restrict__ src, T* __restrict__ dst, int nslots) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nslots) {
    const int e = map[k];
    dst[k] = e >= 0 ? src[e] : T(0);
  }
}

// b_hat = D_r b_int; c_hat = D_c c; l_hat = l / D_c; u_hat = u / D_c
__global__ void k_scale_vectors(int m, int n, const double* Dr, const double* Dc, const double* b_int,
                                const double* c, const double* l, const double* u, double* bhat,
                                double* chat, double* lhat, double* uhat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) bhat[i] = Dr[i] * b_int[i];
  if (i < n) {
    chat[i] = Dc[i] * c[i];
    lhat[i] = l[i] / Dc[i];
    uhat[i] = u[i] / Dc[i];
  }
}

// one CTA: out[0] = sum v^2 (fixed order)
__global__ void k_norm2(const double* __restrict__ v, int n, double* out) {
  __shared__ double s_tmp[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += v[i] * v[i];
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = s_tmp[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
    out[0] = t;
  }
}

// power iteration: nw = ||w|| from partials; flag A_hat = 0
__global__ void k_pi_norm(Scalars* S, const double* partials, int ntiles, double* nw_out) {
  __shared__ double s_tmp[32];
  if (S->pi_zero) return;
  const double s = block_fold(partials, ntiles, false, s_tmp);
  if (threadIdx.x == 0) {
    const double nw = sqrt(s);
    nw_out[0] = nw;
    if (nw == 0.0) S->pi_zero = 1;
  }
}

__global__ void k_pi_scale(const Scalars* S, const double* w, const double* nw, double* v, int n) {
  if (S->pi_zero) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = w[i] / nw[0];
}

// sigma_max, eta, initial primal weight
__global__ void k_pi_final(Scalars* S, const double* partials, int ntiles, double eta_factor,
                           const double* nb2, const double* nc2) {
  __shared__ double s_tmp[32];
  double s = 0.0;
  if (!S->pi_zero) s = block_fold(partials, ntiles, false, s_tmp);
  if (threadIdx.x == 0) {
    const double smax = S->pi_zero ? 0.0 : sqrt(s);
    S->sigma_max = smax;
    S->eta = smax > 0.0 ? eta_factor / smax : 1.0;
    S->nb_hat = sqrt(nb2[0]);
    S->nc_hat = sqrt(nc2[0]);
  }
}

// start of a phase: x (from x_start, or proj(0)), y = 0, sums = 0, restart point
// FP32 copies of the iterates (FP32-bulk precision only; all null otherwise)
struct Iter32 {
  float* x;
  float* xbar;
  float* y;
  float* xlo;  // low parts of the float-float iterates
  float* ylo;
  float2* sx;  // float-float running sums
  float2* sy;
  float2* xa;  // Halpern loop: float-float anchors
  float2* ya;
  float* gy;   // Halpern loop: fl(y - y_0), gathered by the primal pass (xbar holds fl(x_bar - x_0))
  float2* q;   // Halpern loop: c_hat - A_hat' y_0 and b_hat - A_hat x_0 at the anchor
  float2* r0;
};

__global__ void k_init_iterates(int n, int m, DevModel md, DevIter w, const double* x_start, Iter32 w32,
                                const double* y_start = nullptr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double x0 = x_start ? x_start[i] : fmin(fmax(0.0, md.lhat[i]), md.uhat[i]);
    w.x[i] = x0;
    w.xbar[i] = x0;
    w.x_r[i] = x0;
    w.sum_x[i] = 0.0;
    if (w32.x) {
      const float h = (float)x0;
      w32.x[i] = h;
      w32.xlo[i] = (float)(x0 - (double)h);
      w32.xbar[i] = h;
      w32.sx[i] = make_float2(0.f, 0.f);
      w32.xa[i] = make_float2(h, w32.xlo[i]);
    }
  }
  if (i < m) {
    const double y0 = y_start ? y_start[i] : 0.0;
    w.y[i] = y0;
    w.y_r[i] = y0;
    w.sum_y[i] = 0.0;
    if (w32.y) {
      const float h = (float)y0, lo = (float)(y0 - (double)h);
      w32.y[i] = h;
      w32.ylo[i] = lo;
      w32.sy[i] = make_float2(0.f, 0.f);
      w32.ya[i] = make_float2(h, lo);
      w32.gy[i] = 0.0f;  // y = y_0
    }
  }
}

// FP32 bulk: FP64 copies of the current iterates for the FP64 evaluation; x is
// clamped to the FP64 bounds (an FP32-rounded bound may lie an ulp outside)
__global__ void k_to64(const Scalars* S, int n, int m, const float* __restrict__ x32, const float* __restrict__ y32,
                       const float* __restrict__ xlo, const float* __restrict__ ylo, const float2* __restrict__ sx,
                       const float2* __restrict__ sy, const double* __restrict__ lhat,
                       const double* __restrict__ uhat, double* __restrict__ x, double* __restrict__ y,
                       double* __restrict__ sum_x, double* __restrict__ sum_y) {
  if (S->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    x[i] = fmin(fmax((double)x32[i] + (double)xlo[i], lhat[i]), uhat[i]);
    sum_x[i] = (double)sx[i].x + (double)sx[i].y;
  }
  if (i < m) {
    y[i] = (double)y32[i] + (double)ylo[i];
    sum_y[i] = (double)sy[i].x + (double)sy[i].y;
  }
}

// FP64 -> FP32 copy
__global__ void k_to32(const double* __restrict__ a, float* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

struct PhaseInit {
  double eps_rel, beta_suff, beta_nec, beta_art, theta, time_limit_s, nb, nc;
  long long max_iters, min_iters;
  int check_period, phase, stop_rule;
  int use_cc2;  // corner: primal weight from ||c_hat'|| (cc2[0]) and ||c'|| (cc2[1])
  int use_bb2;  // dual corner: primal weight from ||b_hat'|| (cc2[2])
  int algorithm;  // PDHGC_ALG_*
  double rho, pid_kp, pid_ki, pid_kd;  // Halpern loop
  double omega0;  // > 0: the starting primal weight (corner omega_rule 1); else from ||c_hat|| / ||b_hat||
};

__global__ void k_init_scalars(Scalars* S, PhaseInit pi, const double* cc2) {
  if (threadIdx.x != 0) return;
  S->eps_rel = pi.eps_rel;
  S->beta_suff = pi.beta_suff;
  S->beta_nec = pi.beta_nec;
  S->beta_art = pi.beta_art;
  S->theta = pi.theta;
  S->time_limit_s = pi.time_limit_s;
  S->nb = pi.nb;
  S->nc = pi.use_cc2 ? sqrt(cc2[1]) : pi.nc;
  const double nch = pi.use_cc2 ? sqrt(cc2[0]) : S->nc_hat;
  const double nbh = pi.use_bb2 ? sqrt(cc2[2]) : S->nb_hat;
  S->max_iters = pi.max_iters;
  S->min_iters = pi.min_iters;
  S->check_period = pi.check_period;
  S->phase = pi.phase;
  S->stop_rule = pi.stop_rule;
  S->omega = pi.omega0 > 0.0 ? pi.omega0 : ((nch > 1e-10 && nbh > 1e-10) ? nch / nbh : 1.0);
  S->tau = S->eta / S->omega;
  S->sigma = S->eta * S->omega;
  S->k = 0;
  S->t = 0;
  S->restarts = 0;
  S->chunks = 0;
  S->max_chunks = pi.max_iters / pi.check_period + 2;
  S->done = 0;
  S->status = PDHGC_STATUS_NONE;
  S->chosen = 0;
  S->restart_to = 0;
  S->inv_t = 0.0;
  S->at_check = 0;
  S->at_limit = 0;
  S->error = 0;
  S->kkt_prev = INFINITY;
  S->algorithm = pi.algorithm;
  S->rho = pi.rho;
  S->pid_kp = pi.pid_kp;
  S->pid_ki = pi.pid_ki;
  S->pid_kd = pi.pid_kd;
  S->fpr = S->fpr0 = 0.0;
  S->fpr_prev = INFINITY;
  S->pid_int = 0.0;
  S->pid_eprev = 0.0;
  S->t0_ns = global_ns();
}

// Halpern loop: the anchoring weights (t + i + 1) / (t + i + 2) of the
// steps i < P of the next chunk, t = steps since the anchor, and their
// complements 1 / (t + i + 2) in FP32 (hs, FP32 bulk)
__global__ void k_halpern_weights(const Scalars* S, double* hw, float* hs, int P) {
  if (S->done) return;
  const long long t = S->t;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    hw[i] = (double)(t + i + 1) / (double)(t + i + 2);
    hs[i] = (float)(1.0 / (double)(t + i + 2));
  }
}

// FP32-bulk Halpern loop, end of a phase: FP64 copies of the float-float
// iterate z for the accessors
__global__ void k_h32_to64(const Scalars* S, int n, int m, const float* __restrict__ x32,
                           const float* __restrict__ xlo, const float* __restrict__ y32,
                           const float* __restrict__ ylo, double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (double)x32[i] + (double)xlo[i];
  if (i < m) y[i] = (double)y32[i] + (double)ylo[i];
}

// after a chunk of iterations: iteration counters and 1/t for the averages
__global__ void k_pre_check(Scalars* S) {
  if (threadIdx.x != 0 || S->done) return;
  long long run = S->max_iters - S->k;
  if (run > S->check_period) run = S->check_period;
  if (run < 0) run = 0;
  S->k += run;
  S->t += run;
  S->inv_t = S->t > 0 ? 1.0 / (double)S->t : 0.0;
  S->at_check = (S->k % S->check_period) == 0;
  S->at_limit = S->k >= S->max_iters;
  S->chunks += 1;
  if (S->chunks > S->max_chunks) S->at_limit = 1;
}

// The fold of block_fold (256 threads) for several quantities at once: a CTA
// of kFoldGroups x 256 threads, where group g folds quantities g, g + 4, ...
// with exactly block_fold's arithmetic (thread t of the group sums entries
// t, t + 256, ... in order, a shuffle tree per warp, then the 8 warp totals
// in warp order), so each result is bit for bit block_fold's.  part(qi, &p,
// &n) names quantity qi's partials; bit qi of max_mask makes it a maximum.
constexpr int kFoldGroups = 4;
constexpr int kFoldThreads = 256 * kFoldGroups;
template <class Parts>
__device__ inline void group_fold(const Parts& part, int nq, unsigned max_mask, double* q_out,
                                  double (*s_grp)[8]) {
  const int g = threadIdx.x >> 8, t = threadIdx.x & 255;
  const int lane = t & 31, w = t >> 5;
  for (int r = 0; r * kFoldGroups < nq; ++r) {
    const int qi = r * kFoldGroups + g;
    const bool is_max = qi < nq && ((max_mask >> qi) & 1u);
    double v = 0.0;
    if (qi < nq) {
      const double* p = nullptr;
      int n = 0;
      part(qi, p, n);
      for (int k = t; k < n; k += 256) v = is_max ? fmax(v, p[k]) : v + p[k];
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, v, off);
      v = is_max ? fmax(v, o) : v + o;
    }
    __syncthreads();
    if (lane == 0) s_grp[g][w] = v;
    __syncthreads();
    if (qi < nq && t == 0) {
      double tot = s_grp[g][0];
      for (int w2 = 1; w2 < 8; ++w2) tot = is_max ? fmax(tot, s_grp[g][w2]) : tot + s_grp[g][w2];
      q_out[qi] = tot;
    }
  }
  __syncthreads();
}

// Fold the KKT partials, then: termination (Section 2 test, or the Section
// 3.1 rule in the corner phase), limits, and the adaptive restart with the
// primal-weight update.  mode 0: initial restart point only.
__global__ void k_decide(Scalars* S, const double* __restrict__ pA, int ntA, const double* __restrict__ pT,
                         int ntT, int mode, cudaGraphConditionalHandle h, int use_handle) {
  __shared__ double s_grp[kFoldGroups][8];
  __shared__ double q[22];
  if (S->done) {
    if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(h, 0u);
    return;
  }
  // rows: quantities 0..9 of pA (2 and 7 maxima); columns: 10..21 of pT (2 and 8)
  auto parts = [&](int qi, const double*& p, int& n) {
    if (qi < 10) {
      p = pA + (size_t)qi * ntA;
      n = ntA;
    } else {
      p = pT + (size_t)(qi - 10) * ntT;
      n = ntT;
    }
  };
  group_fold(parts, 22, (1u << 2) | (1u << 7) | (1u << 12) | (1u << 18), q, s_grp);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    decide_step(S, q, 0);
    return;
  }
  decide_step(S, q, 1);
  S->t1_ns = global_ns();
  if (use_handle) cudaGraphSetConditional(h, S->done ? 0u : 1u);
}

// Fold the 7 + 7 Halpern check quantities, then decide_halpern.
__global__ void k_decide_h(Scalars* S, const double* __restrict__ pA, int ntA, const double* __restrict__ pT,
                           int ntT, int mode, cudaGraphConditionalHandle h, int use_handle) {
  __shared__ double s_grp[kFoldGroups][8];
  __shared__ double q[14];
  if (S->done) {
    if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(h, 0u);
    return;
  }
  // rows: quantities 0..6 of pA; columns: 7..13 of pT (2 and 9 maxima)
  auto parts = [&](int qi, const double*& p, int& n) {
    if (qi < 7) {
      p = pA + (size_t)qi * ntA;
      n = ntA;
    } else {
      p = pT + (size_t)(qi - 7) * ntT;
      n = ntT;
    }
  };
  group_fold(parts, 14, (1u << 2) | (1u << 9), q, s_grp);
  if (threadIdx.x != 0) return;
  decide_halpern(S, q, mode);
  if (mode != 0 && use_handle) cudaGraphSetConditional(h, S->done ? 0u : 1u);
}

// restart history of phase 1 (guidance features): slot e mod 8 holds
// (x_hat, z_hat) of restart point e, the start point being e = 0
struct RingRec {
  float* rx;
  float* rz;
  const double* z_cur;
  const double* z_avg;
};

// restart: jump to the candidate, new restart point, sums cleared.
// restart_to 3 (Halpern loop): the iterate and the anchor become T(z).
__global__ void k_restart_apply(const Scalars* S, int n, int m, DevIter w, Iter32 w32, RingRec rr, DevHalpern hz) {
  const int rt = S->restart_to;
  if (rt == 0 || S->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (rt == 3) {
    if (i < n) {
      const double xn = hz.xp[i];
      w.x[i] = xn;
      w.x_r[i] = xn;
      if (w32.x) {  // FP32 bulk: the float-float iterate and anchor
        const float h = (float)xn, lo = (float)(xn - (double)h);
        w32.x[i] = h;
        w32.xlo[i] = lo;
        w32.xa[i] = make_float2(h, lo);
      }
      if (rr.rx) {
        const size_t slot = (size_t)(S->restarts % 8) * (size_t)n;
        rr.rx[slot + i] = (float)xn;
        rr.rz[slot + i] = (float)rr.z_cur[i];
      }
    }
    if (i < m) {
      const double yn = hz.yp[i];
      w.y[i] = yn;
      w.y_r[i] = yn;
      if (w32.y) {
        const float h = (float)yn, lo = (float)(yn - (double)h);
        w32.y[i] = h;
        w32.ylo[i] = lo;
        w32.ya[i] = make_float2(h, lo);
        w32.gy[i] = 0.0f;  // y is the anchor now
      }
    }
    return;
  }
  const double inv_t = S->inv_t;
  if (i < n) {
    const double xn = rt == 2 ? w.sum_x[i] * inv_t : w.x[i];
    w.x[i] = xn;
    w.x_r[i] = xn;
    w.sum_x[i] = 0.0;
    if (w32.x) {
      w32.sx[i] = make_float2(0.f, 0.f);
      if (rt == 2) {
        const float h = (float)xn;
        w32.x[i] = h;
        w32.xlo[i] = (float)(xn - (double)h);
      }
    }
    if (rr.rx) {
      const size_t slot = (size_t)(S->restarts % 8) * (size_t)n;
      rr.rx[slot + i] = (float)xn;
      rr.rz[slot + i] = (float)(rt == 2 ? rr.z_avg[i] : rr.z_cur[i]);
    }
  }
  if (i < m) {
    const double yn = rt == 2 ? w.sum_y[i] * inv_t : w.y[i];
    w.y[i] = yn;
    w.y_r[i] = yn;
    w.sum_y[i] = 0.0;
    if (w32.y) {
      w32.sy[i] = make_float2(0.f, 0.f);
      if (rt == 2) {
        const float h = (float)yn;
        w32.y[i] = h;
        w32.ylo[i] = (float)(yn - (double)h);
      }
    }
  }
}

__global__ void k_ring_init(int n, const double* __restrict__ x, RingRec rr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    rr.rx[i] = (float)x[i];
    rr.rz[i] = (float)rr.z_cur[i];
  }
}

// end of a phase: the returned point (current, average or T(z); the phase-1 x on a
// corner limit)
// The returned x is clamped to the phase's box: an average of FP32-bulk
// iterates may lie an FP32 ulp outside it (a no-op for the FP64 iteration)
// (chosen 2, Halpern loop: the PDHG output T(z) of the last check)
__global__ void k_finalize(const Scalars* S, int n, int m, DevIter w, double* xo, double* yo,
                           const double* x_fallback, const double* __restrict__ lhat,
                           const double* __restrict__ uhat, DevHalpern hz, const double* y_fallback = nullptr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool out = S->chosen == 2;
  const bool avg = S->chosen == 1 && S->t > 0;
  const double inv_t = S->inv_t;
  const bool fallback = x_fallback && S->status == PDHGC_STATUS_CORNER_LIMIT;
  if (i < n) {
    const double xv = out ? hz.xp[i] : (avg ? w.sum_x[i] * inv_t : w.x[i]);
    xo[i] = fallback ? x_fallback[i] : fmin(fmax(xv, lhat[i]), uhat[i]);
  }
  if (yo && i < m) {
    const bool yfb = y_fallback && S->status == PDHGC_STATUS_CORNER_LIMIT;
    yo[i] = yfb ? y_fallback[i] : (out ? hz.yp[i] : (avg ? w.sum_y[i] * inv_t : w.y[i]));
  }
}

// Section 3: a '>' row whose dual is non-trivial becomes '='.  ax (optional,
// the row_rule = 1 option): A_hat x1; such a row then stays '>' unless it also
// looks active at x1, its slack (A_hat x1)_i / D_r,i - b_i no larger than |y_i|
__global__ void k_corner_rows(int m, const int8_t* ge, const double* Dr, const double* y1, double eps_abs,
                              const double* ax, const double* b_int, int8_t* ge_c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double yu = fabs(Dr[i] * y1[i]);
  bool to_eq = ge[i] && yu > eps_abs;
  if (to_eq && ax) to_eq = ax[i] / Dr[i] - b_int[i] <= yu;
  ge_c[i] = (ge[i] && !to_eq) ? 1 : 0;
}

__global__ void k_report_final(const double* __restrict__ pR, int ntA, const double* __restrict__ pC, int ntT,
                               double nb, double nc, DevReport* out) {
  __shared__ double s_tmp[32];
  __shared__ double q[15];
  for (int qi = 0; qi < 7; ++qi) {
    const double v = block_fold(pR + (size_t)qi * ntA, ntA, qi == 2, s_tmp);
    if (threadIdx.x == 0) q[qi] = v;
    __syncthreads();
  }
  for (int qi = 0; qi < 8; ++qi) {
    const double v = block_fold(pC + (size_t)qi * ntT, ntT, qi == 2, s_tmp);
    if (threadIdx.x == 0) q[7 + qi] = v;
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  DevReport r;
  r.rP2 = sqrt(q[1]);
  r.rPinf = q[2];
  r.rD2 = sqrt(q[8]);
  r.rDinf = q[9];
  r.pobj = q[10];
  r.dobj = q[3] + q[11];
  r.gap = r.pobj - r.dobj;
  r.rel_p = r.rP2 / (1.0 + nb);
  r.rel_d = r.rD2 / (1.0 + nc);
  r.rel_gap = fabs(r.gap) / (1.0 + fabs(r.pobj) + fabs(r.dobj));
  r.rel_kkt = fmax(r.rel_p, fmax(r.rel_d, r.rel_gap));
  r.p = q[4] + q[12];
  r.d = q[5] + q[13];
  r.cand = q[6] + q[14];
  *out = r;
}

// reduced costs of the original model, z = proj(c_hat - A_hat' y) / D_c
struct ZOp {
  using Acc = SumD<1>;
  static constexpr int NQ = 0;
  static constexpr unsigned kMaxMask = 0;
  const double* __restrict__ y;
  DevModel md;
  double* __restrict__ z;
  __device__ bool skip() const { return false; }
  __device__ double row_ctx(int) const { return 0.0; }
  static constexpr int NG = 1;
  using VT = double;
  using GT = double;
  __device__ const double* gsrc(int) const { return y; }
  __device__ void accum(Acc& a, double, double v, const GV<double, 1>& g) const { a.v[0] = fma(v, g.v[0], a.v[0]); }
  __device__ void epilogue(int j, const Acc& a, double*) const {
    z[j] = proj_dual(md.chat[j] - a.v[0], md.lhat[j], md.uhat[j]) / md.Dc[j];
  }
};

// out_user[perm[i]] = a[i] * f1[i] * f2[i] (f1, f2 optional)
__global__ void k_unpermute(int len, const int* perm, const double* a, const double* f1, const double* f2,
                            double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double v = a[i];
  if (f1) v = f1[i] * v;
  if (f2) v = f2[i] * v;
  out[perm[i]] = v;
}

// random-gather ceiling: `count` loads of v[h(i)] with h a multiplicative
// hash onto [0, n_vec), kGatherProbeBatch independent loads in flight per
// thread; the sum is kept live through `sink`.  A launch makes
// kGatherProbeScale times more loads than it is charged for, so that the
// launch latency and the grid's ramp and tail do not set the rate
constexpr int kGatherProbeBatch = 8;
constexpr int kGatherProbeScale = 16;
template <class T>
__global__ void k_gather_probe(const T* __restrict__ v, long long n_vec, long long count, double* sink) {
  const long long stride = (long long)gridDim.x * blockDim.x * kGatherProbeBatch;
  T acc = T(0);  // summed in the element type: no FP64 work for 4-byte loads
  for (long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kGatherProbeBatch; i0 < count;
       i0 += stride) {
    T g[kGatherProbeBatch];
#pragma unroll
    for (int u = 0; u < kGatherProbeBatch; ++u) {
      const unsigned long long h = (unsigned long long)(i0 + u + 1) * 0x9E3779B97F4A7C15ull;
      const long long idx = (long long)__umul64hi(h, (unsigned long long)n_vec);
      g[u] = i0 + u < count ? __ldg(v + idx) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kGatherProbeBatch; ++u) acc += g[u];
  }
  if (acc == T(1.0e30)) *sink = (double)acc;
}

__global__ void k_uniform(unsigned long long seed, long long n, double scale, double* out) {
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = scale * splitmix_uniform(seed, (unsigned long long)j);
}

// folds two partial rows (q = 0, 1) of `p` into out[0], out[1]
__global__ void k_fold2(const double* __restrict__ p, int nt, double* out) {
  __shared__ double s_tmp[32];
  const double a = block_fold(p, nt, false, s_tmp);
  __syncthreads();
  const double b = block_fold(p + nt, nt, false, s_tmp);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

__global__ void k_fill_scaled(double* v, int n, double a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = v[i] * a;
}

}  // namespace

// ---------------------------------------------------------------------------
// The handle
// ---------------------------------------------------------------------------
struct pdhgc_lp {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<void*> allocs;
  int64_t launches = 0;

  // matrix (internal numbering)
  // one matrix (A or A') on the device: CSR plus its SELL-32 copy
  struct Mat {
    int rows = 0, cta_rows = 0, long_rows = 0, nslices = 0, nslots = 0;
    int nb_cta = 0, nb_warp = 0, nb_sell = 0;
    int *rp = nullptr, *col = nullptr, *slice_ptr = nullptr, *slice_w = nullptr, *scol = nullptr, *smap = nullptr;
    SellBlock* sblocks = nullptr;
    double *val = nullptr, *hat = nullptr, *sval = nullptr, *shat = nullptr;  // original / scaled values
    float *hat32 = nullptr, *shat32 = nullptr;  // FP32 copies of the scaled values (FP32 bulk)
    int nblocks() const { return nb_cta + nb_warp + nb_sell; }
    SpmvMatT<float> view32() const {
      return SpmvMatT<float>{rp,     col,  hat32,     slice_ptr, slice_w, scol,    shat32,
                             sblocks, rows, cta_rows, long_rows, nslices, nb_cta, nb_warp, nb_sell};
    }
    SpmvMat view(bool scaled) const {
      return SpmvMat{rp,   col,      scaled ? hat : val, slice_ptr, slice_w, scol,   scaled ? shat : sval,
                     sblocks, rows, cta_rows, long_rows, nslices,  nb_cta,  nb_warp, nb_sell};
    }
  } A, T;
  int ntA = 0, ntT = 0;  // blocks of one pass over A / A' (partials per quantity)
  // the chunked primal pass over A' (ChunkPlan), per element size of the
  // gathered vector: slot values are filled from the scaled matrix per solve
  struct Chunked {
    int nch = 0, chunk = 0, blocks = 0;
    int64_t nslots = 0;
    int* map = nullptr;
    uint16_t* idx = nullptr;
    ChunkUnit* units = nullptr;
    int *uc_off = nullptr, *uc_cnt = nullptr, *warp_units = nullptr;
    double* val64 = nullptr;
    float* val32 = nullptr;
  } ch64, ch32;
  int chunked_primal = 0;  // 1: the Halpern loop's primal pass runs chunked (pdhgc_set_primal_layout)
  bool chunk_ready = false;  // the chunk plans are built on the first request for the chunked layout
  int launch_mode = PDHGC_LAUNCH_GRAPH;  // pdhgc_set_launch_mode
  cudaEvent_t loop_done = nullptr;       // blocking-sync event the host waits on for a phase's loop
  // vectors (internal order)
  double *b_int = nullptr, *sign = nullptr, *c = nullptr, *l = nullptr, *u = nullptr;
  int8_t* ge = nullptr;
  double *Dr = nullptr, *Dc = nullptr, *bhat = nullptr, *chat = nullptr, *lhat = nullptr, *uhat = nullptr;
  double *rfac = nullptr, *cfac = nullptr;
  int *row_perm = nullptr, *col_perm = nullptr;
  // iterates
  DevIter it{};
  // Halpern-loop buffers, allocated on the first Halpern solve
  bool have_h = false;
  DevHalpern hz{};
  // FP32-bulk buffers, allocated on the first FP32 solve
  bool have32 = false;
  Iter32 it32{};
  float *chat32 = nullptr, *lhat32 = nullptr, *uhat32 = nullptr, *bhat32 = nullptr;
  float *chat_c32 = nullptr, *lhat_c32 = nullptr, *uhat_c32 = nullptr;
  double *x1 = nullptr, *y1 = nullptr, *xc = nullptr;
  // the dual corner push: its model (allocated on first use) and its y
  bool have_dual_bufs = false, have_dual = false;
  double *lhat_d = nullptr, *uhat_d = nullptr, *bhat_d = nullptr, *yd = nullptr;
  int8_t* ge_d = nullptr;
  float *lhat_d32 = nullptr, *uhat_d32 = nullptr, *bhat_d32 = nullptr;
  pdhgc_report repd{};
  double *chat_c = nullptr, *lhat_c = nullptr, *uhat_c = nullptr;
  int8_t* ge_c = nullptr;
  // phase-1 restart history for the guidance features: 8 slots x n
  float *ring_x = nullptr, *ring_z = nullptr;
  double *z_cur = nullptr, *z_avg = nullptr;  // z_hat of the last evaluated points
  // guidance buffers (allocated on first use)
  bool have_gbufs = false;
  uint16_t* gfeat = nullptr;  // n x 32 BF16 feature rows
  float* gprob = nullptr;
  uint8_t *ghold = nullptr, *gelig = nullptr, *glabel = nullptr, *gstage = nullptr;
  int8_t* gfixed = nullptr;
  double *gnorm = nullptr, *gxs = nullptr, *gpart = nullptr;
  long long* gcount = nullptr;
  int* gblk = nullptr;
  pdhgc_corner_params cp_last{};
  double *pi_v = nullptr, *pi_w = nullptr, *pi_u = nullptr, *tmp_n = nullptr, *tmp_m = nullptr;
  double *pA = nullptr, *pT = nullptr, *scratch = nullptr;
  int* err = nullptr;  // device error word set by a kernel whose bounded wait ran out
  Scalars* S = nullptr;
  DevReport* rep = nullptr;
  double b_norm = 0.0, c_norm = 0.0;
  bool have_phase1 = false, have_corner = false;
  pdhgc_report rep1{}, repc{};
  pdhgc_params params{};

  template <class T>
  int alloc(T** p, size_t count) {
    void* q = nullptr;
    const size_t bytes = (count > 0 ? count : 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess)
      return set_err(PDHGC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return PDHGC_OK;
  }
  ~pdhgc_lp() {
    for (void* q : allocs) cudaFree(q);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (loop_done) cudaEventDestroy(loop_done);
  }
};

namespace {

inline int grid_for(long long n, int block = 256) { return (int)((n + block - 1) / block); }

template <class Op>
int launch_tiles(pdhgc_lp* lp, bool transposed, bool scaled, const Op& op, double* partials, cudaStream_t st,
                 bool pdl = false) {
  const pdhgc_lp::Mat& M = transposed ? lp->T : lp->A;
  const int nb = M.nblocks();
  if (nb == 0) return PDHGC_OK;
  SpmvMatT<typename Op::VT> view;
  if constexpr (std::is_same<typename Op::VT, float>::value) {
    view = M.view32();
  } else {
    view = M.view(scaled);
  }
  if (pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, spmv<Op, true>, view, op, partials));
  } else {
    spmv<Op, false><<<nb, kBlock, 0, st>>>(view, op, partials);
  }
  lp->launches++;
  CKL();
  return PDHGC_OK;
}

// the primal pass over A' as the chunked kernel (ChunkPlan): one CTA per SM,
// the gathered vector staged in shared memory chunk by chunk
template <class Op>
int launch_chunked(pdhgc_lp* lp, const Op& op, cudaStream_t st, bool pdl) {
  using VT = typename Op::VT;
  using GT = typename Op::GT;
  const pdhgc_lp::Chunked& C = std::is_same<VT, float>::value ? lp->ch32 : lp->ch64;
  ChunkMatT<VT> M;
  if constexpr (std::is_same<VT, float>::value) {
    M.val = C.val32;
  } else {
    M.val = C.val64;
  }
  M.idx = C.idx;
  M.units = C.units;
  M.uc_off = C.uc_off;
  M.uc_cnt = C.uc_cnt;
  M.warp_units = C.warp_units;
  M.nch = C.nch;
  M.chunk = C.chunk;
  M.glen = lp->m;
  const size_t smem = (size_t)C.chunk * sizeof(GT);  // the attribute is set at lp_create
  if (pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C.blocks);
    cfg.blockDim = dim3(kChunkThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, spmv_chunked<Op, true>, M, op));
  } else {
    spmv_chunked<Op, false><<<C.blocks, kChunkThreads, smem, st>>>(M, op);
  }
  lp->launches++;
  CKL();
  return PDHGC_OK;
}

// the primal pass of the Halpern loop: chunked, or over the row segments
template <class Op>
int launch_primal(pdhgc_lp* lp, const Op& op, cudaStream_t st, bool pdl) {
  if (lp->chunked_primal) return launch_chunked(lp, op, st, pdl);
  return launch_tiles(lp, true, true, op, nullptr, st, pdl);
}

DevModel model_orig(const pdhgc_lp* lp) {
  return DevModel{lp->chat, lp->lhat, lp->uhat, lp->bhat, lp->Dr, lp->Dc, lp->ge};
}
DevModel32 model32_orig(const pdhgc_lp* lp) {
  return DevModel32{lp->chat32, lp->lhat32, lp->uhat32, lp->bhat32, lp->ge};
}
DevModel32 model32_corner(const pdhgc_lp* lp) {
  return DevModel32{lp->chat_c32, lp->lhat_c32, lp->uhat_c32, lp->bhat32, lp->ge_c};
}
DevModel model_corner(const pdhgc_lp* lp) {
  return DevModel{lp->chat_c, lp->lhat_c, lp->uhat_c, lp->bhat, lp->Dr, lp->Dc, lp->ge_c};
}

#define RET(x)                 \
  do {                         \
    int r_ = (x);              \
    if (r_ != PDHGC_OK) return r_; \
  } while (0)

int to32(pdhgc_lp* lp, const double* a, float* b, long long n, cudaStream_t st) {
  if (n <= 0) return PDHGC_OK;
  k_to32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  lp->launches++;
  CKL();
  return PDHGC_OK;
}

// FP32-bulk buffers (allocated once per handle, on the first FP32 solve)
int ensure_fp32(pdhgc_lp* lp) {
  if (lp->have32) return PDHGC_OK;
  const size_t n = lp->n, m = lp->m;
  for (pdhgc_lp::Mat* M : {&lp->A, &lp->T}) {
    RET(lp->alloc(&M->hat32, (size_t)lp->nnz + kPad));
    RET(lp->alloc(&M->shat32, (size_t)M->nslots + kPad));
  }
  RET(lp->alloc(&lp->it32.x, n));
  RET(lp->alloc(&lp->it32.xbar, n));
  RET(lp->alloc(&lp->it32.y, m));
  RET(lp->alloc(&lp->it32.xlo, n));
  RET(lp->alloc(&lp->it32.ylo, m));
  RET(lp->alloc(&lp->it32.sx, n));
  RET(lp->alloc(&lp->it32.sy, m));
  RET(lp->alloc(&lp->it32.xa, n));
  RET(lp->alloc(&lp->it32.ya, m));
  RET(lp->alloc(&lp->it32.gy, m));
  RET(lp->alloc(&lp->it32.q, n));
  RET(lp->alloc(&lp->it32.r0, m));
  RET(lp->alloc(&lp->chat32, n));
  RET(lp->alloc(&lp->lhat32, n));
  RET(lp->alloc(&lp->uhat32, n));
  RET(lp->alloc(&lp->bhat32, m));
  RET(lp->alloc(&lp->chat_c32, n));
  RET(lp->alloc(&lp->lhat_c32, n));
  RET(lp->alloc(&lp->uhat_c32, n));
  lp->have32 = true;
  return PDHGC_OK;
}

// FP32 copies of the scaled matrix and model (after setup_scaling)
int convert_fp32(pdhgc_lp* lp, cudaStream_t st) {
  for (pdhgc_lp::Mat* M : {&lp->A, &lp->T}) {
    RET(to32(lp, M->hat, M->hat32, lp->nnz, st));
    RET(to32(lp, M->shat, M->shat32, M->nslots, st));
  }
  RET(to32(lp, lp->chat, lp->chat32, lp->n, st));
  RET(to32(lp, lp->lhat, lp->lhat32, lp->n, st));
  RET(to32(lp, lp->uhat, lp->uhat32, lp->n, st));
  RET(to32(lp, lp->bhat, lp->bhat32, lp->m, st));
  if (lp->ch32.nslots > 0) {  // the chunked pass's FP32 slots
    k_sell_fill<<<grid_for(lp->ch32.nslots), 256, 0, st>>>(lp->ch32.map, lp->T.hat32, lp->ch32.val32,
                                                          (int)lp->ch32.nslots);
    lp->launches++;
    CKL();
  }
  return PDHGC_OK;
}

// a0: Ruiz + Pock-Chambolle scaling, scaled copies, power iteration
int setup_scaling(pdhgc_lp* lp, const pdhgc_params& p) {
  cudaStream_t st = lp->stream;
  const int m = lp->m, n = lp->n;
  k_fill<<<grid_for(m), 256, 0, st>>>(lp->Dr, m, 1.0);
  k_fill<<<grid_for(n), 256, 0, st>>>(lp->Dc, n, 1.0);
  lp->launches += 2;
  CKL();
  for (int pass = 0; pass < p.ruiz_iters; ++pass) {
    RET(launch_tiles(lp, false, false, ScaleMaxOp<false>{lp->Dr, lp->Dc, lp->rfac}, nullptr, st));
    RET(launch_tiles(lp, true, false, ScaleMaxOp<true>{lp->Dc, lp->Dr, lp->cfac}, nullptr, st));
    k_mul_inplace<<<grid_for(m), 256, 0, st>>>(lp->Dr, lp->rfac, m);
    k_mul_inplace<<<grid_for(n), 256, 0, st>>>(lp->Dc, lp->cfac, n);
    lp->launches += 2;
    CKL();
  }
  RET(launch_tiles(lp, false, false, ScaleSumOp<false>{lp->Dr, lp->Dc, lp->rfac}, nullptr, st));
  RET(launch_tiles(lp, true, false, ScaleSumOp<true>{lp->Dc, lp->Dr, lp->cfac}, nullptr, st));
  k_mul_inplace<<<grid_for(m), 256, 0, st>>>(lp->Dr, lp->rfac, m);
  k_mul_inplace<<<grid_for(n), 256, 0, st>>>(lp->Dc, lp->cfac, n);
  k_scale_values<<<grid_for((long long)m * 32), 256, 0, st>>>(lp->A.rp, lp->A.col, lp->A.val, lp->A.hat, m,
                                                              lp->Dr, lp->Dc, 0);
  k_scale_values<<<grid_for((long long)n * 32), 256, 0, st>>>(lp->T.rp, lp->T.col, lp->T.val, lp->T.hat, n,
                                                              lp->Dr, lp->Dc, 1);
  for (const pdhgc_lp::Mat* M : {&lp->A, &lp->T}) {
    if (M->nslots == 0) continue;  // no nonzeros in SELL rows
    k_sell_fill<<<grid_for(M->nslots), 256, 0, st>>>(M->smap, M->hat, M->shat, M->nslots);
    lp->launches++;
  }
  if (lp->ch64.nslots > 0) {  // the chunked pass's FP64 slots
    k_sell_fill<<<grid_for(lp->ch64.nslots), 256, 0, st>>>(lp->ch64.map, lp->T.hat, lp->ch64.val64,
                                                          (int)lp->ch64.nslots);
    lp->launches++;
  }
  k_scale_vectors<<<grid_for(m > n ? m : n), 256, 0, st>>>(m, n, lp->Dr, lp->Dc, lp->b_int, lp->c, lp->l,
                                                            lp->u, lp->bhat, lp->chat, lp->lhat, lp->uhat);
  k_norm2<<<1, 1024, 0, st>>>(lp->bhat, m, lp->scratch + 0);
  k_norm2<<<1, 1024, 0, st>>>(lp->chat, n, lp->scratch + 1);
  lp->launches += 7;
  CKL();
  // power iteration on A_hat' A_hat from v = 1/sqrt(n)
  CK(cudaMemsetAsync(&lp->S->pi_zero, 0, sizeof(int), st));
  k_fill<<<grid_for(n), 256, 0, st>>>(lp->pi_v, n, 1.0 / std::sqrt((double)n));
  lp->launches++;
  for (int k = 0; k < p.power_iters; ++k) {
    RET(launch_tiles(lp, false, true, SpmvOp<false>{lp->S, lp->pi_v, lp->pi_u}, nullptr, st));
    RET(launch_tiles(lp, true, true, SpmvOp<true>{lp->S, lp->pi_u, lp->pi_w}, lp->pT, st));
    k_pi_norm<<<1, 1024, 0, st>>>(lp->S, lp->pT, lp->ntT, lp->scratch + 2);
    k_pi_scale<<<grid_for(n), 256, 0, st>>>(lp->S, lp->pi_w, lp->scratch + 2, lp->pi_v, n);
    lp->launches += 2;
    CKL();
  }
  RET(launch_tiles(lp, false, true, SpmvOp<true>{lp->S, lp->pi_v, lp->pi_u}, lp->pA, st));
  k_pi_final<<<1, 1024, 0, st>>>(lp->S, lp->pA, lp->ntA, p.eta_factor, lp->scratch + 0, lp->scratch + 1);
  lp->launches++;
  CKL();
  return PDHGC_OK;
}

// the KKT evaluation of the current and average points (two matrix passes)
int launch_eval(pdhgc_lp* lp, const DevModel& md, cudaStream_t st, bool record_z) {
  const DevIter& w = lp->it;
  RET(launch_tiles(lp, false, true, EvalRowsOp{lp->S, w.x, w.sum_x, w.y, w.sum_y, w.y_r, md}, lp->pA, st));
  RET(launch_tiles(lp, true, true,
                   EvalColsOp{lp->S, w.y, w.sum_y, w.x, w.sum_x, w.x_r, md, record_z ? lp->z_cur : nullptr,
                              record_z ? lp->z_avg : nullptr},
                   lp->pT, st));
  return PDHGC_OK;
}

// the Halpern check: T(z) and z - T(z) of the last step against the anchor
int launch_eval_h(pdhgc_lp* lp, const DevModel& md, cudaStream_t st, bool record_z) {
  const DevIter& w = lp->it;
  RET(launch_tiles(lp, false, true, EvalRowsH{lp->S, lp->hz, w.y_r, md}, lp->pA, st));
  RET(launch_tiles(lp, true, true, EvalColsH{lp->S, lp->hz, w.x_r, md, record_z ? lp->z_cur : nullptr}, lp->pT,
                   st));
  return PDHGC_OK;
}

int ensure_halpern(pdhgc_lp* lp) {
  if (lp->have_h) return PDHGC_OK;
  RET(lp->alloc(&lp->hz.xp, (size_t)lp->n));
  RET(lp->alloc(&lp->hz.yp, (size_t)lp->m));
  RET(lp->alloc(&lp->hz.dx, (size_t)lp->n));
  RET(lp->alloc(&lp->hz.dy, (size_t)lp->m));
  RET(lp->alloc(&lp->hz.hw, (size_t)4096));
  RET(lp->alloc(&lp->hz.hs, (size_t)4096));
  lp->have_h = true;
  return PDHGC_OK;
}

// the FP32-bulk Halpern iterate of the handle (the gathered x_bar difference
// lives in it32.xbar)
DevH32 h32_of(const pdhgc_lp* lp) {
  const Iter32& w = lp->it32;
  return DevH32{w.x, w.xlo, w.y, w.ylo, w.xa, w.ya, w.xbar, w.gy, w.q, w.r0};
}

// q = c_hat - A_hat' y_0 and r0 = b_hat - A_hat x_0 at the current anchor
// (FP64 copies x_r, y_r); force = 0: only when the last decision restarted
int launch_anchor(pdhgc_lp* lp, const DevModel& md, int force, cudaStream_t st) {
  RET(launch_tiles(lp, true, true, AnchorColsOp{lp->S, force, lp->it.y_r, md.chat, lp->it32.q}, nullptr, st));
  RET(launch_tiles(lp, false, true, AnchorRowsOp{lp->S, force, lp->it.x_r, md.bhat, lp->it32.r0}, nullptr, st));
  return PDHGC_OK;
}

// Enqueues one loop body on `cs`: P iterations; pre-check; eval; decide;
// restart; weights.  fp32 selects the FP32-bulk iteration kernels; the
// evaluation and the decisions are FP64 in both.  use_handle: the decision
// kernel sets the graph's WHILE condition (`handle`) from S->done.
int enqueue_body(pdhgc_lp* lp, const DevModel& md, const DevModel32& md32, const PhaseInit& pi, bool fp32,
                 bool ring, const RingRec& rr, cudaStream_t cs, cudaGraphConditionalHandle handle, int use_handle) {
  const int n = lp->n, m = lp->m;
  const int gnm = grid_for(n > m ? n : m);
  const bool halpern = pi.algorithm == PDHGC_ALG_HALPERN;
  const DevHalpern hz = lp->hz;
  const Iter32 w32 = fp32 ? lp->it32 : Iter32{};
  const DevIter32 it32{lp->it32.x,  lp->it32.y,   lp->it32.xbar, lp->it32.sx, lp->it32.sy,
                       lp->it32.xlo, lp->it32.ylo, lp->it32.xa,   lp->it32.ya};
  int rc = PDHGC_OK;
  for (int i = 0; i < pi.check_period && rc == PDHGC_OK; ++i) {
    if (halpern && fp32) {
      const int last = pi.check_period - 1;
      rc = pi.rho == 1.0 ? launch_primal(lp, PrimalOpH32T<true>{lp->S, i, last, 0, md32, h32_of(lp), hz}, cs, true)
                         : launch_primal(lp, PrimalOpH32{lp->S, i, last, 0, md32, h32_of(lp), hz}, cs, true);
      if (rc == PDHGC_OK)
        rc = launch_tiles(lp, false, true, DualOpH32{lp->S, i, last, 0, md32, h32_of(lp), hz}, nullptr, cs, true);
    } else if (halpern && pi.rho == 1.0) {  // the default reflection: the reflected point is x_bar
      const int last = pi.check_period - 1;
      rc = launch_primal(lp, PrimalOpHT<true>{lp->S, i, last, 0, lp->it.y, md, lp->it, hz}, cs, true);
      if (rc == PDHGC_OK)
        rc = launch_tiles(lp, false, true, DualOpHT<true>{lp->S, i, last, 0, lp->it.xbar, md, lp->it, hz}, nullptr,
                          cs, true);
    } else if (halpern) {
      const int last = pi.check_period - 1;
      rc = launch_primal(lp, PrimalOpH{lp->S, i, last, 0, lp->it.y, md, lp->it, hz}, cs, true);
      if (rc == PDHGC_OK)
        rc = launch_tiles(lp, false, true, DualOpH{lp->S, i, last, 0, lp->it.xbar, md, lp->it, hz}, nullptr, cs,
                          true);
    } else if (fp32) {
      rc = launch_tiles(lp, true, true, PrimalOp32{lp->S, i, lp->it32.y, md32, it32}, nullptr, cs, true);
      if (rc == PDHGC_OK)
        rc = launch_tiles(lp, false, true, DualOp32{lp->S, i, lp->it32.xbar, md32, it32}, nullptr, cs, true);
    } else {
      rc = launch_tiles(lp, true, true, PrimalOp{lp->S, i, lp->it.y, md, lp->it}, nullptr, cs, true);
      if (rc == PDHGC_OK)
        rc = launch_tiles(lp, false, true, DualOp{lp->S, i, lp->it.xbar, md, lp->it}, nullptr, cs, true);
    }
  }
  if (rc == PDHGC_OK && fp32 && !halpern) {
    k_to64<<<gnm, 256, 0, cs>>>(lp->S, n, m, lp->it32.x, lp->it32.y, lp->it32.xlo, lp->it32.ylo, lp->it32.sx,
                                lp->it32.sy, md.lhat, md.uhat, lp->it.x, lp->it.y, lp->it.sum_x, lp->it.sum_y);
    lp->launches++;
  }
  if (rc == PDHGC_OK) {
    k_pre_check<<<1, 32, 0, cs>>>(lp->S);
    lp->launches++;
    rc = halpern ? launch_eval_h(lp, md, cs, ring) : launch_eval(lp, md, cs, ring);
  }
  if (rc == PDHGC_OK) {
    if (halpern)
      k_decide_h<<<1, kFoldThreads, 0, cs>>>(lp->S, lp->pA, lp->ntA, lp->pT, lp->ntT, 1, handle, use_handle);
    else
      k_decide<<<1, kFoldThreads, 0, cs>>>(lp->S, lp->pA, lp->ntA, lp->pT, lp->ntT, 1, handle, use_handle);
    k_restart_apply<<<gnm, 256, 0, cs>>>(lp->S, n, m, lp->it, w32, rr, hz);
    lp->launches += 2;
    if (halpern && fp32) rc = launch_anchor(lp, md, 0, cs);  // a restart moved the anchor
    if (halpern && rc == PDHGC_OK) {
      k_halpern_weights<<<1, 256, 0, cs>>>(lp->S, hz.hw, hz.hs, pi.check_period);
      lp->launches++;
    }
  }
  return rc;
}

// Runs the loop of a phase on the handle's stream until S->done.  Graph mode
// (the default) builds one graph whose conditional WHILE node repeats the
// body with no host round trip, and adds the kernels of the executed bodies
// to lp->launches once the graph has finished (*per_body_out per body; the
// caller multiplies by S->chunks).  Stream mode (pdhgc_set_launch_mode)
// enqueues each body as plain launches and reads S->done back after it, so
// that every kernel is a separate launch a profiler can see; the launches are
// counted as they are made (*per_body_out = 0).
int launch_loop(pdhgc_lp* lp, const DevModel& md, const DevModel32& md32, const PhaseInit& pi, bool fp32,
                bool ring, const RingRec& rr, int64_t* per_body_out) {
  if (lp->launch_mode == PDHGC_LAUNCH_STREAM) {
    *per_body_out = 0;
    for (;;) {
      RET(enqueue_body(lp, md, md32, pi, fp32, ring, rr, lp->stream, cudaGraphConditionalHandle{}, 0));
      int done = 0;
      CK(cudaMemcpyAsync(&done, &lp->S->done, sizeof(int), cudaMemcpyDeviceToHost, lp->stream));
      CK(cudaStreamSynchronize(lp->stream));
      if (done) break;
    }
    return PDHGC_OK;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  std::unique_ptr<CUgraph_st, void (*)(cudaGraph_t)> g_guard(graph, [](cudaGraph_t g) { cudaGraphDestroy(g); });
  cudaGraphConditionalHandle handle;
  CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs = lp->cap_stream;
  CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const int64_t before = lp->launches;
  const int rc = enqueue_body(lp, md, md32, pi, fp32, ring, rr, cs, handle, 1);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(cs, &captured);
  *per_body_out = lp->launches - before;
  lp->launches = before;  // counted per executed body by the caller
  if (rc != PDHGC_OK) return rc;
  if (ce != cudaSuccess) return set_err(PDHGC_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
  CK(cudaGraphInstantiate(&exec, graph, 0));
  std::unique_ptr<CUgraphExec_st, void (*)(cudaGraphExec_t)> e_guard(exec,
                                                                    [](cudaGraphExec_t e) { cudaGraphExecDestroy(e); });
  CK(cudaGraphLaunch(exec, lp->stream));
  // the loop runs for up to seconds: wait on an event with blocking sync, so
  // that the calling thread sleeps instead of spinning on a core (the batched
  // solver finishes several handed-off LPs at once, a host thread each)
  if (!lp->loop_done) CK(cudaEventCreateWithFlags(&lp->loop_done, cudaEventBlockingSync | cudaEventDisableTiming));
  CK(cudaEventRecord(lp->loop_done, lp->stream));
  CK(cudaEventSynchronize(lp->loop_done));  // the executable graph is destroyed on return
  return PDHGC_OK;
}

// Runs one phase: init, the device-driven loop graph, finalize.
int run_phase(pdhgc_lp* lp, const DevModel& md, const DevModel32& md32, const PhaseInit& pi,
              const double* x_start, const double* cc2, double* xo, double* yo, const double* x_fallback,
              const double* y_start = nullptr, const double* y_fallback = nullptr) {
  cudaStream_t st = lp->stream;
  const int n = lp->n, m = lp->m;
  const int gnm = grid_for(n > m ? n : m);
  const bool fp32 = lp->params.precision == PDHGC_FP32_BULK;
  const bool halpern = pi.algorithm == PDHGC_ALG_HALPERN;
  if (halpern) RET(ensure_halpern(lp));
  const DevHalpern hz = lp->hz;
  const Iter32 w32 = fp32 ? lp->it32 : Iter32{};
  const DevIter32 it32{lp->it32.x,  lp->it32.y,   lp->it32.xbar, lp->it32.sx, lp->it32.sy,
                       lp->it32.xlo, lp->it32.ylo, lp->it32.xa,   lp->it32.ya};
  k_init_iterates<<<gnm, 256, 0, st>>>(n, m, md, lp->it, x_start, w32, y_start);
  k_init_scalars<<<1, 32, 0, st>>>(lp->S, pi, cc2);
  lp->launches += 2;
  CKL();
  // phase 1 records its restart history (start point and restart points)
  const bool ring = pi.phase == 0;
  const RingRec rr = ring ? RingRec{lp->ring_x, lp->ring_z, lp->z_cur, lp->z_avg} : RingRec{};
  RET(launch_eval(lp, md, st, ring));
  k_decide<<<1, kFoldThreads, 0, st>>>(lp->S, lp->pA, lp->ntA, lp->pT, lp->ntT, 0, cudaGraphConditionalHandle{}, 0);
  lp->launches++;
  CKL();
  if (ring) {
    k_ring_init<<<grid_for(n), 256, 0, st>>>(n, lp->it.x, rr);
    lp->launches++;
    CKL();
  }
  if (halpern) {
    // the anchor's fixed-point residual: T of the start point (not an
    // iteration), its check quantities, and the first chunk's weights
    if (fp32) {
      RET(launch_anchor(lp, md, 1, st));
      RET(launch_primal(lp, PrimalOpH32{lp->S, 0, 0, 1, md32, h32_of(lp), hz}, st, false));
      RET(launch_tiles(lp, false, true, DualOpH32{lp->S, 0, 0, 1, md32, h32_of(lp), hz}, nullptr, st));
    } else {
      RET(launch_primal(lp, PrimalOpH{lp->S, 0, 0, 1, lp->it.y, md, lp->it, hz}, st, false));
      RET(launch_tiles(lp, false, true, DualOpH{lp->S, 0, 0, 1, lp->it.xbar, md, lp->it, hz}, nullptr, st));
    }
    RET(launch_eval_h(lp, md, st, false));
    k_decide_h<<<1, kFoldThreads, 0, st>>>(lp->S, lp->pA, lp->ntA, lp->pT, lp->ntT, 0, cudaGraphConditionalHandle{}, 0);
    k_halpern_weights<<<1, 256, 0, st>>>(lp->S, hz.hw, hz.hs, pi.check_period);
    lp->launches += 2;
    CKL();
  }
  int64_t per_body = 0;
  RET(launch_loop(lp, md, md32, pi, fp32, ring, rr, &per_body));
  long long chunks = 0;
  CK(cudaMemcpy(&chunks, &lp->S->chunks, sizeof(chunks), cudaMemcpyDeviceToHost));
  lp->launches += chunks * per_body;
  k_finalize<<<gnm, 256, 0, st>>>(lp->S, n, m, lp->it, xo, yo, x_fallback, md.lhat, md.uhat, hz, y_fallback);
  lp->launches++;
  if (fp32 && halpern) {
    k_h32_to64<<<gnm, 256, 0, st>>>(lp->S, n, m, lp->it32.x, lp->it32.xlo, lp->it32.y, lp->it32.ylo, lp->it.x,
                                    lp->it.y);
    lp->launches++;
  }
  CKL();
  CK(cudaStreamSynchronize(st));
  int derr = 0;
  CK(cudaMemcpy(&derr, lp->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr != 0) return set_err(PDHGC_ERR_DEVICE, "a bounded device wait ran out (error word " +
                                                      std::to_string(derr) + ")");
  return PDHGC_OK;
}

int run_report(pdhgc_lp* lp, const double* x, const double* y, pdhgc_report* out) {
  cudaStream_t st = lp->stream;
  DevModel md = model_orig(lp);
  RET(launch_tiles(lp, false, true, ReportRowsOp{x, y, md, 1e-6}, lp->pA, st));
  RET(launch_tiles(lp, true, true, ReportColsOp{y, x, lp->l, lp->u, md, 1e-6}, lp->pT, st));
  k_report_final<<<1, 256, 0, st>>>(lp->pA, lp->ntA, lp->pT, lp->ntT, lp->b_norm, lp->c_norm, lp->rep);
  lp->launches++;
  CKL();
  DevReport r;
  CK(cudaMemcpyAsync(&r, lp->rep, sizeof(r), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  out->rP2 = r.rP2;
  out->rD2 = r.rD2;
  out->rPinf = r.rPinf;
  out->rDinf = r.rDinf;
  out->pobj = r.pobj;
  out->dobj = r.dobj;
  out->gap = r.gap;
  out->rel_p = r.rel_p;
  out->rel_d = r.rel_d;
  out->rel_gap = r.rel_gap;
  out->rel_kkt = r.rel_kkt;
  const int64_t m = lp->m;
  out->off_bound_p = (int64_t)llround(r.p);
  out->zero_rc_d = (int64_t)llround(r.d);
  out->candidates = (int64_t)llround(r.cand);
  out->corner_measure = out->candidates > m ? out->candidates - m : 0;
  out->primal_push_est = out->off_bound_p > m ? out->off_bound_p - m : 0;
  out->dual_push_est = m > out->zero_rc_d ? m - out->zero_rc_d : 0;
  const int64_t thr = 2 * m > 100000 ? 2 * m : 100000;
  out->should_corner = out->candidates >= thr ? 1 : 0;
  return PDHGC_OK;
}

int fill_phase_report(pdhgc_lp* lp, pdhgc_report* r) {
  Scalars S;
  CK(cudaMemcpy(&S, lp->S, sizeof(S), cudaMemcpyDeviceToHost));
  r->status = S.status;
  r->chosen = S.chosen;
  r->iters = S.k;
  r->restarts = S.restarts;
  r->seconds = (double)(S.t1_ns - S.t0_ns) * 1e-9;
  r->omega = S.omega;
  r->eta = S.eta;
  r->sigma_max = S.sigma_max;
  r->precision = lp->params.precision;
  return PDHGC_OK;
}

int check_params(const pdhgc_params* p) {
  if (!p) return PDHGC_ERR_INVALID_ARG;
  if (p->max_iters < 1 || p->check_period < 1 || p->check_period > 4096 || p->ruiz_iters < 0 ||
      p->ruiz_iters > 100 || p->power_iters < 1 || p->power_iters > 10000 || !(p->eta_factor > 0.0) ||
      !(p->eta_factor < 1.0) || !(p->time_limit_s > 0.0) || !(p->theta >= 0.0 && p->theta <= 1.0))
    return set_err(PDHGC_ERR_INVALID_ARG, "parameter out of range");
  if (p->precision != PDHGC_FP64 && p->precision != PDHGC_FP32_BULK)
    return set_err(PDHGC_ERR_INVALID_ARG, "precision must be PDHGC_FP64 or PDHGC_FP32_BULK");
  if (p->algorithm != PDHGC_ALG_AVERAGED && p->algorithm != PDHGC_ALG_HALPERN)
    return set_err(PDHGC_ERR_INVALID_ARG, "algorithm must be PDHGC_ALG_AVERAGED or PDHGC_ALG_HALPERN");
  if (p->algorithm == PDHGC_ALG_HALPERN) {
    if (!(p->reflection >= 0.0 && p->reflection <= 1.0) || !std::isfinite(p->pid_kp) ||
        !std::isfinite(p->pid_ki) || !std::isfinite(p->pid_kd))
      return set_err(PDHGC_ERR_INVALID_ARG, "reflection must lie in [0, 1] and the PID gains be finite");
  }
  return PDHGC_OK;
}

// uploads one CSR (padded by kPad) and builds its SELL-32 copy on the device
int setup_mat(pdhgc_lp* lp, pdhgc_lp::Mat& M, const Csr& C, cudaStream_t st) {
  const size_t nz = (size_t)C.nnz;
  M.rows = C.rows;
  M.cta_rows = C.cta_rows;
  M.long_rows = C.long_rows;
  M.nslices = C.nslices;
  M.nslots = C.slice_ptr[C.nslices];
  M.nb_cta = C.nb_cta();
  M.nb_warp = C.nb_warp();
  M.nb_sell = C.nb_sell();
  const size_t ns = (size_t)M.nslots;
  RET(lp->alloc(&M.rp, (size_t)C.rows + 1 + kPad));
  RET(lp->alloc(&M.col, nz + kPad));
  RET(lp->alloc(&M.val, nz + kPad));
  RET(lp->alloc(&M.hat, nz + kPad));
  RET(lp->alloc(&M.slice_ptr, (size_t)C.nslices + 1 + kPad));
  RET(lp->alloc(&M.slice_w, (size_t)C.nslices + kPad));
  RET(lp->alloc(&M.scol, ns + kPad));
  RET(lp->alloc(&M.smap, ns + kPad));
  RET(lp->alloc(&M.sval, ns + kPad));
  RET(lp->alloc(&M.shat, ns + kPad));
  RET(lp->alloc(&M.sblocks, C.sell_blocks.size() + 1));
  if (!C.sell_blocks.empty())
    CK(cudaMemcpyAsync(M.sblocks, C.sell_blocks.data(), C.sell_blocks.size() * sizeof(SellBlock),
                       cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(M.hat, 0, (nz + kPad) * 8, st));
  CK(cudaMemsetAsync(M.shat, 0, (ns + kPad) * 8, st));
  CK(cudaMemcpyAsync(M.rp, C.row_ptr.data(), ((size_t)C.rows + 1) * 4, cudaMemcpyHostToDevice, st));
  if (nz) {
    CK(cudaMemcpyAsync(M.col, C.col.data(), nz * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(M.val, C.val.data(), nz * 8, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(M.slice_ptr, C.slice_ptr.data(), ((size_t)C.nslices + 1) * 4, cudaMemcpyHostToDevice, st));
  if (C.nslices) CK(cudaMemcpyAsync(M.slice_w, C.slice_w.data(), (size_t)C.nslices * 4, cudaMemcpyHostToDevice, st));
  if (ns) {
    CK(cudaMemcpyAsync(M.smap, C.sell_map.data(), ns * 4, cudaMemcpyHostToDevice, st));
    k_sell_fill<<<grid_for((long long)ns), 256, 0, st>>>(M.smap, M.col, M.scol, (int)ns);
    k_sell_fill<<<grid_for((long long)ns), 256, 0, st>>>(M.smap, M.val, M.sval, (int)ns);
    lp->launches += 2;
    CKL();
  }
  return PDHGC_OK;
}

// uploads the chunked-pass plans of A' for FP64 and FP32 gathered vectors,
// and lets the chunked kernels use a chunk of dynamic shared memory
int setup_chunked(pdhgc_lp* lp, const Csr& T, cudaStream_t st) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpHT<true>, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpHT<true>, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpH32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpH32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpH32T<true>, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kChunkBytes));
  CK(cudaFuncSetAttribute(spmv_chunked<PrimalOpH32T<true>, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          kChunkBytes));
  for (int which = 0; which < 2; ++which) {
    pdhgc_lp::Chunked& C = which ? lp->ch32 : lp->ch64;
    ChunkPlan P;
    plan_chunks(T, which ? kChunkElems32 : kChunkElems64, sms, P);
    C.nch = P.nch;
    C.chunk = P.chunk;
    C.blocks = P.blocks;
    C.nslots = P.nslots;
    const size_t ns = (size_t)P.nslots, nu = (size_t)P.nunits;
    RET(lp->alloc(&C.map, ns + kPad));
    RET(lp->alloc(&C.idx, ns + kPad));
    RET(lp->alloc(&C.units, nu + 1));
    RET(lp->alloc(&C.uc_off, nu * P.nch + 1));
    RET(lp->alloc(&C.uc_cnt, nu * P.nch + 1));
    RET(lp->alloc(&C.warp_units, P.warp_units.size() + 1));
    if (which)
      RET(lp->alloc(&C.val32, ns + kPad));
    else
      RET(lp->alloc(&C.val64, ns + kPad));
    if (ns) {
      CK(cudaMemcpyAsync(C.map, P.slot_map.data(), ns * 4, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(C.idx, P.slot_idx.data(), ns * 2, cudaMemcpyHostToDevice, st));
    }
    if (nu) {
      CK(cudaMemcpyAsync(C.units, P.units.data(), nu * sizeof(ChunkUnit), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(C.uc_off, P.uc_off.data(), nu * P.nch * 4, cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(C.uc_cnt, P.uc_cnt.data(), nu * P.nch * 4, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(C.warp_units, P.warp_units.data(), P.warp_units.size() * 4, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // P's vectors go out of scope
  }
  return PDHGC_OK;
}

int check_corner_params(const pdhgc_corner_params& cp) {
  if (!(cp.eps_abs >= 0.0) || cp.min_iters < 0 || cp.max_iters < 1 || !(cp.time_limit_s > 0.0) ||
      !std::isfinite(cp.obj_scale) || (cp.stop_rule != 0 && cp.stop_rule != 1) ||
      (cp.row_rule != 0 && cp.row_rule != 1) || (cp.omega_rule != 0 && cp.omega_rule != 1))
    return set_err(PDHGC_ERR_INVALID_ARG, "corner parameter out of range");
  return PDHGC_OK;
}

// Algorithm 1's corner model: new bounds and objective (columns; `fixed`
// optionally flags the columns the reduced-cost rule fixed), new senses
// (rows), and the norms of the new objective for the primal weight
int corner_build(pdhgc_lp* lp, const pdhgc_corner_params& cp, int8_t* fixed) {
  cudaStream_t st = lp->stream;
  const DevModel md = model_orig(lp);
  RET(launch_tiles(lp, true, true,
                   CornerColsOp{lp->y1, lp->x1, lp->col_perm, md, lp->lhat_c, lp->uhat_c, lp->chat_c, cp.eps_abs,
                                cp.obj_scale, (unsigned long long)cp.obj_seed, fixed},
                   lp->pT, st));
  const double* ax = nullptr;
  if (cp.row_rule == 1) {
    k_fill<<<grid_for(lp->m), 256, 0, st>>>(lp->tmp_m, lp->m, 0.0);  // A = 0 leaves the pass empty
    lp->launches++;
    CKL();
    RET(launch_tiles(lp, false, true, SpmvOp<false>{lp->S, lp->x1, lp->tmp_m}, nullptr, st));
    ax = lp->tmp_m;
  }
  k_corner_rows<<<grid_for(lp->m), 256, 0, st>>>(lp->m, lp->ge, lp->Dr, lp->y1, cp.eps_abs, ax, lp->b_int,
                                                 lp->ge_c);
  lp->launches++;
  CKL();
  k_fold2<<<1, 256, 0, st>>>(lp->pT, lp->ntT, lp->scratch + 8);
  lp->launches++;
  CKL();
  return PDHGC_OK;
}

// the corner iterations from x_start (Section 3.1 stopping rule) and the report
int corner_run(pdhgc_lp* lp, const pdhgc_corner_params& cp, const double* x_start, pdhgc_report* r) {
  cudaStream_t st = lp->stream;
  const pdhgc_params& p = lp->params;
  PhaseInit pi{};
  pi.eps_rel = cp.eps_rel;
  pi.beta_suff = p.beta_suff;
  pi.beta_nec = p.beta_nec;
  pi.beta_art = p.beta_art;
  pi.theta = p.theta;
  pi.time_limit_s = cp.time_limit_s;
  pi.nb = lp->b_norm;
  pi.nc = 0.0;
  pi.max_iters = cp.max_iters;
  pi.min_iters = cp.min_iters;
  pi.check_period = p.check_period;
  pi.phase = 1;
  pi.stop_rule = cp.stop_rule;
  pi.use_cc2 = 1;
  pi.omega0 = cp.omega_rule == 1 ? lp->rep1.omega : 0.0;
  pi.algorithm = p.algorithm;
  pi.rho = p.reflection;
  pi.pid_kp = p.pid_kp;
  pi.pid_ki = p.pid_ki;
  pi.pid_kd = p.pid_kd;
  if (p.precision == PDHGC_FP32_BULK) {
    RET(to32(lp, lp->chat_c, lp->chat_c32, lp->n, st));
    RET(to32(lp, lp->lhat_c, lp->lhat_c32, lp->n, st));
    RET(to32(lp, lp->uhat_c, lp->uhat_c32, lp->n, st));
  }
  RET(run_phase(lp, model_corner(lp), model32_corner(lp), pi, x_start, lp->scratch + 8, lp->xc, nullptr, lp->x1));
  *r = pdhgc_report{};
  RET(fill_phase_report(lp, r));
  RET(run_report(lp, lp->xc, lp->y1, r));
  return PDHGC_OK;
}

// ---- the dual corner push (the dual counterpart of Algorithm 1) ----------

// Complementary slackness with the phase-1 point decides the model (user
// space, tolerance eps_abs): a pair (distance of x_j from a bound, the part
// of z_j that bound allows) or (slack of an inequality row, |y_i|) is read as
// "the first is nonzero" when it exceeds both eps_abs and the second.
// Columns: a bound stays unless x_j is off it in that sense, so a column
// strictly inside its bounds becomes free (its reduced cost is fixed at 0).
// z: the phase-1 reduced costs, unscaled (internal order).
__global__ void k_dual_cols(int n, const double* __restrict__ x1, const double* __restrict__ z,
                            const double* __restrict__ Dc, const double* __restrict__ l,
                            const double* __restrict__ u, const double* __restrict__ lhat,
                            const double* __restrict__ uhat, double eps_abs, double* __restrict__ lhat_d,
                            double* __restrict__ uhat_d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = Dc[j] * x1[j];
  const double dl = x - l[j], du = u[j] - x;
  const bool off_l = dl > eps_abs && dl > fmax(z[j], 0.0);
  const bool off_u = du > eps_abs && du > fmax(-z[j], 0.0);
  lhat_d[j] = (l[j] != -INFINITY && !off_l) ? lhat[j] : -INFINITY;
  uhat_d[j] = (u[j] != INFINITY && !off_u) ? uhat[j] : INFINITY;
}

// Rows: an inequality row whose slack exceeds eps_abs and |y_i| is inactive,
// and its dual is fixed at 0 (ge_d = kRowDualZero, b_hat' = 0); the other
// rows keep their sense and get the new objective b' = obj_scale U[0,1) per
// user row, negated on '<' rows and scaled by D_r.  part: per-block sums of
// b_hat'^2
__global__ void k_dual_rows(int m, const int8_t* __restrict__ ge, const double* __restrict__ Dr,
                            const double* __restrict__ sign, const double* __restrict__ b_int,
                            const int* __restrict__ row_perm, const double* __restrict__ ax,
                            const double* __restrict__ y1, double eps_abs, unsigned long long seed, double scale,
                            int8_t* __restrict__ ge_d, double* __restrict__ bhat_d, double* __restrict__ part) {
  __shared__ double s_red[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (i < m) {
    const double slack = ax[i] / Dr[i] - b_int[i];
    const bool zero = ge[i] && slack > eps_abs && slack > fabs(Dr[i] * y1[i]);
    ge_d[i] = zero ? kRowDualZero : ge[i];
    const double bh = zero ? 0.0 : Dr[i] * (sign[i] * (scale * splitmix_uniform(seed, (unsigned long long)row_perm[i])));
    bhat_d[i] = bh;
    sq = bh * bh;
  }
  for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    part[blockIdx.x] = t;
  }
}

// the start dual: y1, with 0 on the rows whose dual is fixed
__global__ void k_dual_start(int m, const double* __restrict__ y1, const int8_t* __restrict__ ge_d,
                             double* __restrict__ y0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) y0[i] = ge_d[i] == kRowDualZero ? 0.0 : y1[i];
}

__global__ void k_fold_into(const double* __restrict__ p, int nt, double* out) {
  __shared__ double s_tmp[32];
  const double v = block_fold(p, nt, false, s_tmp);
  if (threadIdx.x == 0) *out = v;
}

DevModel model_dual(const pdhgc_lp* lp) {
  return DevModel{lp->chat, lp->lhat_d, lp->uhat_d, lp->bhat_d, lp->Dr, lp->Dc, lp->ge_d};
}
DevModel32 model32_dual(const pdhgc_lp* lp) {
  return DevModel32{lp->chat32, lp->lhat_d32, lp->uhat_d32, lp->bhat_d32, lp->ge_d};
}

int ensure_dual(pdhgc_lp* lp) {
  if (!lp->have_dual_bufs) {
    RET(lp->alloc(&lp->lhat_d, (size_t)lp->n));
    RET(lp->alloc(&lp->uhat_d, (size_t)lp->n));
    RET(lp->alloc(&lp->bhat_d, (size_t)lp->m));
    RET(lp->alloc(&lp->yd, (size_t)lp->m));
    RET(lp->alloc(&lp->ge_d, (size_t)lp->m));
    lp->have_dual_bufs = true;
  }
  if (lp->params.precision == PDHGC_FP32_BULK && !lp->lhat_d32) {
    RET(lp->alloc(&lp->lhat_d32, (size_t)lp->n));
    RET(lp->alloc(&lp->uhat_d32, (size_t)lp->n));
    RET(lp->alloc(&lp->bhat_d32, (size_t)lp->m));
  }
  return PDHGC_OK;
}

// builds the dual corner model from the phase-1 point and runs its phase
int dual_corner_run(pdhgc_lp* lp, const pdhgc_corner_params& cp, pdhgc_report* r) {
  cudaStream_t st = lp->stream;
  const int m = lp->m, n = lp->n;
  RET(ensure_dual(lp));
  // the phase-1 reduced costs (unscaled) for the column rule
  RET(launch_tiles(lp, true, true, ZOp{lp->y1, model_orig(lp), lp->pi_w}, nullptr, st));
  k_dual_cols<<<grid_for(n), 256, 0, st>>>(n, lp->x1, lp->pi_w, lp->Dc, lp->l, lp->u, lp->lhat, lp->uhat,
                                           cp.eps_abs, lp->lhat_d, lp->uhat_d);
  k_fill<<<grid_for(m), 256, 0, st>>>(lp->tmp_m, m, 0.0);  // A = 0 leaves the pass empty
  lp->launches += 2;
  CKL();
  CK(cudaMemsetAsync(&lp->S->pi_zero, 0, sizeof(int), st));
  RET(launch_tiles(lp, false, true, SpmvOp<false>{lp->S, lp->x1, lp->tmp_m}, nullptr, st));
  const int gm = grid_for(m);
  k_dual_rows<<<gm, 256, 0, st>>>(m, lp->ge, lp->Dr, lp->sign, lp->b_int, lp->row_perm, lp->tmp_m, lp->y1,
                                  cp.eps_abs, (unsigned long long)cp.obj_seed, cp.obj_scale, lp->ge_d, lp->bhat_d,
                                  lp->pA);
  k_fold_into<<<1, 256, 0, st>>>(lp->pA, gm, lp->scratch + 10);  // pA holds >= ceil(m / 256) entries
  k_dual_start<<<gm, 256, 0, st>>>(m, lp->y1, lp->ge_d, lp->yd);
  lp->launches += 3;
  CKL();
  const pdhgc_params& p = lp->params;
  if (p.precision == PDHGC_FP32_BULK) {
    RET(to32(lp, lp->lhat_d, lp->lhat_d32, n, st));
    RET(to32(lp, lp->uhat_d, lp->uhat_d32, n, st));
    RET(to32(lp, lp->bhat_d, lp->bhat_d32, m, st));
  }
  PhaseInit pi{};
  pi.eps_rel = cp.eps_rel;
  pi.beta_suff = p.beta_suff;
  pi.beta_nec = p.beta_nec;
  pi.beta_art = p.beta_art;
  pi.theta = p.theta;
  pi.time_limit_s = cp.time_limit_s;
  pi.nb = lp->b_norm;
  pi.nc = lp->c_norm;
  pi.max_iters = cp.max_iters;
  pi.min_iters = cp.min_iters;
  pi.check_period = p.check_period;
  pi.phase = 1;
  pi.stop_rule = cp.stop_rule == 1 ? 1 : 2;
  pi.use_bb2 = 1;
  pi.algorithm = p.algorithm;
  pi.rho = p.reflection;
  pi.pid_kp = p.pid_kp;
  pi.pid_ki = p.pid_ki;
  pi.pid_kd = p.pid_kd;
  // x starts at proj(0) of the dual corner model's box, y at y1 (0 on fixed rows)
  RET(run_phase(lp, model_dual(lp), model32_dual(lp), pi, nullptr, lp->scratch + 8, lp->tmp_n, lp->yd, nullptr,
                lp->yd, lp->y1));
  *r = pdhgc_report{};
  RET(fill_phase_report(lp, r));
  RET(run_report(lp, lp->x1, lp->yd, r));
  return PDHGC_OK;
}

// ---- learned guidance: features, labels, held columns ---------------------

int ensure_gbufs(pdhgc_lp* lp) {
  if (lp->have_gbufs) return PDHGC_OK;
  const int n = lp->n, nb = grid_for(n);
  RET(lp->alloc(&lp->gfeat, (size_t)n * 32));
  RET(lp->alloc(&lp->gprob, n));
  RET(lp->alloc(&lp->ghold, n));
  RET(lp->alloc(&lp->gelig, n));
  RET(lp->alloc(&lp->glabel, n));
  RET(lp->alloc(&lp->gstage, n));
  RET(lp->alloc(&lp->gfixed, n));
  RET(lp->alloc(&lp->gnorm, n));
  RET(lp->alloc(&lp->gxs, n));
  RET(lp->alloc(&lp->gpart, (size_t)4 * nb + 4));
  RET(lp->alloc(&lp->gcount, 2));
  RET(lp->alloc(&lp->gblk, (size_t)nb + 1));
  lp->have_gbufs = true;
  return PDHGC_OK;
}

// the 8 ring slots of the history features, newest first: restart point e
// (e = 0 the start point) sits in slot e mod 8; fewer than 8 points are
// padded with the oldest
struct RingIdx {
  int slot[8];
};
RingIdx ring_index(long long restarts) {
  RingIdx ri{};
  const long long oldest = restarts > 7 ? restarts - 7 : 0;
  for (int k = 0; k < 8; ++k) {
    long long e = restarts - k;
    if (e < oldest) e = oldest;
    ri.slot[k] = (int)(e % 8);
  }
  return ri;
}

// ||A_hat_j||_2: one warp per row of A_hat'
__global__ void k_col_norm(int n, const int* __restrict__ rp, const double* __restrict__ hat, double* __restrict__ out) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= n) return;
  const int j = (int)wid;
  double s = 0.0;
  for (int k = rp[j] + lane; k < rp[j + 1]; k += 32) s = fma(hat[k], hat[k], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[j] = sqrt(s);
}

// per-block sums of squares of the four feature groups (c', ||A_j||, x history, z history)
__global__ void k_feat_sums(int n, const double* __restrict__ cc, const double* __restrict__ cn,
                            const float* __restrict__ rx, const float* __restrict__ rz, RingIdx ri,
                            double* __restrict__ part) {
  __shared__ double s_w[4][8];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (j < n) {
    v[0] = cc[j] * cc[j];
    v[1] = cn[j] * cn[j];
    for (int k = 0; k < 8; ++k) {
      const double a = rx[(size_t)ri.slot[k] * n + j], b = rz[(size_t)ri.slot[k] * n + j];
      v[2] += a * a;
      v[3] += b * b;
    }
  }
  for (int q = 0; q < 4; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) s_w[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[threadIdx.x][w];
    part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// 1 / RMS of each group (1 when the group is all zero)
__global__ void k_feat_fold(const double* __restrict__ part, int nb, int n, double* __restrict__ inv) {
  __shared__ double s_tmp[32];
  for (int q = 0; q < 4; ++q) {
    const double v = block_fold(part + (size_t)q * nb, nb, false, s_tmp);
    if (threadIdx.x == 0) {
      const double cnt = q < 2 ? (double)n : 8.0 * (double)n;
      const double r = sqrt(v / cnt);
      inv[q] = r > 0.0 ? 1.0 / r : 1.0;
    }
    __syncthreads();
  }
}

// feature row of column j (row col_perm[j] when perm is given, else j) and
// its eligibility: not fixed by the reduced-cost rule, a finite bound
__global__ void k_feat_write(int n, const double* __restrict__ cc, const double* __restrict__ cn,
                             const float* __restrict__ rx, const float* __restrict__ rz, RingIdx ri,
                             const double* __restrict__ inv, const int* __restrict__ perm,
                             const int8_t* __restrict__ fixed, const double* __restrict__ lhat,
                             const double* __restrict__ uhat, uint16_t* __restrict__ feat,
                             uint8_t* __restrict__ elig) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const size_t row = perm ? (size_t)perm[j] : (size_t)j;
  double f[18];
  f[0] = cc[j] * inv[0];
  f[1] = cn[j] * inv[1];
  for (int k = 0; k < 8; ++k) {
    f[2 + k] = (double)rx[(size_t)ri.slot[k] * n + j] * inv[2];
    f[10 + k] = (double)rz[(size_t)ri.slot[k] * n + j] * inv[3];
  }
  uint32_t* dst = reinterpret_cast<uint32_t*>(feat + row * 32);
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    const uint32_t lo = 2 * w < 18 ? __bfloat16_as_ushort(__double2bfloat16(f[2 * w])) : 0u;
    const uint32_t hi = 2 * w + 1 < 18 ? __bfloat16_as_ushort(__double2bfloat16(f[2 * w + 1])) : 0u;
    dst[w] = lo | (hi << 16);
  }
  if (elig) elig[row] = (!fixed[j] && (lhat[j] != -INFINITY || uhat[j] != INFINITY)) ? 1 : 0;
}

int build_features(pdhgc_lp* lp, const pdhgc_corner_params& cp, bool user_order, uint16_t* feat, uint8_t* elig) {
  cudaStream_t st = lp->stream;
  const int n = lp->n, nb = grid_for(n);
  RET(corner_build(lp, cp, lp->gfixed));
  k_col_norm<<<grid_for((long long)n * 32), 256, 0, st>>>(n, lp->T.rp, lp->T.hat, lp->gnorm);
  const RingIdx ri = ring_index(lp->rep1.restarts);
  double* inv = lp->gpart + (size_t)4 * nb;
  k_feat_sums<<<nb, 256, 0, st>>>(n, lp->chat_c, lp->gnorm, lp->ring_x, lp->ring_z, ri, lp->gpart);
  k_feat_fold<<<1, 256, 0, st>>>(lp->gpart, nb, n, inv);
  k_feat_write<<<nb, 256, 0, st>>>(n, lp->chat_c, lp->gnorm, lp->ring_x, lp->ring_z, ri, inv,
                                   user_order ? lp->col_perm : nullptr, lp->gfixed, lp->lhat, lp->uhat, feat, elig);
  lp->launches += 4;
  CKL();
  return PDHGC_OK;
}

__global__ void k_hold_from_p(int n, const float* __restrict__ p, double thr, uint8_t* __restrict__ hold) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) hold[j] = (double)p[j] >= thr ? 1 : 0;
}

__global__ void k_gather_u8(int n, const int* __restrict__ perm, const uint8_t* __restrict__ src,
                            uint8_t* __restrict__ dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) dst[j] = src[perm[j]] != 0 ? 1 : 0;
}

// held columns: l_hat' = u_hat' = the bound nearest to x1 (ties: lower), the
// start point there; count[0] eligible columns, count[1] held columns
__global__ void k_apply_hold(int n, const uint8_t* __restrict__ hold, const int8_t* __restrict__ fixed,
                             const double* __restrict__ x1, const double* __restrict__ lhat,
                             const double* __restrict__ uhat, double* __restrict__ lc, double* __restrict__ uc,
                             double* __restrict__ xs, long long* __restrict__ count) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = x1[j], l = lhat[j], u = uhat[j];
  const bool lf = l != -INFINITY, uf = u != INFINITY;
  double xj = x;
  if (!fixed[j] && (lf || uf)) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&count[0]), 1ull);
    if (hold[j]) {
      const double dl = lf ? x - l : INFINITY, du = uf ? u - x : INFINITY;
      const double b = dl <= du ? l : u;
      lc[j] = b;
      uc[j] = b;
      xj = b;
      atomicAdd(reinterpret_cast<unsigned long long*>(&count[1]), 1ull);
    }
  }
  xs[j] = xj;
}

// training label of column j (user row): the corner x_j within 1e-6 (user
// space) of the bound a hold would use, the one of [l_hat, u_hat] nearest to
// the phase-1 x1_j; explicit roundings keep the products out of an FMA
__global__ void k_labels(int n, const double* __restrict__ xc, const double* __restrict__ x1,
                         const double* __restrict__ Dc, const double* __restrict__ lhat,
                         const double* __restrict__ uhat, const int* __restrict__ perm, uint8_t* __restrict__ lab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double l = lhat[j], u = uhat[j], v = x1[j];
  const bool lf = l != -INFINITY, uf = u != INFINITY;
  uint8_t out = 0;
  if (lf || uf) {
    const double dl = lf ? v - l : INFINITY, du = uf ? u - v : INFINITY;
    const double nb = dl <= du ? l : u;
    const double x = __dmul_rn(Dc[j], xc[j]), b = __dmul_rn(Dc[j], nb);
    out = fabs(x - b) <= 1e-6 ? 1 : 0;
  }
  lab[perm[j]] = out;
}

// deterministic stream compaction of the flagged rows (256-row blocks)
__global__ void k_count_flags(int n, const uint8_t* __restrict__ flag, int* __restrict__ blk) {
  __shared__ int s_w[8];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned b = __ballot_sync(0xffffffffu, j < n && flag[j] != 0);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
    blk[blockIdx.x] = t;
  }
}

__global__ void k_scan_blocks(int nb, int* __restrict__ blk, long long* __restrict__ total) {
  long long run = 0;
  for (int b = 0; b < nb; ++b) {
    const int c = blk[b];
    blk[b] = (int)run;
    run += c;
  }
  total[0] = run;
}

__global__ void k_compact(int n, const uint8_t* __restrict__ flag, const int* __restrict__ blk_off,
                          const uint16_t* __restrict__ feat_in, const uint8_t* __restrict__ lab_in,
                          uint16_t* __restrict__ feat_out, uint8_t* __restrict__ lab_out) {
  __shared__ int s_w[8];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool f = j < n && flag[j] != 0;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_w[warp] = __popc(b);
  __syncthreads();
  int off = blk_off[blockIdx.x];
  for (int w = 0; w < warp; ++w) off += s_w[w];
  off += __popc(b & ((1u << lane) - 1u));
  if (f) {
    const uint4* src = reinterpret_cast<const uint4*>(feat_in + (size_t)j * 32);
    uint4* dst = reinterpret_cast<uint4*>(feat_out + (size_t)off * 32);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = src[q];
    lab_out[off] = lab_in[j];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

void pdhgc_default_params(pdhgc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps_rel = 1e-6;
  p->max_iters = 1000000;
  p->time_limit_s = 3600.0;
  p->check_period = 64;
  p->beta_suff = 0.2;
  p->beta_nec = 0.8;
  p->beta_art = 0.36;
  p->theta = 0.5;
  p->eta_factor = 0.998;
  p->ruiz_iters = 10;
  p->power_iters = 100;
  p->precision = PDHGC_FP64;
  p->algorithm = PDHGC_ALG_AVERAGED;
  p->reflection = 1.0;
  p->pid_kp = 0.99;
  p->pid_ki = 0.01;
  p->pid_kd = 0.0;
}

void pdhgc_default_corner_params(pdhgc_corner_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps_abs = 1e-6;
  p->eps_rel = 1e-6;
  p->min_iters = 100;
  p->max_iters = 1000000;
  p->time_limit_s = 3600.0;
  p->obj_seed = 0;
  p->obj_scale = 1.0;
  p->stop_rule = 0;
}

int pdhgc_lp_create(pdhgc_lp** out, int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                    const int32_t* col_idx, const double* val, const double* b, const double* c,
                    const double* lb, const double* ub, const int8_t* sense, int inputs_on_device,
                    void* cuda_stream) {
  if (!out) return set_err(PDHGC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (inputs_on_device != 0 && inputs_on_device != 1)
    return set_err(PDHGC_ERR_INVALID_ARG, "inputs_on_device must be 0 or 1");
  if (m < 1 || n < 1 || nnz < 0) return set_err(PDHGC_ERR_INVALID_ARG, "m and n must be >= 1, nnz >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // host copies for validation and layout
  std::vector<int64_t> h_rp;
  std::vector<int32_t> h_col;
  std::vector<double> h_val, h_b, h_c, h_l, h_u;
  std::vector<int8_t> h_s;
  if (inputs_on_device) {
    if (!row_ptr || !b || !c || (nnz > 0 && (!col_idx || !val)))
      return set_err(PDHGC_ERR_INVALID_ARG, "NULL array argument");
    h_rp.resize((size_t)m + 1);
    h_col.resize((size_t)nnz);
    h_val.resize((size_t)nnz);
    h_b.resize(m);
    h_c.resize(n);
    CK(cudaMemcpyAsync(h_rp.data(), row_ptr, h_rp.size() * 8, cudaMemcpyDeviceToHost, st));
    if (nnz > 0) {
      CK(cudaMemcpyAsync(h_col.data(), col_idx, (size_t)nnz * 4, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(h_val.data(), val, (size_t)nnz * 8, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(h_b.data(), b, (size_t)m * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h_c.data(), c, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    if (lb) {
      h_l.resize(n);
      CK(cudaMemcpyAsync(h_l.data(), lb, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    }
    if (ub) {
      h_u.resize(n);
      CK(cudaMemcpyAsync(h_u.data(), ub, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    }
    if (sense) {
      h_s.resize(m);
      CK(cudaMemcpyAsync(h_s.data(), sense, (size_t)m, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    row_ptr = h_rp.data();
    col_idx = h_col.data();
    val = h_val.data();
    b = h_b.data();
    c = h_c.data();
    lb = lb ? h_l.data() : nullptr;
    ub = ub ? h_u.data() : nullptr;
    sense = sense ? h_s.data() : nullptr;
  }
  Prepared P;
  std::string detail;
  int rc = prepare_lp(P, m, n, nnz, row_ptr, col_idx, val, b, c, lb, ub, sense, detail);
  if (rc != PDHGC_OK) return set_err(rc, detail);

  std::unique_ptr<pdhgc_lp> lp(new pdhgc_lp());
  lp->m = m;
  lp->n = n;
  lp->nnz = nnz;
  lp->stream = st;
  lp->b_norm = P.b_norm;
  lp->c_norm = P.c_norm;
  CK(cudaStreamCreateWithFlags(&lp->cap_stream, cudaStreamNonBlocking));
  const size_t nz = (size_t)nnz;
  RET(setup_mat(lp.get(), lp->A, P.A, st));
  RET(setup_mat(lp.get(), lp->T, P.AT, st));
  lp->ntA = lp->A.nblocks();
  lp->ntT = lp->T.nblocks();
  RET(lp->alloc(&lp->err, 1));
  RET(lp->alloc(&lp->b_int, m));
  RET(lp->alloc(&lp->sign, m));
  RET(lp->alloc(&lp->ge, m));
  RET(lp->alloc(&lp->ge_c, m));
  RET(lp->alloc(&lp->c, n));
  RET(lp->alloc(&lp->l, n));
  RET(lp->alloc(&lp->u, n));
  RET(lp->alloc(&lp->Dr, m));
  RET(lp->alloc(&lp->Dc, n));
  RET(lp->alloc(&lp->bhat, m));
  RET(lp->alloc(&lp->chat, n));
  RET(lp->alloc(&lp->lhat, n));
  RET(lp->alloc(&lp->uhat, n));
  RET(lp->alloc(&lp->rfac, m));
  RET(lp->alloc(&lp->cfac, n));
  RET(lp->alloc(&lp->row_perm, m));
  RET(lp->alloc(&lp->col_perm, n));
  RET(lp->alloc(&lp->it.x, n));
  RET(lp->alloc(&lp->it.xbar, n));
  RET(lp->alloc(&lp->it.sum_x, n));
  RET(lp->alloc(&lp->it.x_r, n));
  RET(lp->alloc(&lp->it.y, m));
  RET(lp->alloc(&lp->it.sum_y, m));
  RET(lp->alloc(&lp->it.y_r, m));
  RET(lp->alloc(&lp->x1, n));
  RET(lp->alloc(&lp->y1, m));
  RET(lp->alloc(&lp->xc, n));
  RET(lp->alloc(&lp->chat_c, n));
  RET(lp->alloc(&lp->ring_x, (size_t)8 * n));
  RET(lp->alloc(&lp->ring_z, (size_t)8 * n));
  RET(lp->alloc(&lp->z_cur, n));
  RET(lp->alloc(&lp->z_avg, n));
  RET(lp->alloc(&lp->lhat_c, n));
  RET(lp->alloc(&lp->uhat_c, n));
  RET(lp->alloc(&lp->pi_v, n));
  RET(lp->alloc(&lp->pi_w, n));
  RET(lp->alloc(&lp->pi_u, m));
  RET(lp->alloc(&lp->tmp_n, n));
  RET(lp->alloc(&lp->tmp_m, m));
  RET(lp->alloc(&lp->pA, (size_t)16 * (lp->ntA > 0 ? lp->ntA : 1)));
  RET(lp->alloc(&lp->pT, (size_t)16 * (lp->ntT > 0 ? lp->ntT : 1)));
  RET(lp->alloc(&lp->scratch, 64));
  RET(lp->alloc(&lp->S, 1));
  RET(lp->alloc(&lp->rep, 1));
  CK(cudaMemsetAsync(lp->err, 0, sizeof(int), st));
  CK(cudaMemcpyAsync(lp->b_int, P.b_int.data(), (size_t)m * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->sign, P.sign.data(), (size_t)m * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->ge, P.ge.data(), (size_t)m, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->c, P.c.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->l, P.l.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->u, P.u.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->row_perm, P.row_perm.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(lp->col_perm, P.col_perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(lp->S, 0, sizeof(Scalars), st));
  CK(cudaStreamSynchronize(st));  // the host vectors of P go out of scope
  pdhgc_default_params(&lp->params);
  *out = lp.release();
  return PDHGC_OK;
}

int pdhgc_solve(pdhgc_lp* lp, const pdhgc_params* params, pdhgc_report* out) {
  if (!lp) return set_err(PDHGC_ERR_INVALID_ARG, "lp is NULL");
  pdhgc_params p;
  if (params) p = *params; else pdhgc_default_params(&p);
  RET(check_params(&p));
  lp->params = p;
  lp->have_phase1 = false;
  lp->have_corner = false;
  lp->have_dual = false;
  RET(setup_scaling(lp, p));
  if (p.precision == PDHGC_FP32_BULK) {
    RET(ensure_fp32(lp));
    RET(convert_fp32(lp, lp->stream));
  }
  PhaseInit pi{};
  pi.eps_rel = p.eps_rel;
  pi.beta_suff = p.beta_suff;
  pi.beta_nec = p.beta_nec;
  pi.beta_art = p.beta_art;
  pi.theta = p.theta;
  pi.time_limit_s = p.time_limit_s;
  pi.nb = lp->b_norm;
  pi.nc = lp->c_norm;
  pi.max_iters = p.max_iters;
  pi.min_iters = 0;
  pi.check_period = p.check_period;
  pi.phase = 0;
  pi.stop_rule = 0;
  pi.use_cc2 = 0;
  pi.algorithm = p.algorithm;
  pi.rho = p.reflection;
  pi.pid_kp = p.pid_kp;
  pi.pid_ki = p.pid_ki;
  pi.pid_kd = p.pid_kd;
  RET(run_phase(lp, model_orig(lp), model32_orig(lp), pi, nullptr, nullptr, lp->x1, lp->y1, nullptr));
  pdhgc_report r{};
  RET(fill_phase_report(lp, &r));
  RET(run_report(lp, lp->x1, lp->y1, &r));
  lp->rep1 = r;
  lp->have_phase1 = true;
  if (out) *out = r;
  return PDHGC_OK;
}

int pdhgc_corner_phase(pdhgc_lp* lp, const pdhgc_corner_params* params, pdhgc_report* out) {
  if (!lp) return set_err(PDHGC_ERR_INVALID_ARG, "lp is NULL");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run on this handle");
  pdhgc_corner_params cp;
  if (params) cp = *params; else pdhgc_default_corner_params(&cp);
  RET(check_corner_params(cp));
  lp->have_corner = false;
  RET(corner_build(lp, cp, nullptr));
  pdhgc_report r{};
  RET(corner_run(lp, cp, lp->x1, &r));
  lp->repc = r;
  lp->have_corner = true;
  lp->cp_last = cp;
  if (out) *out = r;
  return PDHGC_OK;
}

int pdhgc_dual_corner_phase(pdhgc_lp* lp, const pdhgc_corner_params* params, pdhgc_report* out) {
  if (!lp) return set_err(PDHGC_ERR_INVALID_ARG, "lp is NULL");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run on this handle");
  pdhgc_corner_params cp;
  if (params) cp = *params; else pdhgc_default_corner_params(&cp);
  RET(check_corner_params(cp));
  if (cp.row_rule != 0 || cp.omega_rule != 0)
    return set_err(PDHGC_ERR_INVALID_ARG, "the dual corner phase takes row_rule 0 and omega_rule 0");
  lp->have_dual = false;
  pdhgc_report r{};
  RET(dual_corner_run(lp, cp, &r));
  lp->repd = r;
  lp->have_dual = true;
  if (out) *out = r;
  return PDHGC_OK;
}

void pdhgc_default_guide_params(pdhgc_guide_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->threshold = 0.9;
  p->guided_max_iters = 0;
  p->fallback = 1;
}

int pdhgc_guide_features(pdhgc_lp* lp, const pdhgc_corner_params* params, uint16_t* feat, uint8_t* eligible) {
  if (!lp || !feat) return set_err(PDHGC_ERR_INVALID_ARG, "lp or feat is NULL");
  if (((uintptr_t)feat & 15u) != 0u) return set_err(PDHGC_ERR_INVALID_ARG, "feat must be 16-byte aligned");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run on this handle");
  pdhgc_corner_params cp;
  if (params) cp = *params; else pdhgc_default_corner_params(&cp);
  RET(check_corner_params(cp));
  RET(ensure_gbufs(lp));
  RET(build_features(lp, cp, true, feat, eligible));
  CK(cudaStreamSynchronize(lp->stream));
  return PDHGC_OK;
}

int pdhgc_guide_dataset_append(pdhgc_lp* lp, uint16_t* feat, uint8_t* labels, int64_t capacity, int64_t* count) {
  if (!lp || !feat || !labels || !count) return set_err(PDHGC_ERR_INVALID_ARG, "NULL argument");
  if (((uintptr_t)feat & 15u) != 0u) return set_err(PDHGC_ERR_INVALID_ARG, "feat must be 16-byte aligned");
  if (*count < 0 || *count > capacity) return set_err(PDHGC_ERR_INVALID_ARG, "count outside [0, capacity]");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run on this handle");
  if (!lp->have_corner) return set_err(PDHGC_ERR_NO_CORNER, "no corner result on this handle");
  RET(ensure_gbufs(lp));
  cudaStream_t st = lp->stream;
  const int n = lp->n, nb = grid_for(n);
  RET(build_features(lp, lp->cp_last, true, lp->gfeat, lp->gelig));
  k_labels<<<nb, 256, 0, st>>>(n, lp->xc, lp->x1, lp->Dc, lp->lhat, lp->uhat, lp->col_perm, lp->glabel);
  k_count_flags<<<nb, 256, 0, st>>>(n, lp->gelig, lp->gblk);
  k_scan_blocks<<<1, 1, 0, st>>>(nb, lp->gblk, lp->gcount);
  lp->launches += 3;
  CKL();
  long long total = 0;
  CK(cudaMemcpyAsync(&total, lp->gcount, sizeof(total), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (total > capacity - *count)
    return set_err(PDHGC_ERR_BUFFER, "dataset capacity too small: need " + std::to_string(*count + total) + " rows");
  k_compact<<<nb, 256, 0, st>>>(n, lp->gelig, lp->gblk, lp->gfeat, lp->glabel, feat + (size_t)(*count) * 32,
                                labels + *count);
  lp->launches++;
  CKL();
  CK(cudaStreamSynchronize(st));
  *count += total;
  return PDHGC_OK;
}

int pdhgc_corner_phase_guided(pdhgc_lp* lp, const pdhgc_corner_params* params, const pdhgc_guide_params* gparams,
                              pdhgc_guide* g, const uint8_t* hold, int hold_on_device, pdhgc_report* out,
                              pdhgc_guide_report* gout) {
  if (!lp) return set_err(PDHGC_ERR_INVALID_ARG, "lp is NULL");
  if ((g == nullptr) == (hold == nullptr))
    return set_err(PDHGC_ERR_INVALID_ARG, "give exactly one of the network and the hold mask");
  if (hold && hold_on_device != 0 && hold_on_device != 1)
    return set_err(PDHGC_ERR_INVALID_ARG, "hold_on_device must be 0 or 1");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run on this handle");
  pdhgc_corner_params cp;
  if (params) cp = *params; else pdhgc_default_corner_params(&cp);
  RET(check_corner_params(cp));
  pdhgc_guide_params gp;
  if (gparams) gp = *gparams; else pdhgc_default_guide_params(&gp);
  if (!std::isfinite(gp.threshold) || (gp.fallback != 0 && gp.fallback != 1) || gp.guided_max_iters < 0)
    return set_err(PDHGC_ERR_INVALID_ARG, "guide parameter out of range");
  pdhgc_corner_params cpg = cp;
  if (gp.guided_max_iters > 0 && gp.guided_max_iters < cp.max_iters) cpg.max_iters = gp.guided_max_iters;
  RET(ensure_gbufs(lp));
  lp->have_corner = false;
  cudaStream_t st = lp->stream;
  const int n = lp->n, nb = grid_for(n);
  const auto t0 = std::chrono::steady_clock::now();
  RET(corner_build(lp, cp, lp->gfixed));
  if (g) {
    RET(build_features(lp, cp, false, lp->gfeat, nullptr));
    RET(guide_forward(g, reinterpret_cast<const __nv_bfloat16*>(lp->gfeat), n, lp->gprob, st));
    RET(guide_check_error(g, st));
    k_hold_from_p<<<nb, 256, 0, st>>>(n, lp->gprob, gp.threshold, lp->ghold);
  } else {
    const uint8_t* src = hold;
    if (!hold_on_device) {
      CK(cudaMemcpyAsync(lp->gstage, hold, (size_t)n, cudaMemcpyHostToDevice, st));
      src = lp->gstage;
    }
    k_gather_u8<<<nb, 256, 0, st>>>(n, lp->col_perm, src, lp->ghold);
  }
  CK(cudaMemsetAsync(lp->gcount, 0, 2 * sizeof(long long), st));
  k_apply_hold<<<nb, 256, 0, st>>>(n, lp->ghold, lp->gfixed, lp->x1, lp->lhat, lp->uhat, lp->lhat_c, lp->uhat_c,
                                   lp->gxs, lp->gcount);
  lp->launches += 2;
  CKL();
  long long counts[2] = {0, 0};
  CK(cudaMemcpyAsync(counts, lp->gcount, sizeof(counts), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const auto t1 = std::chrono::steady_clock::now();
  pdhgc_report r{};
  RET(corner_run(lp, cpg, lp->gxs, &r));
  const auto t2 = std::chrono::steady_clock::now();
  pdhgc_guide_report gr{};
  gr.status = r.status;
  gr.eligible = counts[0];
  gr.held = counts[1];
  gr.guided_iters = r.iters;
  gr.guided_seconds = std::chrono::duration<double>(t2 - t0).count();
  gr.infer_seconds = std::chrono::duration<double>(t1 - t0).count();
  gr.guided_rel_kkt = r.rel_kkt;
  gr.guided_corner_measure = r.corner_measure;
  const bool regressed = r.status == PDHGC_STATUS_CORNER_LIMIT ||
                         r.rel_kkt > std::fmax(lp->rep1.rel_kkt, cp.eps_rel) ||
                         r.corner_measure > lp->rep1.corner_measure;
  if (gp.fallback && regressed) {
    RET(corner_build(lp, cp, nullptr));
    RET(corner_run(lp, cp, lp->x1, &r));
    gr.fell_back = 1;
    gr.status = PDHGC_STATUS_GUIDE_FALLBACK;
  }
  lp->repc = r;
  lp->have_corner = true;
  lp->cp_last = cp;
  if (out) *out = r;
  if (gout) *gout = gr;
  return PDHGC_OK;
}

// ---- checkpoint / restore of a handle's results ----------------------------

namespace {
struct StateHeader {
  char magic[8];  // "PDHGCST1"
  int32_t version, m, n, pad;
  int64_t nnz;
  int32_t have_phase1, have_corner;
  pdhgc_params params;
  pdhgc_corner_params cp_last;
  pdhgc_report rep1, repc;
};
constexpr char kStateMagic[8] = {'P', 'D', 'H', 'G', 'C', 'S', 'T', '1'};
size_t state_bytes(int m, int n) {
  return sizeof(StateHeader) + 8 * (2 * (size_t)m + 3 * (size_t)n) + 4 * 16 * (size_t)n;
}
}  // namespace

int pdhgc_get_state(pdhgc_lp* lp, void* buf, size_t* bytes) {
  if (!lp || !bytes) return set_err(PDHGC_ERR_INVALID_ARG, "lp or bytes is NULL");
  const int m = lp->m, n = lp->n;
  const size_t need = state_bytes(m, n);
  if (!buf) {
    *bytes = need;
    return PDHGC_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return set_err(PDHGC_ERR_BUFFER, "state buffer too small: need " + std::to_string(need) + " bytes");
  }
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.version = 3;  // 2: pdhgc_params carries the inner-loop fields; 3: corner omega_rule
  h.m = m;
  h.n = n;
  h.nnz = lp->nnz;
  h.have_phase1 = lp->have_phase1 ? 1 : 0;
  h.have_corner = lp->have_corner ? 1 : 0;
  h.params = lp->params;
  h.cp_last = lp->cp_last;
  h.rep1 = lp->rep1;
  h.repc = lp->repc;
  unsigned char* o = static_cast<unsigned char*>(buf);
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  cudaStream_t st = lp->stream;
  struct Part {
    const void* src;
    size_t bytes;
  } parts[] = {{lp->Dr, 8 * (size_t)m},      {lp->Dc, 8 * (size_t)n},         {lp->x1, 8 * (size_t)n},
               {lp->y1, 8 * (size_t)m},      {lp->xc, 8 * (size_t)n},         {lp->ring_x, 32 * (size_t)n},
               {lp->ring_z, 32 * (size_t)n}};
  for (const Part& q : parts) {
    CK(cudaMemcpyAsync(o, q.src, q.bytes, cudaMemcpyDeviceToHost, st));
    o += q.bytes;
  }
  CK(cudaStreamSynchronize(st));
  *bytes = need;
  return PDHGC_OK;
}

int pdhgc_set_state(pdhgc_lp* lp, const void* buf, size_t bytes) {
  if (!lp || !buf) return set_err(PDHGC_ERR_INVALID_ARG, "lp or buf is NULL");
  const int m = lp->m, n = lp->n;
  if (bytes < sizeof(StateHeader)) return set_err(PDHGC_ERR_INVALID_ARG, "state buffer too short");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 3)
    return set_err(PDHGC_ERR_INVALID_ARG, "not a pdhgc state (magic or version)");
  if (h.m != m || h.n != n || h.nnz != lp->nnz || bytes != state_bytes(m, n))
    return set_err(PDHGC_ERR_INVALID_ARG, "state was taken from an LP of another shape");
  RET(check_params(&h.params));
  const unsigned char* in = static_cast<const unsigned char*>(buf) + sizeof(StateHeader);
  const double* Dr_s = reinterpret_cast<const double*>(in);
  const double* Dc_s = Dr_s + m;
  cudaStream_t st = lp->stream;
  lp->have_phase1 = false;
  lp->have_corner = false;
  // the scaling, step size and FP32 copies are recomputed (deterministic) and
  // must reproduce the saved factors bit for bit
  RET(setup_scaling(lp, h.params));
  if (h.params.precision == PDHGC_FP32_BULK) {
    RET(ensure_fp32(lp));
    RET(convert_fp32(lp, st));
  }
  std::vector<double> Dr(m), Dc(n);
  CK(cudaMemcpyAsync(Dr.data(), lp->Dr, 8 * (size_t)m, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(Dc.data(), lp->Dc, 8 * (size_t)n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (std::memcmp(Dr.data(), Dr_s, 8 * (size_t)m) != 0 || std::memcmp(Dc.data(), Dc_s, 8 * (size_t)n) != 0)
    return set_err(PDHGC_ERR_INVALID_ARG, "state was taken from another LP (scaling factors differ)");
  const unsigned char* o = in + 8 * ((size_t)m + n);
  struct Part {
    void* dst;
    size_t bytes;
  } parts[] = {{lp->x1, 8 * (size_t)n}, {lp->y1, 8 * (size_t)m}, {lp->xc, 8 * (size_t)n},
               {lp->ring_x, 32 * (size_t)n}, {lp->ring_z, 32 * (size_t)n}};
  for (const Part& q : parts) {
    CK(cudaMemcpyAsync(q.dst, o, q.bytes, cudaMemcpyHostToDevice, st));
    o += q.bytes;
  }
  CK(cudaStreamSynchronize(st));
  lp->params = h.params;
  lp->cp_last = h.cp_last;
  lp->rep1 = h.rep1;
  lp->repc = h.repc;
  lp->have_phase1 = h.have_phase1 != 0;
  lp->have_corner = h.have_corner != 0 && lp->have_phase1;
  return PDHGC_OK;
}

int pdhgc_kkt_report(pdhgc_lp* lp, int which, pdhgc_report* out) {
  if (!lp || !out || (which != PDHGC_PHASE1 && which != PDHGC_CORNER && which != PDHGC_DUAL_CORNER))
    return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run");
  if (which == PDHGC_CORNER && !lp->have_corner) return set_err(PDHGC_ERR_NO_CORNER, "no corner result");
  if (which == PDHGC_DUAL_CORNER && !lp->have_dual) return set_err(PDHGC_ERR_NO_CORNER, "no dual corner result");
  pdhgc_report r = which == PDHGC_PHASE1 ? lp->rep1 : (which == PDHGC_CORNER ? lp->repc : lp->repd);
  RET(run_report(lp, which == PDHGC_CORNER ? lp->xc : lp->x1, which == PDHGC_DUAL_CORNER ? lp->yd : lp->y1, &r));
  *out = r;
  return PDHGC_OK;
}

static int copy_out(pdhgc_lp* lp, double* dst, const double* dev_user, size_t count, int on_device) {
  CK(cudaMemcpyAsync(dst, dev_user, count * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     lp->stream));
  return PDHGC_OK;
}

int pdhgc_get_solution(pdhgc_lp* lp, int which, double* x, double* y, double* z, int on_device) {
  if (!lp || (which != PDHGC_PHASE1 && which != PDHGC_CORNER && which != PDHGC_DUAL_CORNER) ||
      (on_device != 0 && on_device != 1))
    return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run");
  if (which == PDHGC_CORNER && !lp->have_corner) return set_err(PDHGC_ERR_NO_CORNER, "no corner result");
  if (which == PDHGC_DUAL_CORNER && !lp->have_dual) return set_err(PDHGC_ERR_NO_CORNER, "no dual corner result");
  cudaStream_t st = lp->stream;
  const int m = lp->m, n = lp->n;
  const double* ysrc = which == PDHGC_DUAL_CORNER ? lp->yd : lp->y1;
  if (x) {
    k_unpermute<<<grid_for(n), 256, 0, st>>>(n, lp->col_perm, which == PDHGC_CORNER ? lp->xc : lp->x1, lp->Dc,
                                            nullptr, lp->tmp_n);
    lp->launches++;
    CKL();
    RET(copy_out(lp, x, lp->tmp_n, n, on_device));
  }
  if (y) {
    k_unpermute<<<grid_for(m), 256, 0, st>>>(m, lp->row_perm, ysrc, lp->Dr, lp->sign, lp->tmp_m);
    lp->launches++;
    CKL();
    RET(copy_out(lp, y, lp->tmp_m, m, on_device));
  }
  if (z) {
    // the unpermute below reads pi_w; the stream orders it after the ZOp pass
    RET(launch_tiles(lp, true, true, ZOp{ysrc, model_orig(lp), lp->pi_w}, nullptr, st));
    k_unpermute<<<grid_for(n), 256, 0, st>>>(n, lp->col_perm, lp->pi_w, nullptr, nullptr, lp->tmp_n);
    lp->launches++;
    CKL();
    RET(copy_out(lp, z, lp->tmp_n, n, on_device));
  }
  CK(cudaStreamSynchronize(st));
  return PDHGC_OK;
}

int pdhgc_get_iterates(pdhgc_lp* lp, double* x, double* y, double* x_avg, double* y_avg, int64_t* iters_out,
                       int on_device) {
  if (!lp || (on_device != 0 && on_device != 1)) return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = lp->stream;
  const int m = lp->m, n = lp->n;
  Scalars S;
  CK(cudaMemcpyAsync(&S, lp->S, sizeof(S), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double inv_t = S.t > 0 ? 1.0 / (double)S.t : 0.0;
  // after a Halpern-loop phase the second pair is the PDHG output T(z)
  const bool out = S.algorithm == PDHGC_ALG_HALPERN && lp->have_h;
  struct V {
    double* dst;
    const double* src;
    const int* perm;
    int len;
    double scale;
  } vs[4] = {{x, lp->it.x, lp->col_perm, n, 1.0},
             {y, lp->it.y, lp->row_perm, m, 1.0},
             {x_avg, out ? lp->hz.xp : lp->it.sum_x, lp->col_perm, n, out ? 1.0 : inv_t},
             {y_avg, out ? lp->hz.yp : lp->it.sum_y, lp->row_perm, m, out ? 1.0 : inv_t}};
  for (const V& v : vs) {
    if (!v.dst) continue;
    double* tmp = v.len == n ? lp->tmp_n : lp->tmp_m;
    if (v.len == n && v.len == m && v.perm == lp->row_perm) tmp = lp->tmp_m;
    k_unpermute<<<grid_for(v.len), 256, 0, st>>>(v.len, v.perm, v.src, nullptr, nullptr, tmp);
    lp->launches++;
    CKL();
    if (v.scale != 1.0) {
      k_fill_scaled<<<grid_for(v.len), 256, 0, st>>>(tmp, v.len, v.scale);
      lp->launches++;
      CKL();
    }
    RET(copy_out(lp, v.dst, tmp, v.len, on_device));
    CK(cudaStreamSynchronize(st));
  }
  if (iters_out) {
    iters_out[0] = S.k;
    iters_out[1] = S.t;
    iters_out[2] = S.restarts;
  }
  return PDHGC_OK;
}

int pdhgc_get_scaling(pdhgc_lp* lp, double* d_row, double* d_col, double* scalars, int on_device) {
  if (!lp || (on_device != 0 && on_device != 1)) return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = lp->stream;
  if (d_row) {
    k_unpermute<<<grid_for(lp->m), 256, 0, st>>>(lp->m, lp->row_perm, lp->Dr, nullptr, nullptr, lp->tmp_m);
    lp->launches++;
    CKL();
    RET(copy_out(lp, d_row, lp->tmp_m, lp->m, on_device));
  }
  if (d_col) {
    k_unpermute<<<grid_for(lp->n), 256, 0, st>>>(lp->n, lp->col_perm, lp->Dc, nullptr, nullptr, lp->tmp_n);
    lp->launches++;
    CKL();
    RET(copy_out(lp, d_col, lp->tmp_n, lp->n, on_device));
  }
  CK(cudaStreamSynchronize(st));
  if (scalars) {
    Scalars S;
    CK(cudaMemcpy(&S, lp->S, sizeof(S), cudaMemcpyDeviceToHost));
    const double v[5] = {S.sigma_max, S.eta, S.omega, S.tau, S.sigma};
    if (on_device) {
      CK(cudaMemcpy(scalars, v, sizeof(v), cudaMemcpyHostToDevice));
    } else {
      std::memcpy(scalars, v, sizeof(v));
    }
  }
  return PDHGC_OK;
}

int pdhgc_uniform(uint64_t seed, int64_t n, double obj_scale, double* out, void* cuda_stream) {
  if (n < 0 || (n > 0 && !out)) return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return PDHGC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_uniform<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((unsigned long long)seed, (long long)n, obj_scale, out);
  CKL();
  CK(cudaStreamSynchronize(st));
  return PDHGC_OK;
}

int pdhgc_probe_gather(int64_t n_vec, int64_t count, int32_t elem_bytes, int32_t reps, double* ms_out,
                       void* cuda_stream) {
  if (n_vec < 1 || count < 1 || (elem_bytes != 4 && elem_bytes != 8) || reps < 1 || !ms_out)
    return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  void* vec = nullptr;
  double* sink = nullptr;
  CK(cudaMalloc(&vec, (size_t)n_vec * elem_bytes));
  std::unique_ptr<void, void (*)(void*)> vg(vec, [](void* q) { cudaFree(q); });
  CK(cudaMalloc(&sink, sizeof(double)));
  std::unique_ptr<double, void (*)(double*)> sg(sink, [](double* q) { cudaFree(q); });
  CK(cudaMemsetAsync(vec, 0, (size_t)n_vec * elem_bytes, st));
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long loads = count * kGatherProbeScale;
  const long long per_block = 256LL * kGatherProbeBatch;
  long long grid = (loads + per_block - 1) / per_block;
  if (grid > (long long)sms * 8) grid = (long long)sms * 8;
  auto launch = [&]() {
    if (elem_bytes == 8)
      k_gather_probe<double><<<(unsigned)grid, 256, 0, st>>>(static_cast<const double*>(vec), n_vec, loads, sink);
    else
      k_gather_probe<float><<<(unsigned)grid, 256, 0, st>>>(static_cast<const float*>(vec), n_vec, loads, sink);
  };
  launch();  // warm: the vector into L2
  CKL();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) launch();
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CKL();
  *ms_out = (double)ms / reps / kGatherProbeScale;
  return PDHGC_OK;
}

int64_t pdhgc_kernel_launches(const pdhgc_lp* lp) { return lp ? lp->launches : 0; }

int pdhgc_set_primal_layout(pdhgc_lp* lp, int32_t chunked) {
  if (!lp || (chunked != 0 && chunked != 1)) return set_err(PDHGC_ERR_INVALID_ARG, "chunked must be 0 or 1");
  if (chunked && !lp->chunk_ready) {
    // the chunk plan is built on first use (lp_create leaves it out): from
    // A' as laid out on the device, then the slots take the scaled values the
    // last scaling left (each solve's scaling refills them)
    cudaStream_t st = lp->stream;
    Csr T;
    T.rows = lp->T.rows;
    T.cols = lp->m;
    T.nnz = lp->nnz;
    T.row_ptr.resize((size_t)T.rows + 1);
    T.col.resize((size_t)lp->nnz);
    CK(cudaMemcpyAsync(T.row_ptr.data(), lp->T.rp, T.row_ptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (lp->nnz > 0)
      CK(cudaMemcpyAsync(T.col.data(), lp->T.col, T.col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    RET(setup_chunked(lp, T, st));
    if (lp->ch64.nslots > 0) {
      k_sell_fill<<<grid_for(lp->ch64.nslots), 256, 0, st>>>(lp->ch64.map, lp->T.hat, lp->ch64.val64,
                                                            (int)lp->ch64.nslots);
      lp->launches++;
    }
    if (lp->have32 && lp->ch32.nslots > 0) {
      k_sell_fill<<<grid_for(lp->ch32.nslots), 256, 0, st>>>(lp->ch32.map, lp->T.hat32, lp->ch32.val32,
                                                            (int)lp->ch32.nslots);
      lp->launches++;
    }
    CKL();
    CK(cudaStreamSynchronize(st));
    lp->chunk_ready = true;
  }
  lp->chunked_primal = chunked;
  return PDHGC_OK;
}

int pdhgc_set_launch_mode(pdhgc_lp* lp, int32_t mode) {
  if (!lp || (mode != PDHGC_LAUNCH_GRAPH && mode != PDHGC_LAUNCH_STREAM))
    return set_err(PDHGC_ERR_INVALID_ARG, "mode must be PDHGC_LAUNCH_GRAPH or PDHGC_LAUNCH_STREAM");
  lp->launch_mode = mode;
  return PDHGC_OK;
}

int pdhgc_get_layout(const pdhgc_lp* lp, int64_t* out) {
  if (!lp || !out) return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  const pdhgc_lp::Mat* mats[2] = {&lp->A, &lp->T};
  for (int k = 0; k < 2; ++k) {
    out[4 * k + 0] = mats[k]->nb_cta;
    out[4 * k + 1] = mats[k]->nb_warp;
    out[4 * k + 2] = mats[k]->nb_sell;
    out[4 * k + 3] = mats[k]->cta_rows;
  }
  return PDHGC_OK;
}

int pdhgc_profile_iteration(pdhgc_lp* lp, int32_t iters, double* ms_out) {
  if (!lp || iters < 1 || !ms_out) return set_err(PDHGC_ERR_INVALID_ARG, "bad argument");
  if (!lp->have_phase1) return set_err(PDHGC_ERR_NO_PHASE1, "pdhgc_solve has not run");
  cudaStream_t st = lp->stream;
  const DevModel md = lp->have_corner ? model_corner(lp) : model_orig(lp);
  const bool fp32 = lp->params.precision == PDHGC_FP32_BULK;
  const bool halpern = lp->params.algorithm == PDHGC_ALG_HALPERN && lp->have_h;
  const bool unit_rho = lp->params.reflection == 1.0;  // the operator the loop launches
  const DevModel32 md32 = lp->have_corner ? model32_corner(lp) : model32_orig(lp);
  const DevIter32 it32{lp->it32.x,  lp->it32.y,   lp->it32.xbar, lp->it32.sx, lp->it32.sy,
                       lp->it32.xlo, lp->it32.ylo, lp->it32.xa,   lp->it32.ya};
  // the replay must not stop on the phase's done flag or iteration limit
  Scalars S;
  CK(cudaMemcpy(&S, lp->S, sizeof(S), cudaMemcpyDeviceToHost));
  const int saved_done = S.done;
  const long long saved_max = S.max_iters;
  const int zero = 0;
  const long long big = (long long)1 << 62;
  CK(cudaMemcpy(&lp->S->done, &zero, sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(&lp->S->max_iters, &big, sizeof(long long), cudaMemcpyHostToDevice));
  std::vector<cudaEvent_t> ev(3 * (size_t)iters);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  int rc = PDHGC_OK;
  for (int i = 0; i < iters && rc == PDHGC_OK; ++i) {
    CK(cudaEventRecord(ev[3 * i], st));
    // the Halpern loop's kernels as a step inside a chunk (it 0, not a check step)
    if (halpern && fp32)
      rc = unit_rho ? launch_primal(lp, PrimalOpH32T<true>{lp->S, 0, 1, 0, md32, h32_of(lp), lp->hz}, st, false)
                    : launch_primal(lp, PrimalOpH32{lp->S, 0, 1, 0, md32, h32_of(lp), lp->hz}, st, false);
    else if (halpern && unit_rho)
      rc = launch_primal(lp, PrimalOpHT<true>{lp->S, 0, 1, 0, lp->it.y, md, lp->it, lp->hz}, st, false);
    else if (halpern)
      rc = launch_primal(lp, PrimalOpH{lp->S, 0, 1, 0, lp->it.y, md, lp->it, lp->hz}, st, false);
    else if (fp32)
      rc = launch_tiles(lp, true, true, PrimalOp32{lp->S, 0, lp->it32.y, md32, it32}, nullptr, st);
    else
      rc = launch_tiles(lp, true, true, PrimalOp{lp->S, 0, lp->it.y, md, lp->it}, nullptr, st);
    if (rc != PDHGC_OK) break;
    CK(cudaEventRecord(ev[3 * i + 1], st));
    if (halpern && fp32)
      rc = launch_tiles(lp, false, true, DualOpH32{lp->S, 0, 1, 0, md32, h32_of(lp), lp->hz}, nullptr, st);
    else if (halpern && unit_rho)
      rc = launch_tiles(lp, false, true, DualOpHT<true>{lp->S, 0, 1, 0, lp->it.xbar, md, lp->it, lp->hz}, nullptr,
                        st);
    else if (halpern)
      rc = launch_tiles(lp, false, true, DualOpH{lp->S, 0, 1, 0, lp->it.xbar, md, lp->it, lp->hz}, nullptr, st);
    else if (fp32)
      rc = launch_tiles(lp, false, true, DualOp32{lp->S, 0, lp->it32.xbar, md32, it32}, nullptr, st);
    else
      rc = launch_tiles(lp, false, true, DualOp{lp->S, 0, lp->it.xbar, md, lp->it}, nullptr, st);
    if (rc != PDHGC_OK) break;
    CK(cudaEventRecord(ev[3 * i + 2], st));
  }
  CK(cudaStreamSynchronize(st));
  double tp = 0.0, td = 0.0;
  for (int i = 0; i < iters && rc == PDHGC_OK; ++i) {
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]));
    CK(cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]));
    tp += a;
    td += b;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  CK(cudaMemcpy(&lp->S->done, &saved_done, sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(&lp->S->max_iters, &saved_max, sizeof(long long), cudaMemcpyHostToDevice));
  if (rc != PDHGC_OK) return rc;
  ms_out[0] = tp / iters;
  ms_out[1] = td / iters;
  return PDHGC_OK;
}

void pdhgc_lp_destroy(pdhgc_lp* lp) {
  if (!lp) return;
  cudaStreamSynchronize(lp->stream);
  delete lp;
}

const char* pdhgc_strerror(int code) {
  switch (code) {
    case PDHGC_OK: return "ok";
    case PDHGC_ERR_INVALID_ARG: return "invalid argument";
    case PDHGC_ERR_INVALID_CSR: return "invalid CSR structure";
    case PDHGC_ERR_NONFINITE: return "non-finite input";
    case PDHGC_ERR_BOUNDS: return "lower bound above upper bound";
    case PDHGC_ERR_CUDA: return "CUDA error";
    case PDHGC_ERR_OOM: return "out of memory";
    case PDHGC_ERR_NO_PHASE1: return "no phase-1 solution";
    case PDHGC_ERR_NO_CORNER: return "no corner solution";
    case PDHGC_ERR_TOO_LARGE: return "problem too large";
    case PDHGC_ERR_DEVICE: return "device-side check failed";
    case PDHGC_ERR_BUFFER: return "buffer too small";
    case PDHGC_ERR_IO: return "file input/output error";
    default: return "unknown error";
  }
}

const char* pdhgc_last_error_detail(void) { return g_detail.c_str(); }

}  // extern "C"
