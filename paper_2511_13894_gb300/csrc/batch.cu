// Batched solve: many independent LPs in one persistent launch.
//
// A CTA takes LPs from a work queue (largest first) and runs the whole method
// on each one: Ruiz + Pock-Chambolle scaling, power iteration, restarted PDHG
// with its checks, restarts and termination, the report, and on request the
// corner phase of Algorithm 1.  Between the two matrix passes of an iteration
// only a CTA barrier is needed, and an LP's gathered vectors (x_bar and y)
// live in the CTA's shared memory, so the random gathers of the SpMV are
// shared-memory loads.  A finished LP drops out: its CTA pulls the next one.
// The arithmetic of every step is the same operator code as the single-LP
// path (kernels.cuh); only the scheduling differs.  Each phase is one CUDA
// graph (queue reset + the persistent kernel).  Tail handoff: once the queue
// is empty and only a few LPs still run, a long-running LP stops at its next
// check and the host finishes it on the single-LP path (whole-GPU graph
// loop), several concurrently on their own streams; the host watches the
// running kernel's report statuses and starts each handed-off LP at once,
// while the kernel finishes its other LPs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pdhgc.h"
#include "batch.h"
#include "batch_desc.h"
#include "host_prep.h"
#include "kkt_eval.h"

namespace pdhgc {

namespace {

template <class T>
int dalloc(std::vector<void*>& allocs, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (count > 0 ? count : 1) * sizeof(T));
  if (e != cudaSuccess) return PDHGC_ERR_OOM;
  allocs.push_back(q);
  *p = static_cast<T*>(q);
  return PDHGC_OK;
}

}  // namespace

}  // namespace pdhgc

using namespace pdhgc;

struct pdhgc_batch {
  int count = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<void*> allocs;
  std::vector<LpDesc> h_desc;
  std::vector<int> order;
  std::vector<std::vector<int32_t>> row_perm, col_perm;
  std::vector<std::vector<double>> sign;
  LpDesc* d_desc = nullptr;
  int* d_order = nullptr;
  int* d_queue = nullptr;
  BatchReport* d_rep = nullptr;
  BatchReport* d_rep2 = nullptr;  // corner reports of the fused call (pdhgc_batch_solve_corner)
  std::vector<BatchReport> h_rep1, h_repc;
  size_t smem_f32 = 0, smem_f64 = 0;
  int block = 1024;
  int have_phase1 = 0, have_corner = 0;
  int precision = PDHGC_FP32_BULK;
  pdhgc_params params{};
  double tune_ms[4] = {0, 0, 0, 0};
  cudaGraphExec_t gexec = nullptr;  // the last launched batch graph
  int64_t launches = 0;             // kernels launched (batched, and single-LP ones of handed-off LPs)
  int device = 0;
  // the caller's inputs, kept for the single-LP path of handed-off LPs
  struct HostLp {
    int32_t m = 0, n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> col;
    std::vector<double> val, b, c, lb, ub;
    std::vector<int8_t> sense;
  };
  std::vector<HostLp> host;
  int handoff_running = 8;
  long long handoff_min_iters = 8192;
  std::vector<pdhgc_report> ext_rep1, ext_repc;  // reports of handed-off LPs
  std::vector<char> ext1, extc;                  // 1: that phase's result came from the single-LP path
  // watching the running batched kernel for handoffs: a stream for the status
  // copies, pinned host statuses (2 x count), events around the kernel
  cudaStream_t poll_stream = nullptr;
  int32_t* h_stat = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  ~pdhgc_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (void* q : allocs) cudaFree(q);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (poll_stream) cudaStreamDestroy(poll_stream);
    if (h_stat) cudaFreeHost(h_stat);
    if (ev_start) cudaEventDestroy(ev_start);
    if (ev_done) cudaEventDestroy(ev_done);
  }
};

namespace {

int set_berr(int code, const std::string& s) { return pdhgc::set_error_detail(code, s); }

#define RET(x)                     \
  do {                             \
    const int r_ = (x);            \
    if (r_ != PDHGC_OK) return r_; \
  } while (0)

#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_berr(e_ == cudaErrorMemoryAllocation ? PDHGC_ERR_OOM : PDHGC_ERR_CUDA,   \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

// lanes per row from the mean row length (a starting point the tuner refines)
int lanes_for(double mean_len) {
  int g = 1;
  while (g < 32 && g * 4 < mean_len) g <<= 1;
  return g;
}

constexpr size_t kSmemBudget = 200 * 1024;

BatchParams make_params(const pdhgc_params& p, const pdhgc_corner_params* cp) {
  BatchParams b{};
  b.eps_rel = p.eps_rel;
  b.beta_suff = p.beta_suff;
  b.beta_nec = p.beta_nec;
  b.beta_art = p.beta_art;
  b.theta = p.theta;
  b.eta_factor = p.eta_factor;
  b.time_limit_s = p.time_limit_s;
  b.max_iters = p.max_iters;
  b.check_period = p.check_period;
  b.ruiz_iters = p.ruiz_iters;
  b.power_iters = p.power_iters;
  b.algorithm = p.algorithm;
  b.rho = p.reflection;
  b.pid_kp = p.pid_kp;
  b.pid_ki = p.pid_ki;
  b.pid_kd = p.pid_kd;
  if (cp) {
    b.eps_abs = cp->eps_abs;
    b.c_eps_rel = cp->eps_rel;
    b.obj_scale = cp->obj_scale;
    b.c_time_limit_s = cp->time_limit_s;
    b.c_min_iters = cp->min_iters;
    b.c_max_iters = cp->max_iters;
    b.obj_seed = cp->obj_seed;
    b.stop_rule = cp->stop_rule;
    b.row_rule = cp->row_rule;
  }
  return b;
}

template <class VT, int BT>
int launch_batch(pdhgc_batch* B, const BatchParams& bp, int phase, cudaStream_t st) {
  const size_t smem = std::is_same<VT, float>::value ? B->smem_f32 : B->smem_f64;
  int dev = 0, sms = 0, per_sm = 0;
  BCK((batch_kernel_prepare<VT, BT>(smem, &per_sm)));
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return set_berr(PDHGC_ERR_CUDA, "batched kernel does not fit on an SM");
  int grid = sms * per_sm;
  if (grid > B->count) grid = B->count;
  // one CUDA graph: the queue reset and the persistent kernel, captured on the
  // batch's private stream and launched on the caller's stream
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
  const cudaError_t me = cudaMemsetAsync(B->d_queue, 0, 2 * sizeof(int), B->cap_stream);
  const cudaError_t le = batch_kernel_launch<VT, BT>(grid, smem, B->cap_stream, B->d_desc, B->d_order, B->count,
                                                      B->d_queue, bp, phase, B->d_rep, B->d_rep2);
  const cudaError_t ce = cudaStreamEndCapture(B->cap_stream, &graph);
  if (me != cudaSuccess || le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    const cudaError_t e = me != cudaSuccess ? me : (le != cudaSuccess ? le : ce);
    return set_berr(PDHGC_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  }
  // the previous executable graph is freed once its launch completes
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  B->gexec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&B->gexec, graph, 0);
  cudaGraphDestroy(graph);
  BCK(ie);
  BCK(cudaGraphLaunch(B->gexec, st));
  B->launches++;
  return PDHGC_OK;
}

int run_batch(pdhgc_batch* B, const BatchParams& bp, int phase, cudaStream_t st) {
  const bool f32 = B->precision == PDHGC_FP32_BULK;
  if (B->block == 512) return f32 ? launch_batch<float, 512>(B, bp, phase, st) : launch_batch<double, 512>(B, bp, phase, st);
  return f32 ? launch_batch<float, 1024>(B, bp, phase, st) : launch_batch<double, 1024>(B, bp, phase, st);
}

void to_report(const BatchReport& r, int64_t m, double nb, double nc, int precision, pdhgc_report* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = r.status;
  out->chosen = r.chosen;
  out->iters = r.iters;
  out->restarts = r.restarts;
  out->rP2 = r.rP2;
  out->rD2 = r.rD2;
  out->rPinf = r.rPinf;
  out->rDinf = r.rDinf;
  out->pobj = r.pobj;
  out->dobj = r.dobj;
  out->gap = r.pobj - r.dobj;
  out->rel_p = r.rP2 / (1.0 + nb);
  out->rel_d = r.rD2 / (1.0 + nc);
  out->rel_gap = std::fabs(out->gap) / (1.0 + std::fabs(r.pobj) + std::fabs(r.dobj));
  out->rel_kkt = std::fmax(out->rel_p, std::fmax(out->rel_d, out->rel_gap));
  out->off_bound_p = (int64_t)std::llround(r.p);
  out->zero_rc_d = (int64_t)std::llround(r.dd);
  out->candidates = (int64_t)std::llround(r.cand);
  out->corner_measure = out->candidates > m ? out->candidates - m : 0;
  out->primal_push_est = out->off_bound_p > m ? out->off_bound_p - m : 0;
  out->dual_push_est = m > out->zero_rc_d ? m - out->zero_rc_d : 0;
  const int64_t thr = 2 * m > 100000 ? 2 * m : 100000;
  out->should_corner = out->candidates >= thr ? 1 : 0;
  out->precision = precision;
  out->seconds = r.seconds;
  out->omega = r.omega;
  out->eta = r.eta;
  out->sigma_max = r.sigma_max;
}

// One handed-off LP on the single-LP path (its own stream and handle, run
// from a host thread so that several run concurrently).  mode 0: phase 1;
// 1: the corner phase (phase 1 runs first on that handle, and the corner
// phase starts from that handle's own phase-1 result); 2: both, each result
// kept.  The results go back into the batch's scaled internal buffers.
int finish_on_single_path(pdhgc_batch* B, int k, int mode, const pdhgc_params& p, const pdhgc_corner_params* cp,
                          std::string& err, int64_t& launches) {
  BCK(cudaSetDevice(B->device));
  cudaStream_t st = nullptr;
  BCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  const auto& h = B->host[k];
  pdhgc_lp* lp = nullptr;
  int rc = pdhgc_lp_create(&lp, h.m, h.n, (int64_t)h.col.size(), h.rp.data(), h.col.data(), h.val.data(),
                           h.b.data(), h.c.data(), h.lb.empty() ? nullptr : h.lb.data(),
                           h.ub.empty() ? nullptr : h.ub.data(), h.sense.empty() ? nullptr : h.sense.data(), 0, st);
  pdhgc_report r1{}, rc_rep{};
  std::vector<double> x1(h.n), y1(h.m), xc(h.n), yc(h.m);
  if (rc == PDHGC_OK) rc = pdhgc_solve(lp, &p, &r1);
  if (rc == PDHGC_OK && mode != 1) rc = pdhgc_get_solution(lp, PDHGC_PHASE1, x1.data(), y1.data(), nullptr, 0);
  if (rc == PDHGC_OK && mode != 0) rc = pdhgc_corner_phase(lp, cp, &rc_rep);
  if (rc == PDHGC_OK && mode != 0) rc = pdhgc_get_solution(lp, PDHGC_CORNER, xc.data(), yc.data(), nullptr, 0);
  if (rc != PDHGC_OK) err = std::string("handoff of LP ") + std::to_string(k) + ": " + pdhgc_last_error_detail();
  if (lp) {
    launches = pdhgc_kernel_launches(lp);
    pdhgc_lp_destroy(lp);
  }
  if (rc == PDHGC_OK) {
    const LpDesc& d = B->h_desc[k];
    std::vector<double> Dc(d.n), Dr(d.m), x1h(d.n), y1h(d.m), xch(d.n);
    cudaError_t e = cudaMemcpyAsync(Dc.data(), d.Dc, (size_t)d.n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Dr.data(), d.Dr, (size_t)d.m * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && mode != 1) {
      for (int j = 0; j < d.n; ++j) x1h[j] = x1[B->col_perm[k][j]] / Dc[j];
      for (int i = 0; i < d.m; ++i) y1h[i] = B->sign[k][i] * y1[B->row_perm[k][i]] / Dr[i];
      e = cudaMemcpyAsync(d.x1, x1h.data(), (size_t)d.n * 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d.y1, y1h.data(), (size_t)d.m * 8, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess && mode != 0) {
      for (int j = 0; j < d.n; ++j) xch[j] = xc[B->col_perm[k][j]] / Dc[j];
      e = cudaMemcpyAsync(d.xc, xch.data(), (size_t)d.n * 8, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = PDHGC_ERR_CUDA;
      err = std::string("handoff copy-back: ") + cudaGetErrorString(e);
    } else {
      if (mode != 1) {
        B->ext_rep1[k] = r1;
        B->ext1[k] = 1;
      }
      if (mode != 0) {
        B->ext_repc[k] = rc_rep;
        B->extc[k] = 1;
      }
    }
  }
  cudaStreamDestroy(st);
  return rc;
}

// Runs a batched phase and finishes the LPs it hands off on the single-LP
// path, each from its own host thread and stream.  While the batched kernel
// runs, the host copies the LPs' statuses (a strided copy of the status
// field of the device reports, on a stream of its own) every few hundred
// microseconds and starts a worker as soon as an LP shows the handoff
// status, so that the handed-off LPs run while the batched kernel finishes
// its other LPs, on the SMs its exited CTAs leave free.  phase 0 or 1: that
// phase's handoffs; 2 (the fused call): an LP handed off in phase 1 runs
// both phases on the single-LP path, one handed off in its corner phase runs
// the corner phase there (mode 1).  The reports are copied to h_rep1 /
// h_repc when the kernel has finished.
int run_batch_and_handoffs(pdhgc_batch* B, const BatchParams& bp, int phase, cudaStream_t st, const pdhgc_params& p,
                           const pdhgc_corner_params* cp) {
  const int count = B->count;
  if (!B->poll_stream) BCK(cudaStreamCreateWithFlags(&B->poll_stream, cudaStreamNonBlocking));
  if (!B->h_stat) BCK(cudaMallocHost(&B->h_stat, 2 * (size_t)count * sizeof(int32_t)));
  if (!B->ev_start) BCK(cudaEventCreateWithFlags(&B->ev_start, cudaEventDisableTiming));
  if (!B->ev_done) BCK(cudaEventCreateWithFlags(&B->ev_done, cudaEventDisableTiming));
  // statuses start at 0 (NONE): a report of an earlier call never reads as a handoff
  BCK(cudaMemsetAsync(B->d_rep, 0, count * sizeof(BatchReport), st));
  BCK(cudaMemsetAsync(B->d_rep2, 0, count * sizeof(BatchReport), st));
  BCK(cudaEventRecord(B->ev_start, st));
  RET(run_batch(B, bp, phase, st));
  BCK(cudaEventRecord(B->ev_done, st));
  BCK(cudaStreamWaitEvent(B->poll_stream, B->ev_start, 0));
  std::vector<int> ks, modes;
  std::vector<char> started(count, 0);
  std::vector<int> rcs(count, PDHGC_OK);
  std::vector<std::string> errs(count);
  std::vector<int64_t> lcount(count, 0);
  std::vector<std::thread> th;
  int rc = PDHGC_OK;
  // the handoff mode of LP k from the statuses s1 (phase 1 or the phase run)
  // and s2 (corner, fused call), or -1
  auto mode_of = [&](int32_t s1, int32_t s2) {
    if (phase != 2) return s1 == kStatusHandoff ? phase : -1;
    if (s1 == kStatusHandoff) return 2;
    if (s2 == kStatusHandoff && s1 != 0) return 1;  // phase 1 finished in the batch
    return -1;
  };
  auto start = [&](int k, int mode) {
    started[k] = 1;
    ks.push_back(k);
    modes.push_back(mode);
    try {
      th.emplace_back([&, k, mode] { rcs[k] = finish_on_single_path(B, k, mode, p, cp, errs[k], lcount[k]); });
    } catch (...) {
      rcs[k] = finish_on_single_path(B, k, mode, p, cp, errs[k], lcount[k]);  // no thread: finish it here
    }
  };
  for (;;) {
    const cudaError_t q = cudaEventQuery(B->ev_done);
    if (q != cudaSuccess && q != cudaErrorNotReady) {
      rc = set_berr(PDHGC_ERR_CUDA, std::string("batched kernel: ") + cudaGetErrorString(q));
      break;
    }
    if (q == cudaSuccess) break;
    cudaError_t e = cudaMemcpy2DAsync(B->h_stat, sizeof(int32_t), B->d_rep, sizeof(BatchReport), sizeof(int32_t),
                                      count, cudaMemcpyDeviceToHost, B->poll_stream);
    if (e == cudaSuccess && phase == 2)
      e = cudaMemcpy2DAsync(B->h_stat + count, sizeof(int32_t), B->d_rep2, sizeof(BatchReport), sizeof(int32_t),
                            count, cudaMemcpyDeviceToHost, B->poll_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->poll_stream);
    if (e != cudaSuccess) {
      rc = set_berr(PDHGC_ERR_CUDA, std::string("handoff status copy: ") + cudaGetErrorString(e));
      break;
    }
    for (int k = 0; k < count; ++k) {
      if (started[k]) continue;
      const int mode = mode_of(B->h_stat[k], phase == 2 ? B->h_stat[count + k] : 0);
      if (mode >= 0) start(k, mode);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(300));
  }
  // the kernel has finished (or failed): the final reports, and any handoff
  // the last status copy had not seen yet.  After a failed status copy the
  // batch's stream is still drained, so that no kernel of this call outlives it.
  if (rc != PDHGC_OK) cudaStreamSynchronize(st);
  if (rc == PDHGC_OK) {
    cudaError_t e = cudaMemcpyAsync((phase == 1 ? B->h_repc : B->h_rep1).data(), B->d_rep,
                                    count * sizeof(BatchReport), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && phase == 2)
      e = cudaMemcpyAsync(B->h_repc.data(), B->d_rep2, count * sizeof(BatchReport), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = set_berr(PDHGC_ERR_CUDA, std::string("report copy: ") + cudaGetErrorString(e));
  }
  if (rc == PDHGC_OK) {
    const std::vector<BatchReport>& r1 = phase == 1 ? B->h_repc : B->h_rep1;
    for (int k = 0; k < count; ++k) {
      if (started[k]) continue;
      const int mode = mode_of(r1[k].status, phase == 2 ? B->h_repc[k].status : 0);
      if (mode >= 0) start(k, mode);
    }
  }
  for (auto& t : th) t.join();
  for (int k : ks) B->launches += lcount[k];
  if (rc != PDHGC_OK) return rc;
  for (int k : ks)
    if (rcs[k] != PDHGC_OK) return set_berr(rcs[k], errs[k]);
  return PDHGC_OK;
}

}  // namespace

extern "C" {

int pdhgc_batch_create(pdhgc_batch** out, int32_t count, const int32_t* m, const int32_t* n, const int64_t* nnz,
                       const int64_t* const* row_ptr, const int32_t* const* col_idx, const double* const* val,
                       const double* const* b, const double* const* c, const double* const* lb,
                       const double* const* ub, const int8_t* const* sense, void* cuda_stream) {
  if (!out || count < 1 || !m || !n || !nnz || !row_ptr || !col_idx || !val || !b || !c)
    return set_berr(PDHGC_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  std::unique_ptr<pdhgc_batch> B(new pdhgc_batch());
  B->count = count;
  B->stream = static_cast<cudaStream_t>(cuda_stream);
  std::vector<Prepared> P(count);
  int64_t sm = 0, sn = 0, snz = 0;
  BCK(cudaGetDevice(&B->device));
  B->host.resize(count);
  // the LPs are independent: validated and laid out on several host threads
  // (each writes only its LPs' slots), errors reported for the first bad LP
  std::vector<int> prc(count, PDHGC_OK);
  std::vector<std::string> pdetail(count);
  auto prepare_one = [&](int k) {
    prc[k] = prepare_lp(P[k], m[k], n[k], nnz[k], row_ptr[k], col_idx[k], val[k], b[k], c[k], lb ? lb[k] : nullptr,
                        ub ? ub[k] : nullptr, sense ? sense[k] : nullptr, pdetail[k]);
    if (prc[k] != PDHGC_OK) return;
    auto& h = B->host[k];
    h.m = m[k];
    h.n = n[k];
    h.rp.assign(row_ptr[k], row_ptr[k] + m[k] + 1);
    h.col.assign(col_idx[k], col_idx[k] + nnz[k]);
    h.val.assign(val[k], val[k] + nnz[k]);
    h.b.assign(b[k], b[k] + m[k]);
    h.c.assign(c[k], c[k] + n[k]);
    if (lb && lb[k]) h.lb.assign(lb[k], lb[k] + n[k]);
    if (ub && ub[k]) h.ub.assign(ub[k], ub[k] + n[k]);
    if (sense && sense[k]) h.sense.assign(sense[k], sense[k] + m[k]);
  };
  {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = std::max(1, std::min(count, (int)std::min(hw == 0 ? 1u : hw, 16u)));
    std::vector<std::thread> pth;
    int started = 0;
    try {
      for (; started < nt - 1; ++started)
        pth.emplace_back([&, started] {
          for (int k = started + 1; k < count; k += nt) prepare_one(k);
        });
    } catch (...) {
      // no more threads: this thread takes the remaining strides
    }
    for (int t = started + 1; t < nt; ++t)
      for (int k = t; k < count; k += nt) prepare_one(k);
    for (int k = 0; k < count; k += nt) prepare_one(k);
    for (auto& t : pth) t.join();
  }
  for (int k = 0; k < count; ++k) {
    if (prc[k] != PDHGC_OK) return set_berr(prc[k], "LP " + std::to_string(k) + ": " + pdetail[k]);
    sm += m[k];
    sn += n[k];
    snz += nnz[k];
  }
  if (snz >= (int64_t(1) << 31)) return set_berr(PDHGC_ERR_TOO_LARGE, "total nnz must be < 2^31");
  auto& A = B->allocs;
  // packed arrays
  int *rpA, *colA, *rpT, *colT, *rperm, *cperm;
  double *valA, *valT, *hatA, *hatT;
  float *hatA32, *hatT32;
  const size_t M = (size_t)sm, N = (size_t)sn, NZ = (size_t)snz, K = (size_t)count;
  int rc = PDHGC_OK;
#define BAL(p, cnt)                                   \
  do {                                                \
    rc = dalloc(A, &p, cnt);                          \
    if (rc != PDHGC_OK) return set_berr(rc, "cudaMalloc failed"); \
  } while (0)
  BAL(rpA, M + K);
  BAL(colA, NZ);
  BAL(rpT, N + K);
  BAL(colT, NZ);
  BAL(rperm, M);
  BAL(cperm, N);
  BAL(valA, NZ);
  BAL(valT, NZ);
  BAL(hatA, NZ);
  BAL(hatT, NZ);
  BAL(hatA32, NZ);
  BAL(hatT32, NZ);
  size_t SA = 0, ST = 0, SNA = 0, SNT = 0;  // SELL slots and slices of A and A'
  for (int k = 0; k < count; ++k) {
    SA += P[k].A.sell_map.size();
    ST += P[k].AT.sell_map.size();
    SNA += P[k].A.nslices;
    SNT += P[k].AT.nslices;
  }
  int *sptrA, *swA, *scolA, *smapA, *sptrT, *swT, *scolT, *smapT;
  double *svalA, *svalT, *shatA, *shatT;
  float *shatA32, *shatT32;
  BAL(sptrA, SNA + K); BAL(swA, SNA + 1); BAL(scolA, SA + kPad); BAL(smapA, SA + 1);
  BAL(sptrT, SNT + K); BAL(swT, SNT + 1); BAL(scolT, ST + kPad); BAL(smapT, ST + 1);
  BAL(svalA, SA + kPad); BAL(svalT, ST + kPad); BAL(shatA, SA + kPad); BAL(shatT, ST + kPad);
  BAL(shatA32, SA + kPad); BAL(shatT32, ST + kPad);
  double *b_int, *cc, *l, *u, *Dr, *Dc, *rfac, *cfac, *bhat, *chat, *lhat, *uhat, *chat_c, *lhat_c, *uhat_c;
  double *x, *xbar, *sum_x, *x_r, *y, *sum_y, *y_r, *x1, *y1, *xc, *pi_v, *pi_w, *pi_u;
  float *bhat32, *chat32, *lhat32, *uhat32, *chat_c32, *lhat_c32, *uhat_c32, *x32, *xbar32, *y32, *x32lo, *y32lo;
  float2 *sx32, *sy32;
  int8_t *ge, *ge_c;
  BAL(b_int, M); BAL(cc, N); BAL(l, N); BAL(u, N); BAL(Dr, M); BAL(Dc, N); BAL(rfac, M); BAL(cfac, N);
  BAL(bhat, M); BAL(chat, N); BAL(lhat, N); BAL(uhat, N); BAL(chat_c, N); BAL(lhat_c, N); BAL(uhat_c, N);
  BAL(x, N); BAL(xbar, N); BAL(sum_x, N); BAL(x_r, N); BAL(y, M); BAL(sum_y, M); BAL(y_r, M);
  BAL(x1, N); BAL(y1, M); BAL(xc, N); BAL(pi_v, N); BAL(pi_w, N); BAL(pi_u, M);
  double* keep;
  BAL(keep, 4 * K);
  BAL(bhat32, M); BAL(chat32, N); BAL(lhat32, N); BAL(uhat32, N); BAL(chat_c32, N); BAL(lhat_c32, N);
  BAL(uhat_c32, N); BAL(x32, N); BAL(xbar32, N); BAL(y32, M); BAL(x32lo, N); BAL(y32lo, M);
  BAL(sx32, N); BAL(sy32, M);
  BAL(ge, M); BAL(ge_c, M);
  double *hxp, *hyp, *hdx, *hdy, *hw;
  float* hs;
  float2 *xa32, *ya32;
  BAL(hxp, N); BAL(hyp, M); BAL(hdx, N); BAL(hdy, M); BAL(xa32, N); BAL(ya32, M);
  BAL(hw, 4096 * K); BAL(hs, 4096 * K);
  float* yh32;
  float2 *q32, *r032;
  BAL(yh32, M); BAL(q32, N); BAL(r032, M);
  BAL(B->d_desc, K);
  BAL(B->d_order, K);
  BAL(B->d_queue, 2);
  BAL(B->d_rep, K);
  BAL(B->d_rep2, K);
#undef BAL
  cudaStream_t st = B->stream;
  B->h_desc.resize(count);
  B->row_perm.resize(count);
  B->col_perm.resize(count);
  B->sign.resize(count);
  size_t om = 0, on = 0, onz = 0, orA = 0, orT = 0;
  size_t osA = 0, osT = 0, onsA = 0, onsT = 0;  // SELL slot and slice offsets
  size_t max_f32 = 0, max_f64 = 0;
  for (int k = 0; k < count; ++k) {
    const Prepared& Q = P[k];
    LpDesc& d = B->h_desc[k];
    std::memset(&d, 0, sizeof(d));
    d.m = Q.m;
    d.n = Q.n;
    d.nnz = (int)Q.nnz;
    d.gA = lanes_for(Q.m ? (double)Q.nnz / Q.m : 1.0);
    d.gT = lanes_for(Q.n ? (double)Q.nnz / Q.n : 1.0);
    d.sell = 0;  // CSR rows; pdhgc_batch_tune may switch to SELL-32
    d.b_norm = Q.b_norm;
    d.c_norm = Q.c_norm;
    const size_t v32 = (size_t)(Q.m + Q.n) * 4, v64 = (size_t)(Q.m + Q.n) * 8;
    d.smem = v64 <= kSmemBudget ? 1 : 0;  // FP64 decides; an FP32 run also fits then
    if (d.smem) {
      max_f32 = std::max(max_f32, v32);
      max_f64 = std::max(max_f64, v64);
    }
    d.A_rp = rpA + orA;
    d.A_col = colA + onz;
    d.T_rp = rpT + orT;
    d.T_col = colT + onz;
    d.A_val = valA + onz;
    d.T_val = valT + onz;
    d.A_hat = hatA + onz;
    d.T_hat = hatT + onz;
    d.A_hat32 = hatA32 + onz;
    d.T_hat32 = hatT32 + onz;
    d.b_int = b_int + om;
    d.c = cc + on;
    d.l = l + on;
    d.u = u + on;
    d.ge = ge + om;
    d.ge_c = ge_c + om;
    d.Dr = Dr + om; d.Dc = Dc + on; d.rfac = rfac + om; d.cfac = cfac + on;
    d.bhat = bhat + om; d.chat = chat + on; d.lhat = lhat + on; d.uhat = uhat + on;
    d.chat_c = chat_c + on; d.lhat_c = lhat_c + on; d.uhat_c = uhat_c + on;
    d.bhat32 = bhat32 + om; d.chat32 = chat32 + on; d.lhat32 = lhat32 + on; d.uhat32 = uhat32 + on;
    d.chat_c32 = chat_c32 + on; d.lhat_c32 = lhat_c32 + on; d.uhat_c32 = uhat_c32 + on;
    d.x = x + on; d.xbar = xbar + on; d.sum_x = sum_x + on; d.x_r = x_r + on;
    d.y = y + om; d.sum_y = sum_y + om; d.y_r = y_r + om;
    d.x32 = x32 + on; d.xbar32 = xbar32 + on; d.y32 = y32 + om;
    d.x32lo = x32lo + on; d.y32lo = y32lo + om;
    d.sx32 = sx32 + on; d.sy32 = sy32 + om;
    d.x1 = x1 + on; d.y1 = y1 + om; d.xc = xc + on;
    d.pi_v = pi_v + on; d.pi_w = pi_w + on; d.pi_u = pi_u + om;
    d.keep = keep + 4 * (size_t)k;
    d.hxp = hxp + on; d.hdx = hdx + on; d.hyp = hyp + om; d.hdy = hdy + om;
    d.xa32 = xa32 + on; d.ya32 = ya32 + om;
    d.yh32 = yh32 + om; d.q32 = q32 + on; d.r032 = r032 + om;
    d.hw = hw + 4096 * (size_t)k;
    d.hs = hs + 4096 * (size_t)k;
    d.row_perm = rperm + om;
    d.col_perm = cperm + on;
    // SELL-32 copies (indices and original values filled here from the slot map)
    for (int which = 0; which < 2; ++which) {
      const Csr& C = which ? Q.AT : Q.A;
      const size_t os = which ? osT : osA, ons = which ? onsT : onsA;
      int* sptr = (which ? sptrT : sptrA) + ons + k;  // nslices + 1 per LP
      int* sw = (which ? swT : swA) + ons;
      int* scol = (which ? scolT : scolA) + os;
      int* smap = (which ? smapT : smapA) + os;
      double* sval = (which ? svalT : svalA) + os;
      const size_t slots = C.sell_map.size();
      std::vector<int32_t> hc(slots);
      std::vector<double> hv(slots);
      for (size_t t = 0; t < slots; ++t) {
        const int32_t e = C.sell_map[t];
        hc[t] = e >= 0 ? C.col[e] : 0;
        hv[t] = e >= 0 ? C.val[e] : 0.0;
      }
      BCK(cudaMemcpyAsync(sptr, C.slice_ptr.data(), (C.nslices + 1) * 4, cudaMemcpyHostToDevice, st));
      if (C.nslices) BCK(cudaMemcpyAsync(sw, C.slice_w.data(), (size_t)C.nslices * 4, cudaMemcpyHostToDevice, st));
      if (slots) {
        BCK(cudaMemcpyAsync(scol, hc.data(), slots * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(smap, C.sell_map.data(), slots * 4, cudaMemcpyHostToDevice, st));
        BCK(cudaMemcpyAsync(sval, hv.data(), slots * 8, cudaMemcpyHostToDevice, st));
        BCK(cudaStreamSynchronize(st));  // the host staging vectors go out of scope
      }
      if (which) {
        d.T_long = C.long_rows; d.T_ns = C.nslices; d.T_slots = (int)slots;
        d.T_sptr = sptr; d.T_sw = sw; d.T_scol = scol; d.T_smap = smap; d.T_sval = sval;
        d.T_shat = shatT + os; d.T_shat32 = shatT32 + os;
      } else {
        d.A_long = C.long_rows; d.A_ns = C.nslices; d.A_slots = (int)slots;
        d.A_sptr = sptr; d.A_sw = sw; d.A_scol = scol; d.A_smap = smap; d.A_sval = sval;
        d.A_shat = shatA + os; d.A_shat32 = shatA32 + os;
      }
    }
    const size_t nz = (size_t)Q.nnz;
    BCK(cudaMemcpyAsync((void*)d.A_rp, Q.A.row_ptr.data(), (Q.m + 1) * 4, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.T_rp, Q.AT.row_ptr.data(), ((size_t)Q.n + 1) * 4, cudaMemcpyHostToDevice, st));
    if (nz) {
      BCK(cudaMemcpyAsync((void*)d.A_col, Q.A.col.data(), nz * 4, cudaMemcpyHostToDevice, st));
      BCK(cudaMemcpyAsync((void*)d.T_col, Q.AT.col.data(), nz * 4, cudaMemcpyHostToDevice, st));
      BCK(cudaMemcpyAsync((void*)d.A_val, Q.A.val.data(), nz * 8, cudaMemcpyHostToDevice, st));
      BCK(cudaMemcpyAsync((void*)d.T_val, Q.AT.val.data(), nz * 8, cudaMemcpyHostToDevice, st));
    }
    BCK(cudaMemcpyAsync((void*)d.b_int, Q.b_int.data(), (size_t)Q.m * 8, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.c, Q.c.data(), (size_t)Q.n * 8, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.l, Q.l.data(), (size_t)Q.n * 8, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.u, Q.u.data(), (size_t)Q.n * 8, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.ge, Q.ge.data(), (size_t)Q.m, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.row_perm, Q.row_perm.data(), (size_t)Q.m * 4, cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync((void*)d.col_perm, Q.col_perm.data(), (size_t)Q.n * 4, cudaMemcpyHostToDevice, st));
    B->row_perm[k] = Q.row_perm;
    B->col_perm[k] = Q.col_perm;
    B->sign[k] = Q.sign;
    om += Q.m;
    on += Q.n;
    onz += nz;
    osA += Q.A.sell_map.size();
    osT += Q.AT.sell_map.size();
    onsA += Q.A.nslices;
    onsT += Q.AT.nslices;
    orA += Q.m + 1;
    orT += Q.n + 1;
  }
  B->smem_f32 = std::max<size_t>(max_f32, 16);
  B->smem_f64 = std::max<size_t>(max_f64, 16);
  // largest LPs first
  B->order.resize(count);
  std::iota(B->order.begin(), B->order.end(), 0);
  std::stable_sort(B->order.begin(), B->order.end(),
                   [&](int a, int b2) { return P[a].nnz + P[a].n > P[b2].nnz + P[b2].n; });
  BCK(cudaMemcpyAsync(B->d_desc, B->h_desc.data(), K * sizeof(LpDesc), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(B->d_order, B->order.data(), K * sizeof(int), cudaMemcpyHostToDevice, st));
  BCK(cudaStreamSynchronize(st));
  BCK(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
  B->h_rep1.resize(count);
  B->h_repc.resize(count);
  B->ext_rep1.resize(count);
  B->ext_repc.resize(count);
  B->ext1.assign(count, 0);
  B->extc.assign(count, 0);
  pdhgc_default_params(&B->params);
  *out = B.release();
  return PDHGC_OK;
}

}  // extern "C"

namespace {

int check_batch_params(const pdhgc_params& p) {
  if (p.max_iters < 1 || p.check_period < 1 || p.check_period > 4096 || p.ruiz_iters < 0 || p.power_iters < 1 ||
      !(p.eta_factor > 0.0 && p.eta_factor < 1.0) || !(p.time_limit_s > 0.0) ||
      (p.precision != PDHGC_FP64 && p.precision != PDHGC_FP32_BULK))
    return set_berr(PDHGC_ERR_INVALID_ARG, "parameter out of range");
  if (p.algorithm != PDHGC_ALG_AVERAGED && p.algorithm != PDHGC_ALG_HALPERN)
    return set_berr(PDHGC_ERR_INVALID_ARG, "algorithm must be PDHGC_ALG_AVERAGED or PDHGC_ALG_HALPERN");
  if (p.algorithm == PDHGC_ALG_HALPERN &&
      (!(p.reflection >= 0.0 && p.reflection <= 1.0) || !std::isfinite(p.pid_kp) || !std::isfinite(p.pid_ki) ||
       !std::isfinite(p.pid_kd)))
    return set_berr(PDHGC_ERR_INVALID_ARG, "reflection must lie in [0, 1] and the PID gains be finite");
  return PDHGC_OK;
}

int check_batch_corner_params(const pdhgc_corner_params& cp) {
  if (!(cp.eps_abs >= 0.0) || cp.min_iters < 0 || cp.max_iters < 1 || !(cp.time_limit_s > 0.0) ||
      !std::isfinite(cp.obj_scale) || (cp.stop_rule != 0 && cp.stop_rule != 1) ||
      (cp.row_rule != 0 && cp.row_rule != 1))
    return set_berr(PDHGC_ERR_INVALID_ARG, "corner parameter out of range");
  if (cp.omega_rule != 0)
    return set_berr(PDHGC_ERR_INVALID_ARG, "the batched corner phase starts omega from the corner objective only");
  return PDHGC_OK;
}

void fill_reports(pdhgc_batch* B, int which, pdhgc_report* reports) {
  if (!reports) return;
  const std::vector<BatchReport>& h = which ? B->h_repc : B->h_rep1;
  const std::vector<char>& ext = which ? B->extc : B->ext1;
  const std::vector<pdhgc_report>& er = which ? B->ext_repc : B->ext_rep1;
  for (int k = 0; k < B->count; ++k) {
    if (ext[k])
      reports[k] = er[k];
    else
      to_report(h[k], B->h_desc[k].m, B->h_desc[k].b_norm, B->h_desc[k].c_norm, B->precision, &reports[k]);
  }
}

}  // namespace

extern "C" {

int pdhgc_batch_solve(pdhgc_batch* B, const pdhgc_params* params, pdhgc_report* reports) {
  if (!B) return set_berr(PDHGC_ERR_INVALID_ARG, "batch is NULL");
  pdhgc_params p;
  if (params) p = *params; else pdhgc_default_params(&p);
  RET(check_batch_params(p));
  B->params = p;
  B->precision = p.precision;
  B->have_phase1 = 0;
  B->have_corner = 0;
  std::fill(B->ext1.begin(), B->ext1.end(), 0);
  std::fill(B->extc.begin(), B->extc.end(), 0);
  cudaStream_t st = B->stream;
  BatchParams bp = make_params(p, nullptr);
  bp.handoff_running = B->handoff_running;
  bp.handoff_min_iters = B->handoff_min_iters;
  RET(run_batch_and_handoffs(B, bp, 0, st, p, nullptr));
  fill_reports(B, 0, reports);
  B->have_phase1 = 1;
  return PDHGC_OK;
}

int pdhgc_batch_corner_phase(pdhgc_batch* B, const pdhgc_corner_params* params, pdhgc_report* reports) {
  if (!B) return set_berr(PDHGC_ERR_INVALID_ARG, "batch is NULL");
  if (!B->have_phase1) return set_berr(PDHGC_ERR_NO_PHASE1, "pdhgc_batch_solve has not run");
  pdhgc_corner_params cp;
  if (params) cp = *params; else pdhgc_default_corner_params(&cp);
  RET(check_batch_corner_params(cp));
  cudaStream_t st = B->stream;
  std::fill(B->extc.begin(), B->extc.end(), 0);
  BatchParams bp = make_params(B->params, &cp);
  bp.handoff_running = B->handoff_running;
  bp.handoff_min_iters = B->handoff_min_iters;
  RET(run_batch_and_handoffs(B, bp, 1, st, B->params, &cp));
  fill_reports(B, 1, reports);
  B->have_corner = 1;
  return PDHGC_OK;
}

int pdhgc_batch_solve_corner(pdhgc_batch* B, const pdhgc_params* params, const pdhgc_corner_params* cparams,
                             pdhgc_report* reports1, pdhgc_report* reports_c) {
  if (!B) return set_berr(PDHGC_ERR_INVALID_ARG, "batch is NULL");
  pdhgc_params p;
  if (params) p = *params; else pdhgc_default_params(&p);
  pdhgc_corner_params cp;
  if (cparams) cp = *cparams; else pdhgc_default_corner_params(&cp);
  RET(check_batch_params(p));
  RET(check_batch_corner_params(cp));
  B->params = p;
  B->precision = p.precision;
  B->have_phase1 = 0;
  B->have_corner = 0;
  std::fill(B->ext1.begin(), B->ext1.end(), 0);
  std::fill(B->extc.begin(), B->extc.end(), 0);
  cudaStream_t st = B->stream;
  BatchParams bp = make_params(p, &cp);
  bp.handoff_running = B->handoff_running;
  bp.handoff_min_iters = B->handoff_min_iters;
  RET(run_batch_and_handoffs(B, bp, 2, st, p, &cp));
  fill_reports(B, 0, reports1);
  fill_reports(B, 1, reports_c);
  B->have_phase1 = 1;
  B->have_corner = 1;
  return PDHGC_OK;
}

int pdhgc_batch_get_solution(pdhgc_batch* B, int32_t lp, int which, double* x, double* y) {
  if (!B || lp < 0 || lp >= B->count || (which != PDHGC_PHASE1 && which != PDHGC_CORNER))
    return set_berr(PDHGC_ERR_INVALID_ARG, "bad argument");
  if (!B->have_phase1) return set_berr(PDHGC_ERR_NO_PHASE1, "pdhgc_batch_solve has not run");
  if (which == PDHGC_CORNER && !B->have_corner) return set_berr(PDHGC_ERR_NO_CORNER, "no corner result");
  const LpDesc& d = B->h_desc[lp];
  std::vector<double> xs(d.n), ys(d.m), Dc(d.n), Dr(d.m);
  cudaStream_t st = B->stream;
  BCK(cudaMemcpyAsync(xs.data(), which == PDHGC_PHASE1 ? d.x1 : d.xc, (size_t)d.n * 8, cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(ys.data(), d.y1, (size_t)d.m * 8, cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(Dc.data(), d.Dc, (size_t)d.n * 8, cudaMemcpyDeviceToHost, st));
  BCK(cudaMemcpyAsync(Dr.data(), d.Dr, (size_t)d.m * 8, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  if (x)
    for (int j = 0; j < d.n; ++j) x[B->col_perm[lp][j]] = Dc[j] * xs[j];
  if (y)
    for (int i = 0; i < d.m; ++i) y[B->row_perm[lp][i]] = B->sign[lp][i] * (Dr[i] * ys[i]);
  return PDHGC_OK;
}

int pdhgc_batch_set_block(pdhgc_batch* B, int32_t threads) {
  if (!B || (threads != 512 && threads != 1024)) return set_berr(PDHGC_ERR_INVALID_ARG, "threads must be 512 or 1024");
  B->block = threads;
  return PDHGC_OK;
}

int pdhgc_batch_set_lanes(pdhgc_batch* B, int32_t lanes_a, int32_t lanes_t) {
  if (!B) return set_berr(PDHGC_ERR_INVALID_ARG, "batch is NULL");
  auto ok = [](int g) { return g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32; };
  if (!ok(lanes_a) || !ok(lanes_t)) return set_berr(PDHGC_ERR_INVALID_ARG, "lanes must be 0 (auto) or 1..32, a power of two");
  for (int k = 0; k < B->count; ++k) {
    LpDesc& d = B->h_desc[k];
    d.gA = lanes_a ? lanes_a : lanes_for(d.m ? (double)d.nnz / d.m : 1.0);
    d.gT = lanes_t ? lanes_t : lanes_for(d.n ? (double)d.nnz / d.n : 1.0);
  }
  BCK(cudaMemcpyAsync(B->d_desc, B->h_desc.data(), B->count * sizeof(LpDesc), cudaMemcpyHostToDevice, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return PDHGC_OK;
}

int pdhgc_batch_set_layout(pdhgc_batch* B, int32_t sell) {
  if (!B || (sell != 0 && sell != 1)) return set_berr(PDHGC_ERR_INVALID_ARG, "sell must be 0 or 1");
  for (int k = 0; k < B->count; ++k) B->h_desc[k].sell = sell;
  BCK(cudaMemcpyAsync(B->d_desc, B->h_desc.data(), B->count * sizeof(LpDesc), cudaMemcpyHostToDevice, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  return PDHGC_OK;
}

// The schedule autotuner: times a fixed number of iterations of the whole
// batch (setup included, no early termination, so every candidate does the
// same work) for each candidate schedule and keeps the fastest.
int pdhgc_batch_tune(pdhgc_batch* B, const pdhgc_params* params, int32_t tune_iters, int32_t* chosen,
                     double* timings_ms) {
  if (!B || tune_iters < 1) return set_berr(PDHGC_ERR_INVALID_ARG, "bad argument");
  pdhgc_params p;
  if (params) p = *params; else pdhgc_default_params(&p);
  if (p.precision != PDHGC_FP64 && p.precision != PDHGC_FP32_BULK)
    return set_berr(PDHGC_ERR_INVALID_ARG, "precision must be PDHGC_FP64 or PDHGC_FP32_BULK");
  if (p.algorithm != PDHGC_ALG_AVERAGED && p.algorithm != PDHGC_ALG_HALPERN)
    return set_berr(PDHGC_ERR_INVALID_ARG, "algorithm must be PDHGC_ALG_AVERAGED or PDHGC_ALG_HALPERN");
  p.max_iters = tune_iters;
  p.eps_rel = -1.0;
  B->precision = p.precision;
  struct Cand {
    int block, sell, la, lt;
  };
  const Cand cands[] = {{1024, 1, 0, 0}, {512, 1, 0, 0}, {1024, 0, 0, 0}, {512, 0, 0, 0},
                        {1024, 0, 4, 2}, {1024, 0, 1, 1}, {1024, 0, 8, 4}};
  const int nc = (int)(sizeof(cands) / sizeof(cands[0]));
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  const BatchParams bp = make_params(p, nullptr);
  for (int ci = 0; ci < nc; ++ci) {
    RET(pdhgc_batch_set_block(B, cands[ci].block));
    RET(pdhgc_batch_set_layout(B, cands[ci].sell));
    RET(pdhgc_batch_set_lanes(B, cands[ci].la, cands[ci].lt));
    BCK(cudaEventRecord(e0, B->stream));
    RET(run_batch(B, bp, 0, B->stream));
    BCK(cudaEventRecord(e1, B->stream));
    BCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, e0, e1));
    if (timings_ms) timings_ms[ci] = ms;
    if (ci == 0 || ms < best_ms) {
      best = ci;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RET(pdhgc_batch_set_block(B, cands[best].block));
  RET(pdhgc_batch_set_layout(B, cands[best].sell));
  RET(pdhgc_batch_set_lanes(B, cands[best].la, cands[best].lt));
  if (chosen) {
    chosen[0] = cands[best].block;
    chosen[1] = cands[best].sell;
    chosen[2] = cands[best].la;
    chosen[3] = cands[best].lt;
  }
  B->have_phase1 = 0;  // the tuning runs overwrote the phase-1 state
  B->have_corner = 0;
  return PDHGC_OK;
}

int64_t pdhgc_batch_kernel_launches(const pdhgc_batch* B) { return B ? B->launches : 0; }

int pdhgc_batch_set_handoff(pdhgc_batch* B, int32_t max_running, int64_t min_iters) {
  if (!B || max_running < 0 || min_iters < 0) return set_berr(PDHGC_ERR_INVALID_ARG, "bad argument");
  B->handoff_running = max_running;
  B->handoff_min_iters = min_iters;
  return PDHGC_OK;
}

int32_t pdhgc_batch_handed_off(const pdhgc_batch* B, int32_t lp, int which) {
  if (!B || lp < 0 || lp >= B->count) return 0;
  return which == PDHGC_CORNER ? B->extc[lp] : B->ext1[lp];
}

void pdhgc_batch_destroy(pdhgc_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->stream);
  delete B;
}

}  // extern "C"
