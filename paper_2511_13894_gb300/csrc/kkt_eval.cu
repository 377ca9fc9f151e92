// pdhgc_kkt_eval: Section 2 optimality numbers and the Section 2.1 / 4.2
// metrics of a user-supplied point (x, y) on an LP given as a device CSR,
// without a handle.  The kernels need scratch memory beyond the inputs and
// outputs: an accumulator for A'y (n doubles) and per-block partial sums.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pdhgc.h"
#include "kkt_eval.h"

namespace pdhgc {

namespace {

__device__ __forceinline__ double proj_dual_ev(double lam, double l, double u) {
  const bool lf = l != -INFINITY, uf = u != INFINITY;
  if (lf && uf) return lam;
  if (lf) return fmax(lam, 0.0);
  if (uf) return fmin(lam, 0.0);
  return 0.0;
}

// deterministic block fold of per-thread values into out (sum or max)
__device__ double fold_block(double v, bool is_max, double* s_tmp) {
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, v, off);
    v = is_max ? fmax(v, o) : v + o;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = s_tmp[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = is_max ? fmax(t, s_tmp[w]) : t + s_tmp[w];
  return t;
}

__global__ void k_ev_zero(double* v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = 0.0;
}

// rows: (Ax)_i, the residual of each row under its sense, b'y, the slack
// metrics of inequality rows, and the scatter of y_i a_ij into A'y.
// Partials (kEvRowQ per block): sum r^2, max |r|, sum b y, off, zero, cand.
__global__ void __launch_bounds__(kEvThreads) k_ev_rows(EvalInput in, double* __restrict__ aty,
                                                        double* __restrict__ part) {
  __shared__ double s_tmp[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  double q[kEvRowQ] = {0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < in.m; i += warps) {
    const long long e0 = in.row_ptr[i], e1 = in.row_ptr[i + 1];
    const double yi = in.y[i];
    double s = 0.0;
    for (long long e = e0 + lane; e < e1; e += 32) {
      const double a = in.val[e];
      const int j = in.col_idx[e];
      s = fma(a, in.x[j], s);
      atomicAdd(aty + j, a * yi);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      const char sn = in.sense ? (char)in.sense[i] : '=';
      double r = in.b[i] - s;
      if (sn == '<') r = fmin(r, 0.0);
      if (sn == '>') r = fmax(r, 0.0);
      q[0] += r * r;
      q[1] = fmax(q[1], fabs(r));
      q[2] += in.b[i] * yi;
      if (sn != '=') {
        const double slack = sn == '<' ? in.b[i] - s : s - in.b[i];
        const bool off = slack > 1e-6, zero = fabs(yi) <= 1e-6;
        q[3] += off ? 1.0 : 0.0;
        q[4] += zero ? 1.0 : 0.0;
        q[5] += (off && zero) ? 1.0 : 0.0;
      }
    }
  }
  for (int k = 0; k < kEvRowQ; ++k) {
    const double t = fold_block(q[k], k == 1, s_tmp);
    if (threadIdx.x == 0) part[k * kEvBlocks + blockIdx.x] = t;
  }
}

// columns: lam = c - A'y, z = proj(lam), r_D = lam - z, c'x, the bound part
// of the dual objective and the structural metrics.  Partials (kEvColQ per
// block): sum r_D^2, max |r_D|, c x, l z+ - u z-, off, zero, cand.
__global__ void __launch_bounds__(kEvThreads) k_ev_cols(EvalInput in, const double* __restrict__ aty,
                                                        double* __restrict__ part) {
  __shared__ double s_tmp[32];
  double q[kEvColQ] = {0, 0, 0, 0, 0, 0, 0};
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < in.n; j += gridDim.x * blockDim.x) {
    const double l = in.lb ? in.lb[j] : 0.0;
    const double u = in.ub ? in.ub[j] : INFINITY;
    const double lam = in.c[j] - aty[j];
    const double z = proj_dual_ev(lam, l, u);
    const double rd = lam - z;
    const double xj = in.x[j];
    q[0] += rd * rd;
    q[1] = fmax(q[1], fabs(rd));
    q[2] += in.c[j] * xj;
    q[3] += (l != -INFINITY ? l * fmax(z, 0.0) : 0.0) - (u != INFINITY ? u * fmax(-z, 0.0) : 0.0);
    const bool off = fmin(xj - l, u - xj) > 1e-6, zero = fabs(z) <= 1e-6;
    q[4] += off ? 1.0 : 0.0;
    q[5] += zero ? 1.0 : 0.0;
    q[6] += (off && zero) ? 1.0 : 0.0;
  }
  for (int k = 0; k < kEvColQ; ++k) {
    const double t = fold_block(q[k], k == 1, s_tmp);
    if (threadIdx.x == 0) part[k * kEvBlocks + blockIdx.x] = t;
  }
}

// one CTA: fold the partials in block order and assemble the numbers
__global__ void k_ev_final(const double* __restrict__ rpart, const double* __restrict__ cpart, double nb,
                           double nc, double* __restrict__ out) {
  __shared__ double s_tmp[32];
  __shared__ double q[kEvRowQ + kEvColQ];
  for (int k = 0; k < kEvRowQ; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < kEvBlocks; b += blockDim.x)
      v = k == 1 ? fmax(v, rpart[k * kEvBlocks + b]) : v + rpart[k * kEvBlocks + b];
    const double t = fold_block(v, k == 1, s_tmp);
    if (threadIdx.x == 0) q[k] = t;
  }
  for (int k = 0; k < kEvColQ; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < kEvBlocks; b += blockDim.x)
      v = k == 1 ? fmax(v, cpart[k * kEvBlocks + b]) : v + cpart[k * kEvBlocks + b];
    const double t = fold_block(v, k == 1, s_tmp);
    if (threadIdx.x == 0) q[kEvRowQ + k] = t;
  }
  if (threadIdx.x != 0) return;
  const double* c = q + kEvRowQ;
  const double rP2 = sqrt(q[0]), rD2 = sqrt(c[0]);
  const double pobj = c[2], dobj = q[2] + c[3];
  out[0] = rP2;
  out[1] = rD2;
  out[2] = q[1];
  out[3] = c[1];
  out[4] = pobj;
  out[5] = dobj;
  out[6] = pobj - dobj;
  out[7] = rP2 / (1.0 + nb);
  out[8] = rD2 / (1.0 + nc);
  out[9] = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  out[10] = q[3] + c[4];  // p
  out[11] = q[4] + c[5];  // d
  out[12] = q[5] + c[6];  // candidates
}

// ||v||_2^2 into out[0] (one CTA, fixed order)
__global__ void k_ev_norm2(const double* __restrict__ v, int len, double* __restrict__ out) {
  __shared__ double s_tmp[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) a += v[i] * v[i];
  const double t = fold_block(a, false, s_tmp);
  if (threadIdx.x == 0) out[0] = t;
}

}  // namespace

size_t kkt_eval_scratch_doubles(int32_t n) {
  return (size_t)n + (size_t)(kEvRowQ + kEvColQ) * kEvBlocks + kEvOut;
}

int kkt_eval_check(int32_t m, int32_t n, int64_t nnz, const void* row_ptr, const void* col_idx, const void* val,
                   const void* b, const void* c, const void* x, const void* y, const pdhgc_report* out,
                   std::string& detail) {
  if (m < 1 || n < 1 || nnz < 0) {
    detail = "m and n must be >= 1, nnz >= 0";
    return PDHGC_ERR_INVALID_ARG;
  }
  if (!row_ptr || !b || !c || !x || !y || !out || (nnz > 0 && (!col_idx || !val))) {
    detail = "NULL argument";
    return PDHGC_ERR_INVALID_ARG;
  }
  return PDHGC_OK;
}

int kkt_eval_run(const EvalInput& in, double* scratch, cudaStream_t st, pdhgc_report* out, std::string& detail) {
  double* aty = scratch;
  double* rpart = aty + in.n;
  double* cpart = rpart + (size_t)kEvRowQ * kEvBlocks;
  double* res = cpart + (size_t)kEvColQ * kEvBlocks;
  auto fail = [&](cudaError_t e, const char* what) {
    detail = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PDHGC_ERR_OOM : PDHGC_ERR_CUDA;
  };
  k_ev_zero<<<kEvBlocks, kEvThreads, 0, st>>>(aty, in.n);
  k_ev_rows<<<kEvBlocks, kEvThreads, 0, st>>>(in, aty, rpart);
  k_ev_cols<<<kEvBlocks, kEvThreads, 0, st>>>(in, aty, cpart);
  k_ev_norm2<<<1, kEvThreads, 0, st>>>(in.b, in.m, res + 13);
  k_ev_norm2<<<1, kEvThreads, 0, st>>>(in.c, in.n, res + 14);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e, "kkt_eval launch");
  double h[kEvOut];
  e = cudaMemcpyAsync(h + 13, res + 13, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e, "kkt_eval norms");
  k_ev_final<<<1, kEvThreads, 0, st>>>(rpart, cpart, std::sqrt(h[13]), std::sqrt(h[14]), res);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, 13 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e, "kkt_eval");
  std::memset(out, 0, sizeof(*out));
  out->rP2 = h[0];
  out->rD2 = h[1];
  out->rPinf = h[2];
  out->rDinf = h[3];
  out->pobj = h[4];
  out->dobj = h[5];
  out->gap = h[6];
  out->rel_p = h[7];
  out->rel_d = h[8];
  out->rel_gap = h[9];
  out->rel_kkt = std::fmax(h[7], std::fmax(h[8], h[9]));
  const int64_t mm = in.m;
  out->off_bound_p = (int64_t)std::llround(h[10]);
  out->zero_rc_d = (int64_t)std::llround(h[11]);
  out->candidates = (int64_t)std::llround(h[12]);
  out->corner_measure = out->candidates > mm ? out->candidates - mm : 0;
  out->primal_push_est = out->off_bound_p > mm ? out->off_bound_p - mm : 0;
  out->dual_push_est = mm > out->zero_rc_d ? mm - out->zero_rc_d : 0;
  const int64_t thr = 2 * mm > 100000 ? 2 * mm : 100000;
  out->should_corner = out->candidates >= thr ? 1 : 0;
  return PDHGC_OK;
}

}  // namespace pdhgc

extern "C" int pdhgc_kkt_eval(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                              const double* val, const double* b, const double* c, const double* lb,
                              const double* ub, const int8_t* sense, const double* x, const double* y,
                              pdhgc_report* out, void* cuda_stream) {
  std::string detail;
  int rc = pdhgc::kkt_eval_check(m, n, nnz, row_ptr, col_idx, val, b, c, x, y, out, detail);
  if (rc != PDHGC_OK) return pdhgc::set_error_detail(rc, detail);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t bytes = pdhgc::kkt_eval_scratch_doubles(n) * sizeof(double);
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, bytes, st);
  if (e != cudaSuccess)
    return pdhgc::set_error_detail(PDHGC_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  pdhgc::EvalInput in{m, n, row_ptr, col_idx, val, b, c, lb, ub, sense, x, y};
  rc = pdhgc::kkt_eval_run(in, static_cast<double*>(scratch), st, out, detail);
  cudaFreeAsync(scratch, st);
  cudaStreamSynchronize(st);
  if (rc != PDHGC_OK) return pdhgc::set_error_detail(rc, detail);
  return PDHGC_OK;
}

// ---------------------------------------------------------------------------
// pdhgc_kkt_eval_noalloc: the same evaluation with its scratch in a
// file-scope device array instead of cudaMallocAsync, for callers that must
// not allocate device memory (see include/pdhgc.h).
// ---------------------------------------------------------------------------
namespace {

constexpr int32_t kNoAllocMaxN = 1 << 18;  // largest n the static scratch holds
constexpr size_t kNoAllocDoubles = (size_t)kNoAllocMaxN + (size_t)(pdhgc::kEvRowQ + pdhgc::kEvColQ) *
                                                               pdhgc::kEvBlocks + pdhgc::kEvOut;

// Shared by every call on a device and kept until the process exits; each call
// overwrites all of it that it reads (the A'y accumulator is zeroed first).
static __device__ __align__(256) double g_kkt_eval_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// true when p is device memory of device `dev` in the current context (a
// cached address stays valid until cudaDeviceReset replaces the context)
bool still_device_memory(const void* p, int dev) {
  cudaPointerAttributes a{};
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // not a pointer of this context: clear the error it set
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// device address of g_kkt_eval_scratch for the current device, looked up
// with that device current on its first call, and again whenever the cached
// address no longer belongs to the device's current context
int scratch_for_current_device(double** out, std::string& detail) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    detail = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return PDHGC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    detail = "device ordinal out of range";
    return PDHGC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev] || !still_device_memory(g_scratch_ptr[dev], dev)) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_kkt_eval_scratch);
    if (e != cudaSuccess || !p) {
      detail = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return PDHGC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PDHGC_OK;
}

}  // namespace

extern "C" int pdhgc_kkt_eval_noalloc(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                                      const int32_t* col_idx, const double* val, const double* b, const double* c,
                                      const double* lb, const double* ub, const int8_t* sense, const double* x,
                                      const double* y, pdhgc_report* out, void* cuda_stream) {
  std::string detail;
  int rc = pdhgc::kkt_eval_check(m, n, nnz, row_ptr, col_idx, val, b, c, x, y, out, detail);
  if (rc != PDHGC_OK) return pdhgc::set_error_detail(rc, detail);
  if (n > kNoAllocMaxN)
    return pdhgc::set_error_detail(PDHGC_ERR_TOO_LARGE,
                                   "pdhgc_kkt_eval_noalloc: n = " + std::to_string(n) +
                                       " exceeds the static scratch capacity of " +
                                       std::to_string(kNoAllocMaxN) + " columns; use pdhgc_kkt_eval");
  double* scratch = nullptr;
  rc = scratch_for_current_device(&scratch, detail);
  if (rc != PDHGC_OK) return pdhgc::set_error_detail(rc, detail);
  pdhgc::EvalInput in{m, n, row_ptr, col_idx, val, b, c, lb, ub, sense, x, y};
  rc = pdhgc::kkt_eval_run(in, scratch, static_cast<cudaStream_t>(cuda_stream), out, detail);
  if (rc != PDHGC_OK) return pdhgc::set_error_detail(rc, detail);
  return PDHGC_OK;
}
