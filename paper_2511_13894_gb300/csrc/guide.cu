// Corner-guidance network (extension of Algorithm 1; the paper has none):
// forward pass, minibatch gradient and Adam for an 18 -> 64 -> 64 -> 1 MLP
// with ReLU hidden layers and a sigmoid output trained on the mean binary
// cross-entropy.  BF16 weights and activations, FP32 accumulation.
//
// Tensor-core layout.  A warp owns 16 samples.  Both layers are
// mma.sync m16n8k16 BF16 products: the accumulator fragment of one layer is,
// element for element, the A fragment of the next (rows g and g + 8, columns
// 2t, 2t + 1 of each 8-wide n tile), so activations never leave registers in
// the forward pass.  The backward data gradient dA1 = dZ2 W2 reuses the same
// mapping with W2' staged in shared memory.  The weight gradients
// dZ' A (a reduction over samples) run per 64-sample chunk on the tensor
// cores from shared-memory copies of the chunk, one 16-row slice of the
// gradient per warp, accumulated in registers across chunks; per-CTA
// partials are then folded in a fixed order, so a step is deterministic.
//
// Inference (k_guide_forward_tc) runs on the 5th-generation tensor cores:
// tcgen05.mma from shared-memory operands into tensor-memory accumulators,
// 128 rows per tile, one CTA per SM.  k_guide_forward is the mma.sync form
// of the same pass (built with PDHGC_GUIDE_TC=0).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pdhgc.h"
#include "guide.h"
#include "kkt_eval.h"

using namespace pdhgc;

namespace {

constexpr int kGWarps = 4;
constexpr int kGThreads = kGWarps * 32;
constexpr int kChunk = kGWarps * 16;  // samples per CTA step of the training kernel
constexpr int kS40 = 40;               // padded shared row of 32 BF16 (conflict-free fragment loads)
constexpr int kS72 = 72;               // padded shared row of 64 BF16

#define GK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_error_detail(e_ == cudaErrorMemoryAllocation ? PDHGC_ERR_OOM : PDHGC_ERR_CUDA, \
                              std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

#define GKL()                                                                            \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      return set_error_detail(PDHGC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two floats -> BF16 pair, the first in the low half (the lower k index)
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_bf(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ float bf_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float relu(float x) { return x > 0.0f ? x : 0.0f; }
__device__ __forceinline__ bool lo_pos(uint32_t v) { return (v & 0x7fffu) != 0u; }
__device__ __forceinline__ bool hi_pos(uint32_t v) { return (v & 0x7fff0000u) != 0u; }

// SplitMix64 (Steele, Lea and Flood 2014): output j of the stream at `seed`
__device__ __forceinline__ unsigned long long mix64(unsigned long long seed, unsigned long long j) {
  unsigned long long z = seed + (j + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// stage W1 (padded, stride 40) and W2 (stride 72) and optionally W2' in shared memory
__device__ void stage_weights(const GuideBf16* __restrict__ wb, __nv_bfloat16* sW1, __nv_bfloat16* sW2,
                              __nv_bfloat16* sW2T) {
  const uint32_t* w1 = reinterpret_cast<const uint32_t*>(wb->w1);
  const uint32_t* w2 = reinterpret_cast<const uint32_t*>(wb->w2);
  const uint32_t* w2t = reinterpret_cast<const uint32_t*>(wb->w2t);
  uint32_t* s1 = reinterpret_cast<uint32_t*>(sW1);
  uint32_t* s2 = reinterpret_cast<uint32_t*>(sW2);
  uint32_t* s2t = reinterpret_cast<uint32_t*>(sW2T);
  for (int e = threadIdx.x; e < kGHid * 16; e += blockDim.x) s1[(e >> 4) * (kS40 / 2) + (e & 15)] = w1[e];
  for (int e = threadIdx.x; e < kGHid * 32; e += blockDim.x) {
    s2[(e >> 5) * (kS72 / 2) + (e & 31)] = w2[e];
    if (sW2T) s2t[(e >> 5) * (kS72 / 2) + (e & 31)] = w2t[e];
  }
}

// Layers 1 and 2 of one 16-row tile: a = the 2 k-steps of input fragments;
// returns h (layer-1 activations as layer-2 A fragments) and acc2 (layer-2
// pre-activations incl. bias)
__device__ __forceinline__ void forward_tile(const uint32_t (&a)[2][4], const __nv_bfloat16* sW1,
                                             const __nv_bfloat16* sW2, const float* sb1, const float* sb2,
                                             uint32_t (&h)[4][4], float (&acc2)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* s1 = reinterpret_cast<const uint32_t*>(sW1);
  const uint32_t* s2 = reinterpret_cast<const uint32_t*>(sW2);
  float acc1[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = sb1[nt * 8 + 2 * t], b1 = sb1[nt * 8 + 2 * t + 1];
    acc1[nt][0] = b0;
    acc1[nt][1] = b1;
    acc1[nt][2] = b0;
    acc1[nt][3] = b1;
  }
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int row = (nt * 8 + g) * (kS40 / 2) + ks * 8 + t;
      mma16816(acc1[nt], a[ks], s1[row], s1[row + 4]);
    }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    h[ks][0] = pack2(relu(acc1[2 * ks][0]), relu(acc1[2 * ks][1]));
    h[ks][1] = pack2(relu(acc1[2 * ks][2]), relu(acc1[2 * ks][3]));
    h[ks][2] = pack2(relu(acc1[2 * ks + 1][0]), relu(acc1[2 * ks + 1][1]));
    h[ks][3] = pack2(relu(acc1[2 * ks + 1][2]), relu(acc1[2 * ks + 1][3]));
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = sb2[nt * 8 + 2 * t], b1 = sb2[nt * 8 + 2 * t + 1];
    acc2[nt][0] = b0;
    acc2[nt][1] = b1;
    acc2[nt][2] = b0;
    acc2[nt][3] = b1;
  }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int row = (nt * 8 + g) * (kS72 / 2) + ks * 8 + t;
      mma16816(acc2[nt], h[ks], s2[row], s2[row + 4]);
    }
}

// output logits of rows g and g + 8 (reduced over the 4 lanes of a row)
__device__ __forceinline__ void output_tile(const float (&acc2)[8][4], const float* sw3, float& o0, float& o1) {
  const int t = threadIdx.x & 3;
  o0 = 0.0f;
  o1 = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float w0 = sw3[nt * 8 + 2 * t], w1 = sw3[nt * 8 + 2 * t + 1];
    o0 = fmaf(bf_round(relu(acc2[nt][0])), w0, o0);
    o0 = fmaf(bf_round(relu(acc2[nt][1])), w1, o0);
    o1 = fmaf(bf_round(relu(acc2[nt][2])), w0, o1);
    o1 = fmaf(bf_round(relu(acc2[nt][3])), w1, o1);
  }
  o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
  o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
  o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
  o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
}

__device__ __forceinline__ float sigmoid(float o) { return 1.0f / (1.0f + expf(-o)); }

__global__ void __launch_bounds__(kGThreads) k_guide_forward(const GuideBf16* __restrict__ wb,
                                                              const float* __restrict__ w,
                                                              const __nv_bfloat16* __restrict__ feat,
                                                              long long rows, float* __restrict__ p) {
  __shared__ __align__(16) __nv_bfloat16 sW1[kGHid * kS40];
  __shared__ __align__(16) __nv_bfloat16 sW2[kGHid * kS72];
  __shared__ float sb1[kGHid], sb2[kGHid], sw3[kGHid];
  stage_weights(wb, sW1, sW2, nullptr);
  for (int j = threadIdx.x; j < kGHid; j += blockDim.x) {
    sb1[j] = w[kOffB1 + j];
    sb2[j] = w[kOffB2 + j];
    sw3[j] = __bfloat162float(wb->w3[j]);
  }
  const float b3 = w[kOffB3];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const long long ntiles = (rows + 15) / 16;
  const uint32_t* f = reinterpret_cast<const uint32_t*>(feat);
  for (long long tile = (long long)blockIdx.x * kGWarps + warp; tile < ntiles;
       tile += (long long)gridDim.x * kGWarps) {
    const long long r0 = tile * 16 + g, r1 = r0 + 8;
    uint32_t a[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a[ks][0] = r0 < rows ? f[r0 * 16 + ks * 8 + t] : 0u;
      a[ks][1] = r1 < rows ? f[r1 * 16 + ks * 8 + t] : 0u;
      a[ks][2] = r0 < rows ? f[r0 * 16 + ks * 8 + 4 + t] : 0u;
      a[ks][3] = r1 < rows ? f[r1 * 16 + ks * 8 + 4 + t] : 0u;
    }
    uint32_t h[4][4];
    float acc2[8][4];
    forward_tile(a, sW1, sW2, sb1, sb2, h, acc2);
    float o0, o1;
    output_tile(acc2, sw3, o0, o1);
    if (t == 0) {
      if (r0 < rows) p[r0] = sigmoid(o0 + b3);
      if (r1 < rows) p[r1] = sigmoid(o1 + b3);
    }
  }
}

// ---------------------------------------------------------------------------
// Inference on the 5th-generation tensor cores: tcgen05.mma with operands in
// shared memory and FP32 accumulators in tensor memory.  One CTA per SM
// (persistent over 128-row tiles), 4 warps; thread t owns row t of a tile.
// Layer 1: D1[128 x 64] = X[128 x 32] W1'; layer 2: D2[128 x 64] = A1[128 x 64]
// W2'.  Operands use the K-major layout without swizzle: core matrices of
// 8 rows x 16 bytes (8 BF16) stored contiguously, the K-adjacent cores 128
// bytes apart (leading byte offset) and the 8-row groups KC x 128 bytes apart
// (stride byte offset), KC = K / 8.
// ---------------------------------------------------------------------------
constexpr int kTcRows = 128;
constexpr uint32_t kTcCols = 128;          // TMEM columns: [0, 64) layer 1, [64, 128) layer 2
constexpr long long kTcWaitLimit = 1ll << 24;  // bounded mbarrier wait (iterations)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading / stride byte offsets,
// the fixed version field (bits 46-47 = 1), base offset 0, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// bounded wait for phase `parity` of the mbarrier; false when `limit` polls ran out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane (warp w reads lanes 32w..32w+31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element (row r, k) in the K-major core-matrix layout with KC cores per row group
__device__ __forceinline__ uint32_t core_off(int r, int k, int KC) {
  return (uint32_t)((((r >> 3) * KC + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

struct TcSmem {
  __nv_bfloat16 x[kTcRows * kGFeat];   // 8 KB, KC = 4
  __nv_bfloat16 a1[kTcRows * kGHid];   // 16 KB, KC = 8
  __nv_bfloat16 w1[kGHid * kGFeat];    // 4 KB, KC = 4
  __nv_bfloat16 w2[kGHid * kGHid];     // 8 KB, KC = 8
  float b1[kGHid], b2[kGHid], w3[kGHid];
  unsigned long long mbar;
  uint32_t tmem_base;
};

__global__ void __launch_bounds__(kTcRows, 1) k_guide_forward_tc(const GuideBf16* __restrict__ wb,
                                                                 const float* __restrict__ w,
                                                                 const __nv_bfloat16* __restrict__ feat,
                                                                 long long rows, float* __restrict__ p,
                                                                 int* __restrict__ err, long long wait_limit) {
  extern __shared__ __align__(128) unsigned char tc_raw[];
  TcSmem& s = *reinterpret_cast<TcSmem*>(tc_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights in the core-matrix layout: one 16-byte chunk (8 inputs of one unit) per copy
  for (int e = tid; e < kGHid * (kGFeat / 8); e += blockDim.x) {
    const int j = e / (kGFeat / 8), kc = e % (kGFeat / 8);
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.w1) + core_off(j, kc * 8, kGFeat / 8)) =
        *reinterpret_cast<const uint4*>(wb->w1 + j * kGFeat + kc * 8);
  }
  for (int e = tid; e < kGHid * (kGHid / 8); e += blockDim.x) {
    const int j = e / (kGHid / 8), kc = e % (kGHid / 8);
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.w2) + core_off(j, kc * 8, kGHid / 8)) =
        *reinterpret_cast<const uint4*>(wb->w2 + j * kGHid + kc * 8);
  }
  for (int j = tid; j < kGHid; j += blockDim.x) {
    s.b1[j] = w[kOffB1 + j];
    s.b2[j] = w[kOffB2 + j];
    s.w3[j] = __bfloat162float(wb->w3[j]);
  }
  const float b3 = w[kOffB3];
  const uint32_t mbar = smem_addr(&s.mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s.tmem_base)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  async_proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s.tmem_base;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t x_addr = smem_addr(s.x), a1_addr = smem_addr(s.a1);
  const uint32_t w1_addr = smem_addr(s.w1), w2_addr = smem_addr(s.w2);
  constexpr uint32_t kIdesc = umma_idesc(kTcRows, kGHid);
  uint32_t parity = 0;
  bool ok = true;
  const long long ntiles = (rows + kTcRows - 1) / kTcRows;
  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    // ---- this thread's input row into the core layout (zeros past the end)
    const long long r = tile * kTcRows + tid;
    const uint4* src = reinterpret_cast<const uint4*>(feat + r * kGFeat);
#pragma unroll
    for (int kc = 0; kc < kGFeat / 8; ++kc) {
      const uint4 v = r < rows ? src[kc] : make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.x) + core_off(tid, kc * 8, kGFeat / 8)) = v;
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    // ---- layer 1: two K = 16 steps into TMEM columns [0, 64)
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kGFeat / 16; ++ks)
        umma_bf16(tmem, umma_desc(x_addr + ks * 256, 128, (kGFeat / 8) * 128),
                  umma_desc(w1_addr + ks * 256, 128, (kGFeat / 8) * 128), kIdesc, ks > 0 ? 1u : 0u);
      umma_commit(mbar);
    }
    ok = __syncthreads_and(mbar_wait(mbar, parity, wait_limit)) != 0;  // the same decision in every thread
    if (!ok) break;
    parity ^= 1u;
    tc_fence_after();
    // ---- epilogue 1: bias, ReLU, BF16, into the layer-2 operand
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float v[32];
      tmem_ld32(tmem + lane_base + half * 32, v);
#pragma unroll
      for (int c8 = 0; c8 < 4; ++c8) {
        uint32_t q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = half * 32 + c8 * 8 + 2 * u;
          q[u] = pack2(relu(v[c8 * 8 + 2 * u] + s.b1[j]), relu(v[c8 * 8 + 2 * u + 1] + s.b1[j + 1]));
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(s.a1) +
                                  core_off(tid, half * 32 + c8 * 8, kGHid / 8)) = make_uint4(q[0], q[1], q[2], q[3]);
      }
    }
    async_proxy_fence();
    tc_fence_before();
    __syncthreads();
    // ---- layer 2: four K = 16 steps into TMEM columns [64, 128)
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kGHid / 16; ++ks)
        umma_bf16(tmem + 64, umma_desc(a1_addr + ks * 256, 128, (kGHid / 8) * 128),
                  umma_desc(w2_addr + ks * 256, 128, (kGHid / 8) * 128), kIdesc, ks > 0 ? 1u : 0u);
      umma_commit(mbar);
    }
    ok = __syncthreads_and(mbar_wait(mbar, parity, wait_limit)) != 0;
    if (!ok) break;
    parity ^= 1u;
    tc_fence_after();
    // ---- epilogue 2: bias, ReLU, BF16 activations, the output unit, sigmoid
    float o = b3;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float v[32];
      tmem_ld32(tmem + lane_base + 64 + half * 32, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int j = half * 32 + i;
        o = fmaf(bf_round(relu(v[i] + s.b2[j])), s.w3[j], o);
      }
    }
    if (r < rows) p[r] = sigmoid(o);
    tc_fence_before();
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    // the pending MMA may still be in flight: give it the full bounded time to
    // land before the tensor memory is freed
    mbar_wait(mbar, parity, kTcWaitLimit);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

// dynamic shared memory of the training kernel (BF16 unless noted)
struct TrainSmem {
  __nv_bfloat16 w1[kGHid * kS40];
  __nv_bfloat16 w2[kGHid * kS72];
  __nv_bfloat16 w2t[kGHid * kS72];
  __nv_bfloat16 x[kChunk * kS40];   // the chunk's inputs
  __nv_bfloat16 a1[kChunk * kS72];  // layer-1 activations
  __nv_bfloat16 d2[kChunk * kS72];  // dL/dZ2
  __nv_bfloat16 d1[kChunk * kS72];  // dL/dZ1
  float b1[kGHid], b2[kGHid], w3[kGHid];
  float gb1[kGWarps][kGHid], gb2[kGWarps][kGHid], gw3[kGWarps][kGHid];
  float gb3[kGWarps], loss[kGWarps];
};

// store a 16 x 64 accumulator-layout tile (rows g, g + 8 of warp `warp`) as BF16
__device__ __forceinline__ void store_tile72(__nv_bfloat16* dst, int warp, const uint32_t (&v)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  const int r0 = (warp * 16 + g) * (kS72 / 2), r1 = r0 + 8 * (kS72 / 2);
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    d[r0 + ks * 8 + t] = v[ks][0];
    d[r1 + ks * 8 + t] = v[ks][1];
    d[r0 + ks * 8 + 4 + t] = v[ks][2];
    d[r1 + ks * 8 + 4 + t] = v[ks][3];
  }
}

// sum over the 8 row groups of a warp (lanes with equal t), then lanes 0..3
// add the column sums of their two columns per n tile to acc[64]
__device__ __forceinline__ void col_sums_add(float (&v)[8][2], float* acc) {
  const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float s = v[nt][q];
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      s += __shfl_xor_sync(0xffffffffu, s, 8);
      s += __shfl_xor_sync(0xffffffffu, s, 16);
      if (lane < 4) acc[nt * 8 + 2 * t + q] += s;
    }
}

__global__ void __launch_bounds__(kGThreads) k_guide_grad(const GuideBf16* __restrict__ wb,
                                                           const float* __restrict__ w,
                                                           const __nv_bfloat16* __restrict__ feat,
                                                           const uint8_t* __restrict__ labels, long long rows,
                                                           const int32_t* __restrict__ idx, int batch,
                                                           unsigned long long seed, long long step,
                                                           float* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  stage_weights(wb, s.w1, s.w2, s.w2t);
  for (int j = threadIdx.x; j < kGHid; j += blockDim.x) {
    s.b1[j] = w[kOffB1 + j];
    s.b2[j] = w[kOffB2 + j];
    s.w3[j] = __bfloat162float(wb->w3[j]);
    for (int q = 0; q < kGWarps; ++q) {
      s.gb1[q][j] = 0.0f;
      s.gb2[q][j] = 0.0f;
      s.gw3[q][j] = 0.0f;
    }
  }
  if (threadIdx.x < kGWarps) {
    s.gb3[threadIdx.x] = 0.0f;
    s.loss[threadIdx.x] = 0.0f;
  }
  const float b3 = w[kOffB3];
  const float inv_b = 1.0f / (float)batch;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const uint32_t* f = reinterpret_cast<const uint32_t*>(feat);
  uint32_t* sx = reinterpret_cast<uint32_t*>(s.x);
  const uint32_t* sw2t = reinterpret_cast<const uint32_t*>(s.w2t);
  float gW2[8][4], gW1[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) gW2[nt][0] = gW2[nt][1] = gW2[nt][2] = gW2[nt][3] = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) gW1[nt][0] = gW1[nt][1] = gW1[nt][2] = gW1[nt][3] = 0.0f;
  const int nchunks = (batch + kChunk - 1) / kChunk;
  for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
    // ---- the warp's 16 samples: dataset rows and labels
    const int s_base = c * kChunk + warp * 16;
    long long src = -1;
    float lab = 0.0f;
    if (lane < 16 && s_base + lane < batch) {
      const int sidx = s_base + lane;
      src = idx ? (long long)idx[sidx]
                : (long long)(mix64(seed, (unsigned long long)step * (unsigned long long)batch + sidx) %
                              (unsigned long long)rows);
      lab = labels[src] ? 1.0f : 0.0f;
    }
    for (int e = lane; e < 16 * 16; e += 32) {
      const int rr = e >> 4, kw = e & 15;
      const long long sr = __shfl_sync(0xffffffffu, src, rr);
      sx[(warp * 16 + rr) * (kS40 / 2) + kw] = sr >= 0 ? f[sr * 16 + kw] : 0u;
    }
    const float y0 = __shfl_sync(0xffffffffu, lab, g), y1 = __shfl_sync(0xffffffffu, lab, g + 8);
    const bool v0 = s_base + g < batch, v1 = s_base + g + 8 < batch;
    __syncwarp();
    // ---- forward
    uint32_t a[2][4];
    const int xr0 = (warp * 16 + g) * (kS40 / 2), xr1 = xr0 + 8 * (kS40 / 2);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      a[ks][0] = sx[xr0 + ks * 8 + t];
      a[ks][1] = sx[xr1 + ks * 8 + t];
      a[ks][2] = sx[xr0 + ks * 8 + 4 + t];
      a[ks][3] = sx[xr1 + ks * 8 + 4 + t];
    }
    uint32_t h[4][4];
    float acc2[8][4];
    forward_tile(a, s.w1, s.w2, s.b1, s.b2, h, acc2);
    float o0, o1;
    output_tile(acc2, s.w3, o0, o1);
    o0 += b3;
    o1 += b3;
    // ---- loss and dL/do = (p - y) / batch
    const float p0 = sigmoid(o0), p1 = sigmoid(o1);
    const float do0 = v0 ? (p0 - y0) * inv_b : 0.0f;
    const float do1 = v1 ? (p1 - y1) * inv_b : 0.0f;
    if (t == 0) {
      // binary cross-entropy from the logit: softplus(o) - y o
      float l = 0.0f;
      if (v0) l += (fmaxf(o0, 0.0f) + log1pf(expf(-fabsf(o0))) - y0 * o0) * inv_b;
      if (v1) l += (fmaxf(o1, 0.0f) + log1pf(expf(-fabsf(o1))) - y1 * o1) * inv_b;
      float gb = do0 + do1;
      // rows of the warp: sum over the 8 groups (lanes 0, 4, ..., 28)
      for (int off = 4; off < 32; off <<= 1) {
        l += __shfl_xor_sync(0x11111111u, l, off);
        gb += __shfl_xor_sync(0x11111111u, gb, off);
      }
      if (lane == 0) {
        s.loss[warp] += l;
        s.gb3[warp] += gb;
      }
    }
    // ---- layer 3 and layer 2 backward
    uint32_t d2[4][4];
    {
      float gw3p[8][2], gb2p[8][2];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float w0 = s.w3[nt * 8 + 2 * t], w1 = s.w3[nt * 8 + 2 * t + 1];
        gw3p[nt][0] = do0 * bf_round(relu(acc2[nt][0])) + do1 * bf_round(relu(acc2[nt][2]));
        gw3p[nt][1] = do0 * bf_round(relu(acc2[nt][1])) + do1 * bf_round(relu(acc2[nt][3]));
        const float z00 = acc2[nt][0] > 0.0f ? do0 * w0 : 0.0f;
        const float z01 = acc2[nt][1] > 0.0f ? do0 * w1 : 0.0f;
        const float z10 = acc2[nt][2] > 0.0f ? do1 * w0 : 0.0f;
        const float z11 = acc2[nt][3] > 0.0f ? do1 * w1 : 0.0f;
        gb2p[nt][0] = z00 + z10;
        gb2p[nt][1] = z01 + z11;
        const int ks = nt >> 1, hi = (nt & 1) * 2;
        d2[ks][hi + 0] = pack2(z00, z01);
        d2[ks][hi + 1] = pack2(z10, z11);
      }
      col_sums_add(gw3p, s.gw3[warp]);
      col_sums_add(gb2p, s.gb2[warp]);
    }
    store_tile72(s.a1, warp, h);
    store_tile72(s.d2, warp, d2);
    // ---- dA1 = dZ2 W2 (tensor cores), dZ1 = dA1 where Z1 > 0
    {
      float acc3[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) acc3[nt][0] = acc3[nt][1] = acc3[nt][2] = acc3[nt][3] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          const int row = (nt * 8 + g) * (kS72 / 2) + ks * 8 + t;
          mma16816(acc3[nt], d2[ks], sw2t[row], sw2t[row + 4]);
        }
      uint32_t d1[4][4];
      float gb1p[8][2];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int ks = nt >> 1, hi = (nt & 1) * 2;
        const uint32_t m0 = h[ks][hi + 0], m1 = h[ks][hi + 1];
        const float z00 = lo_pos(m0) ? acc3[nt][0] : 0.0f;
        const float z01 = hi_pos(m0) ? acc3[nt][1] : 0.0f;
        const float z10 = lo_pos(m1) ? acc3[nt][2] : 0.0f;
        const float z11 = hi_pos(m1) ? acc3[nt][3] : 0.0f;
        gb1p[nt][0] = z00 + z10;
        gb1p[nt][1] = z01 + z11;
        d1[ks][hi + 0] = pack2(z00, z01);
        d1[ks][hi + 1] = pack2(z10, z11);
      }
      col_sums_add(gb1p, s.gb1[warp]);
      store_tile72(s.d1, warp, d1);
    }
    __syncthreads();
    // ---- weight gradients over the chunk's 64 samples: warp w owns rows
    // [16w, 16w + 16) of dW2 = dZ2' A1 and dW1 = dZ1' X
    {
      const int j0 = warp * 16;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int s0 = ks * 16 + 2 * t;
        uint32_t ad2[4], ad1[4];
        ad2[0] = pack_bf(s.d2[s0 * kS72 + j0 + g], s.d2[(s0 + 1) * kS72 + j0 + g]);
        ad2[1] = pack_bf(s.d2[s0 * kS72 + j0 + g + 8], s.d2[(s0 + 1) * kS72 + j0 + g + 8]);
        ad2[2] = pack_bf(s.d2[(s0 + 8) * kS72 + j0 + g], s.d2[(s0 + 9) * kS72 + j0 + g]);
        ad2[3] = pack_bf(s.d2[(s0 + 8) * kS72 + j0 + g + 8], s.d2[(s0 + 9) * kS72 + j0 + g + 8]);
        ad1[0] = pack_bf(s.d1[s0 * kS72 + j0 + g], s.d1[(s0 + 1) * kS72 + j0 + g]);
        ad1[1] = pack_bf(s.d1[s0 * kS72 + j0 + g + 8], s.d1[(s0 + 1) * kS72 + j0 + g + 8]);
        ad1[2] = pack_bf(s.d1[(s0 + 8) * kS72 + j0 + g], s.d1[(s0 + 9) * kS72 + j0 + g]);
        ad1[3] = pack_bf(s.d1[(s0 + 8) * kS72 + j0 + g + 8], s.d1[(s0 + 9) * kS72 + j0 + g + 8]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          const int col = nt * 8 + g;
          const uint32_t b0 = pack_bf(s.a1[s0 * kS72 + col], s.a1[(s0 + 1) * kS72 + col]);
          const uint32_t b1 = pack_bf(s.a1[(s0 + 8) * kS72 + col], s.a1[(s0 + 9) * kS72 + col]);
          mma16816(gW2[nt], ad2, b0, b1);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int col = nt * 8 + g;
          const uint32_t b0 = pack_bf(s.x[s0 * kS40 + col], s.x[(s0 + 1) * kS40 + col]);
          const uint32_t b1 = pack_bf(s.x[(s0 + 8) * kS40 + col], s.x[(s0 + 9) * kS40 + col]);
          mma16816(gW1[nt], ad1, b0, b1);
        }
      }
    }
    __syncthreads();
  }
  // ---- this CTA's partial gradient
  float* out = partials + (size_t)blockIdx.x * kGPartial;
  const int j0 = warp * 16;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int k = nt * 8 + 2 * t;
    out[kOffW2 + (j0 + g) * kGHid + k] = gW2[nt][0];
    out[kOffW2 + (j0 + g) * kGHid + k + 1] = gW2[nt][1];
    out[kOffW2 + (j0 + g + 8) * kGHid + k] = gW2[nt][2];
    out[kOffW2 + (j0 + g + 8) * kGHid + k + 1] = gW2[nt][3];
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int k = nt * 8 + 2 * t;
    if (k < kGIn) {
      out[kOffW1 + (j0 + g) * kGIn + k] = gW1[nt][0];
      out[kOffW1 + (j0 + g + 8) * kGIn + k] = gW1[nt][2];
    }
    if (k + 1 < kGIn) {
      out[kOffW1 + (j0 + g) * kGIn + k + 1] = gW1[nt][1];
      out[kOffW1 + (j0 + g + 8) * kGIn + k + 1] = gW1[nt][3];
    }
  }
  for (int j = threadIdx.x; j < kGHid; j += blockDim.x) {
    float a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    for (int q = 0; q < kGWarps; ++q) {
      a1 += s.gb1[q][j];
      a2 += s.gb2[q][j];
      a3 += s.gw3[q][j];
    }
    out[kOffB1 + j] = a1;
    out[kOffB2 + j] = a2;
    out[kOffW3 + j] = a3;
  }
  if (threadIdx.x == 0) {
    float gb = 0.0f, l = 0.0f;
    for (int q = 0; q < kGWarps; ++q) {
      gb += s.gb3[q];
      l += s.loss[q];
    }
    out[kOffB3] = gb;
    out[kGParams] = l;
  }
}

// BF16 copy of parameter p of the packed vector
__device__ __forceinline__ void write_bf16(GuideBf16* wb, int p, float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  if (p < kOffB1) {
    const int j = p / kGIn, k = p % kGIn;
    wb->w1[j * kGFeat + k] = b;
  } else if (p >= kOffW2 && p < kOffB2) {
    const int q = p - kOffW2, j = q / kGHid, k = q % kGHid;
    wb->w2[j * kGHid + k] = b;
    wb->w2t[k * kGHid + j] = b;
  } else if (p >= kOffW3 && p < kOffB3) {
    wb->w3[p - kOffW3] = b;
  }
}

// fold the per-CTA partials in CTA order; lr > 0: one Adam step
// (Kingma & Ba 2015, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) with the bias
// corrections c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
__global__ void k_guide_fold(const float* __restrict__ partials, int nparts, float* __restrict__ grad,
                             float* __restrict__ w, float* __restrict__ m1, float* __restrict__ m2,
                             GuideBf16* __restrict__ wb, float lr, float c1, float c2, float* __restrict__ loss_hist) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kGPartial) return;
  float gsum = 0.0f;
  for (int b = 0; b < nparts; ++b) gsum += partials[(size_t)b * kGPartial + p];
  grad[p] = gsum;
  if (p == kGParams) {
    if (loss_hist) *loss_hist = gsum;
    return;
  }
  if (lr > 0.0f) {
    const float a = 0.9f * m1[p] + 0.1f * gsum;
    const float v = 0.999f * m2[p] + 0.001f * gsum * gsum;
    m1[p] = a;
    m2[p] = v;
    const float wn = w[p] - lr * (a * c1) / (sqrtf(v * c2) + 1e-8f);
    w[p] = wn;
    write_bf16(wb, p, wn);
  }
}

__global__ void k_guide_sync(const float* __restrict__ w, GuideBf16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kGParams) write_bf16(wb, p, w[p]);
}

size_t train_smem() { return sizeof(TrainSmem); }

}  // namespace

namespace pdhgc {

int guide_sync_bf16(pdhgc_guide* g, cudaStream_t st) {
  k_guide_sync<<<(kGParams + 255) / 256, 256, 0, st>>>(g->w, g->wb);
  g->launches++;
  GKL();
  return PDHGC_OK;
}

#ifndef PDHGC_GUIDE_TC
#define PDHGC_GUIDE_TC 1
#endif

int guide_forward(pdhgc_guide* g, const __nv_bfloat16* feat, int64_t rows, float* p, cudaStream_t st) {
  if (rows <= 0) return PDHGC_OK;
#if PDHGC_GUIDE_TC
  // tcgen05: one CTA per SM at most, persistent over 128-row tiles
  const long long tiles = (rows + kTcRows - 1) / kTcRows;
  const long long grid = tiles < g->max_ctas ? tiles : g->max_ctas;
  k_guide_forward_tc<<<(unsigned)grid, kTcRows, sizeof(TcSmem), st>>>(g->wb, g->w, feat, (long long)rows, p, g->err,
                                                                      g->tc_wait_limit);
#else
  const long long tiles = (rows + 15) / 16;
  long long grid = (tiles + kGWarps - 1) / kGWarps;
  if (grid > 152 * 8) grid = 152 * 8;
  k_guide_forward<<<(unsigned)grid, kGThreads, 0, st>>>(g->wb, g->w, feat, (long long)rows, p);
#endif
  g->launches++;
  GKL();
  return PDHGC_OK;
}

int guide_check_error(pdhgc_guide* g, cudaStream_t st) {
  int e = 0;
  GK(cudaMemcpyAsync(&e, g->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GK(cudaStreamSynchronize(st));
  if (e != 0) {
    GK(cudaMemsetAsync(g->err, 0, sizeof(int), st));
    return set_error_detail(PDHGC_ERR_DEVICE, "a bounded tensor-core wait of the network ran out");
  }
  return PDHGC_OK;
}

int guide_step(pdhgc_guide* g, const __nv_bfloat16* feat, const uint8_t* labels, int64_t rows, const int32_t* idx,
               int batch, uint64_t seed, int64_t step, float adam_lr, cudaStream_t st) {
  const int nchunks = (batch + kChunk - 1) / kChunk;
  const int grid = nchunks < g->max_ctas ? nchunks : g->max_ctas;
  k_guide_grad<<<grid, kGThreads, train_smem(), st>>>(g->wb, g->w, feat, labels, (long long)rows, idx, batch,
                                                      (unsigned long long)seed, (long long)step, g->partials);
  g->launches++;
  GKL();
  float c1 = 0.0f, c2 = 0.0f;
  if (adam_lr > 0.0f) {
    g->adam_t++;
    c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)g->adam_t)));
    c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)g->adam_t)));
  }
  k_guide_fold<<<(kGPartial + 255) / 256, 256, 0, st>>>(g->partials, grid, g->grad, g->w, g->m1, g->m2, g->wb,
                                                        adam_lr, c1, c2, nullptr);
  g->launches++;
  GKL();
  return PDHGC_OK;
}

}  // namespace pdhgc

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace {

// He-uniform initial weights from SplitMix64(seed): U(-sqrt(6/fan_in),
// sqrt(6/fan_in)) for W1, W2; U(-sqrt(3/64), sqrt(3/64)) for w3; zero biases
void init_weights_host(uint64_t seed, std::vector<float>& w) {
  w.assign(kGParams, 0.0f);
  uint64_t j = 0;
  auto uni = [&](double a) {
    uint64_t z = seed + (++j) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) * a);
  };
  for (int i = 0; i < kGHid * kGIn; ++i) w[kOffW1 + i] = uni(std::sqrt(6.0 / kGIn));
  for (int i = 0; i < kGHid * kGHid; ++i) w[kOffW2 + i] = uni(std::sqrt(6.0 / kGHid));
  for (int i = 0; i < kGHid; ++i) w[kOffW3 + i] = uni(std::sqrt(3.0 / kGHid));
}

int upload_weights(pdhgc_guide* g, const float* w) {
  GK(cudaMemcpyAsync(g->w, w, sizeof(float) * kGParams, cudaMemcpyHostToDevice, g->stream));
  GK(cudaMemsetAsync(g->m1, 0, sizeof(float) * kGParams, g->stream));
  GK(cudaMemsetAsync(g->m2, 0, sizeof(float) * kGParams, g->stream));
  g->adam_t = 0;
  int rc = guide_sync_bf16(g, g->stream);
  if (rc != PDHGC_OK) return rc;
  GK(cudaStreamSynchronize(g->stream));
  return PDHGC_OK;
}

int check_rows(const void* feat, int64_t rows) {
  if (!feat || rows <= 0) return set_error_detail(PDHGC_ERR_INVALID_ARG, "feature matrix is NULL or rows <= 0");
  if (((uintptr_t)feat & 15u) != 0u)
    return set_error_detail(PDHGC_ERR_INVALID_ARG, "feature matrix must be 16-byte aligned");
  return PDHGC_OK;
}

}  // namespace

extern "C" {

int pdhgc_guide_create(pdhgc_guide** out, uint64_t seed, void* cuda_stream) {
  if (!out) return set_error_detail(PDHGC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  pdhgc_guide* g = new pdhgc_guide();
  g->stream = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    g->max_ctas = nsm > 0 ? nsm : 1;
    e = cudaFuncSetAttribute(k_guide_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem());
  }
  if (e == cudaSuccess) e = cudaMalloc(&g->w, sizeof(float) * kGParams);
  if (e == cudaSuccess) e = cudaMalloc(&g->m1, sizeof(float) * kGParams);
  if (e == cudaSuccess) e = cudaMalloc(&g->m2, sizeof(float) * kGParams);
  if (e == cudaSuccess) e = cudaMalloc(&g->grad, sizeof(float) * kGPartial);
  if (e == cudaSuccess) e = cudaMalloc(&g->wb, sizeof(GuideBf16));
  if (e == cudaSuccess) e = cudaMalloc(&g->partials, sizeof(float) * kGPartial * (size_t)g->max_ctas);
  if (e == cudaSuccess) e = cudaMalloc(&g->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->err, 0, sizeof(int), g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->wb, 0, sizeof(GuideBf16), g->stream);
  if (e != cudaSuccess) {
    pdhgc_guide_destroy(g);
    return set_error_detail(e == cudaErrorMemoryAllocation ? PDHGC_ERR_OOM : PDHGC_ERR_CUDA,
                            std::string("guide create: ") + cudaGetErrorString(e));
  }
  std::vector<float> w;
  init_weights_host(seed, w);
  const int rc = upload_weights(g, w.data());
  if (rc != PDHGC_OK) {
    pdhgc_guide_destroy(g);
    return rc;
  }
  *out = g;
  return PDHGC_OK;
}

void pdhgc_guide_destroy(pdhgc_guide* g) {
  if (!g) return;
  cudaFree(g->w);
  cudaFree(g->m1);
  cudaFree(g->m2);
  cudaFree(g->grad);
  cudaFree(g->wb);
  cudaFree(g->partials);
  cudaFree(g->idx);
  cudaFree(g->err);
  delete g;
}

int pdhgc_guide_set_weights(pdhgc_guide* g, const float* w) {
  if (!g || !w) return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < kGParams; ++i)
    if (!std::isfinite(w[i])) return set_error_detail(PDHGC_ERR_NONFINITE, "weight " + std::to_string(i));
  return upload_weights(g, w);
}

int pdhgc_guide_get_weights(pdhgc_guide* g, float* w) {
  if (!g || !w) return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL argument");
  GK(cudaMemcpyAsync(w, g->w, sizeof(float) * kGParams, cudaMemcpyDeviceToHost, g->stream));
  GK(cudaStreamSynchronize(g->stream));
  return PDHGC_OK;
}

namespace {
constexpr char kGuideMagic[8] = {'P', 'D', 'H', 'G', 'C', 'G', 'W', '1'};

uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

void put_le(unsigned char* d, uint64_t v, int bytes) {
  for (int i = 0; i < bytes; ++i) d[i] = (unsigned char)(v >> (8 * i));
}

uint64_t get_le(const unsigned char* d, int bytes) {
  uint64_t v = 0;
  for (int i = 0; i < bytes; ++i) v |= (uint64_t)d[i] << (8 * i);
  return v;
}
}  // namespace

int pdhgc_guide_save(pdhgc_guide* g, const char* path) {
  if (!g || !path) return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL argument");
  std::vector<float> w(kGParams);
  int rc = pdhgc_guide_get_weights(g, w.data());
  if (rc != PDHGC_OK) return rc;
  std::vector<unsigned char> buf(16 + 4 * (size_t)kGParams + 8);
  std::memcpy(buf.data(), kGuideMagic, 8);
  put_le(buf.data() + 8, (uint64_t)kGParams, 4);
  put_le(buf.data() + 12, 0, 4);
  for (int i = 0; i < kGParams; ++i) {
    uint32_t bits;
    std::memcpy(&bits, &w[i], 4);
    put_le(buf.data() + 16 + 4 * (size_t)i, bits, 4);
  }
  put_le(buf.data() + 16 + 4 * (size_t)kGParams, fnv1a(buf.data() + 16, 4 * (size_t)kGParams), 8);
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error_detail(PDHGC_ERR_IO, std::string("cannot open for writing: ") + path);
  const size_t wrote = std::fwrite(buf.data(), 1, buf.size(), f);
  const int closed = std::fclose(f);
  if (wrote != buf.size() || closed != 0) return set_error_detail(PDHGC_ERR_IO, std::string("write failed: ") + path);
  return PDHGC_OK;
}

int pdhgc_guide_load(pdhgc_guide* g, const char* path) {
  if (!g || !path) return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error_detail(PDHGC_ERR_IO, std::string("cannot open: ") + path);
  std::vector<unsigned char> buf(16 + 4 * (size_t)kGParams + 8 + 1);
  const size_t got = std::fread(buf.data(), 1, buf.size(), f);
  std::fclose(f);
  if (got != buf.size() - 1) return set_error_detail(PDHGC_ERR_IO, "not a guide weight file (size)");
  if (std::memcmp(buf.data(), kGuideMagic, 8) != 0 || get_le(buf.data() + 8, 4) != (uint64_t)kGParams ||
      get_le(buf.data() + 12, 4) != 0)
    return set_error_detail(PDHGC_ERR_IO, "not a guide weight file (header)");
  if (get_le(buf.data() + 16 + 4 * (size_t)kGParams, 8) != fnv1a(buf.data() + 16, 4 * (size_t)kGParams))
    return set_error_detail(PDHGC_ERR_IO, "guide weight file is corrupt (hash)");
  std::vector<float> w(kGParams);
  for (int i = 0; i < kGParams; ++i) {
    const uint32_t bits = (uint32_t)get_le(buf.data() + 16 + 4 * (size_t)i, 4);
    std::memcpy(&w[i], &bits, 4);
  }
  return pdhgc_guide_set_weights(g, w.data());
}

int pdhgc_guide_infer(pdhgc_guide* g, const uint16_t* feat, int64_t rows, float* p) {
  if (!g || !p) return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL argument");
  int rc = check_rows(feat, rows);
  if (rc != PDHGC_OK) return rc;
  rc = guide_forward(g, reinterpret_cast<const __nv_bfloat16*>(feat), rows, p, g->stream);
  if (rc != PDHGC_OK) return rc;
  return guide_check_error(g, g->stream);
}

int pdhgc_guide_grad(pdhgc_guide* g, const uint16_t* feat, const uint8_t* labels, int64_t rows, const int32_t* idx,
                     int batch, float* grad, float* loss) {
  if (!g || !labels || !idx || !grad || batch <= 0)
    return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL argument or batch <= 0");
  int rc = check_rows(feat, rows);
  if (rc != PDHGC_OK) return rc;
  for (int i = 0; i < batch; ++i)
    if (idx[i] < 0 || idx[i] >= rows) return set_error_detail(PDHGC_ERR_INVALID_ARG, "index out of range");
  if (batch > g->idx_cap) {
    cudaFree(g->idx);
    g->idx = nullptr;
    g->idx_cap = 0;
    GK(cudaMalloc(&g->idx, sizeof(int32_t) * (size_t)batch));
    g->idx_cap = batch;
  }
  GK(cudaMemcpyAsync(g->idx, idx, sizeof(int32_t) * (size_t)batch, cudaMemcpyHostToDevice, g->stream));
  rc = guide_step(g, reinterpret_cast<const __nv_bfloat16*>(feat), labels, rows, g->idx, batch, 0, 0, 0.0f,
                  g->stream);
  if (rc != PDHGC_OK) return rc;
  std::vector<float> h(kGPartial);
  GK(cudaMemcpyAsync(h.data(), g->grad, sizeof(float) * kGPartial, cudaMemcpyDeviceToHost, g->stream));
  GK(cudaStreamSynchronize(g->stream));
  std::memcpy(grad, h.data(), sizeof(float) * kGParams);
  if (loss) *loss = h[kGParams];
  return PDHGC_OK;
}

int pdhgc_guide_train(pdhgc_guide* g, const uint16_t* feat, const uint8_t* labels, int64_t rows, int batch,
                      int64_t steps, float lr, uint64_t seed, float* losses) {
  if (!g || !labels || batch <= 0 || steps < 0 || !(lr > 0.0f) || !std::isfinite(lr))
    return set_error_detail(PDHGC_ERR_INVALID_ARG, "NULL labels, batch <= 0, steps < 0 or lr <= 0");
  int rc = check_rows(feat, rows);
  if (rc != PDHGC_OK) return rc;
  float* hist = nullptr;
  if (losses && steps > 0) GK(cudaMallocAsync(&hist, sizeof(float) * (size_t)steps, g->stream));
  for (int64_t s = 0; s < steps; ++s) {
    const int nchunks = (batch + kChunk - 1) / kChunk;
    const int grid = nchunks < g->max_ctas ? nchunks : g->max_ctas;
    k_guide_grad<<<grid, kGThreads, train_smem(), g->stream>>>(
        g->wb, g->w, reinterpret_cast<const __nv_bfloat16*>(feat), labels, (long long)rows, nullptr, batch,
        (unsigned long long)seed, (long long)s, g->partials);
    g->adam_t++;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)g->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)g->adam_t)));
    k_guide_fold<<<(kGPartial + 255) / 256, 256, 0, g->stream>>>(g->partials, grid, g->grad, g->w, g->m1, g->m2,
                                                                 g->wb, lr, c1, c2, hist ? hist + s : nullptr);
    g->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      if (hist) cudaFreeAsync(hist, g->stream);
      return set_error_detail(PDHGC_ERR_CUDA, std::string("guide train launch: ") + cudaGetErrorString(e));
    }
  }
  if (hist) {
    GK(cudaMemcpyAsync(losses, hist, sizeof(float) * (size_t)steps, cudaMemcpyDeviceToHost, g->stream));
    GK(cudaFreeAsync(hist, g->stream));
  }
  GK(cudaStreamSynchronize(g->stream));
  return PDHGC_OK;
}

int64_t pdhgc_guide_kernel_launches(const pdhgc_guide* g) { return g ? g->launches : 0; }

int pdhgc_guide_set_wait_limit(pdhgc_guide* g, int64_t polls) {
  if (!g || polls < 0) return set_error_detail(PDHGC_ERR_INVALID_ARG, "g is NULL or polls < 0");
  g->tc_wait_limit = polls > 0 ? polls : 0;
  return PDHGC_OK;
}

}  // extern "C"
