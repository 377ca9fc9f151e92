// Corner-guidance network (extension of Algorithm 1, not in the paper):
// an 18 -> 64 -> 64 -> 1 per-column MLP with BF16 weights and activations
// and FP32 accumulation on the tensor cores, its training step and Adam.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace pdhgc {

constexpr int kGIn = 18;      // features per column
constexpr int kGFeat = 32;    // stored feature row: 18 values, then zeros (one 64-byte row)
constexpr int kGHid = 64;     // hidden width
// packed FP32 parameter vector: W1 [64][18], b1 [64], W2 [64][64], b2 [64], w3 [64], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kGHid * kGIn;
constexpr int kOffW2 = kOffB1 + kGHid;
constexpr int kOffB2 = kOffW2 + kGHid * kGHid;
constexpr int kOffW3 = kOffB2 + kGHid;
constexpr int kOffB3 = kOffW3 + kGHid;
constexpr int kGParams = kOffB3 + 1;  // 5441
constexpr int kGPartial = kGParams + 1;  // + the loss

// BF16 copies of the matrices in the layouts the kernels read
struct GuideBf16 {
  __nv_bfloat16 w1[kGHid * kGFeat];   // W1 padded to 32 inputs, row j = unit j
  __nv_bfloat16 w2[kGHid * kGHid];    // W2, row j = unit j of layer 2
  __nv_bfloat16 w2t[kGHid * kGHid];   // W2 transposed (backward data gradient)
  __nv_bfloat16 w3[kGHid];
};

}  // namespace pdhgc

struct pdhgc_guide {
  cudaStream_t stream = nullptr;
  float* w = nullptr;        // FP32 master parameters (packed)
  float* m1 = nullptr;       // Adam first moments
  float* m2 = nullptr;       // Adam second moments
  float* grad = nullptr;     // last folded gradient (packed) + loss
  pdhgc::GuideBf16* wb = nullptr;
  float* partials = nullptr;  // per-CTA partial gradients
  int max_ctas = 0;
  int32_t* idx = nullptr;     // explicit minibatch indices (gradient check)
  int* err = nullptr;         // set by a kernel whose bounded wait ran out
  long long tc_wait_limit = 1ll << 24;  // polls of a tensor-core completion wait before it gives up
  int idx_cap = 0;
  int64_t adam_t = 0;         // Adam steps taken
  int64_t launches = 0;
};

namespace pdhgc {

// forward pass: p[r] = sigmoid(network(feat row r)) for r < rows; feat is
// rows x kGFeat BF16 on the device; p FP32 on the device
int guide_forward(pdhgc_guide* g, const __nv_bfloat16* feat, int64_t rows, float* p, cudaStream_t st);

// the error word of the network's kernels (synchronises st); DEVICE when set
int guide_check_error(pdhgc_guide* g, cudaStream_t st);

// one minibatch gradient (idx != nullptr: explicit device indices; else drawn
// from SplitMix64(seed, step * batch + s) mod rows) folded into g->grad;
// adam_lr > 0 also applies one Adam step
int guide_step(pdhgc_guide* g, const __nv_bfloat16* feat, const uint8_t* labels, int64_t rows,
               const int32_t* idx, int batch, uint64_t seed, int64_t step, float adam_lr, cudaStream_t st);

// refresh the BF16 copies from the FP32 master parameters
int guide_sync_bf16(pdhgc_guide* g, cudaStream_t st);

}  // namespace pdhgc
