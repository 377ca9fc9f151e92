// One instantiation of the batched solver's persistent kernel: double iterates,
// 512 threads per CTA (a translation unit of its own, so that the four
// instantiations compile in parallel).
#include "batch_kernel.cuh"

namespace pdhgc {
template cudaError_t batch_kernel_prepare<double, 512>(size_t, int*);
template cudaError_t batch_kernel_launch<double, 512>(int, size_t, cudaStream_t, const LpDesc*, const int*, int, int*,
                                                  const BatchParams&, int, BatchReport*, BatchReport*);
}  // namespace pdhgc
