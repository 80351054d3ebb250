// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): sum-product FP32, red-black half-steps (persistent single-grid issue).
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_sum_kernel_rb() { return (const void *)batch_kernel<1, false, true>; }
}  // namespace bpg
