// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): sum-product FP32, family 2 (two 4-label chunks per lane), synchronous.
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_sum_kernel_f2() { return (const void *)batch_kernel<2, false, false>; }
}  // namespace bpg
