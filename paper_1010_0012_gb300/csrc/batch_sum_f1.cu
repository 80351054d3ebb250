// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): sum-product FP32, family 1 (one 4-label chunk per lane), synchronous.
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_sum_kernel_f1() { return (const void *)batch_kernel<1, false, false>; }
}  // namespace bpg
