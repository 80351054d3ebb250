// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): sum-product FP32, family 2, every MRF with M == Mp
// (no padded-label masks).
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_sum_kernel_f2_full() { return (const void *)batch_kernel<2, false, false, true>; }
}  // namespace bpg
