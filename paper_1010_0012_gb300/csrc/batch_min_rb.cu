// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): min-sum int32, red-black half-steps (persistent single-grid issue).
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_min_kernel_rb() { return (const void *)batch_kernel<1, true, true>; }
}  // namespace bpg
