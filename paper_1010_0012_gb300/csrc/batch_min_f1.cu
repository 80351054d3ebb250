// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): min-sum int32, family 1 (one 4-label chunk per lane), synchronous.
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_min_kernel_f1() { return (const void *)batch_kernel<1, true, false>; }
}  // namespace bpg
