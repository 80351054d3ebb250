// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): min-sum int32, family 2 (two 4-label chunks per lane), synchronous.
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_min_kernel_f2() { return (const void *)batch_kernel<2, true, false>; }
}  // namespace bpg
