// One instantiation of the persistent batch kernel per translation unit (they
// compile in parallel): min-sum int32, each MRF on its own class's lane layout, synchronous.
#include "batch_kernels.cuh"

namespace bpg {
const void *batch_min_kernel_mixed() { return (const void *)batch_kernel<0, true, false>; }
}  // namespace bpg
