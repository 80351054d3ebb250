// Label-mask-free instantiations (M == Mp) of the adjoint kernel, compiled
// apart from the masked ones so that the two halves build in parallel.
#include "band_adjoint.cuh"

namespace bpg {
const void *adjoint_kernel_full(Layout lay, int T) { return pick_kernel<AdjTagT<true>>(lay, T); }
}  // namespace bpg
