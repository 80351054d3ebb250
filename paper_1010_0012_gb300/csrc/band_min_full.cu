// Instantiations of the min-sum O(mM) kernel without padded-label masks
// (M == Mp), compiled apart from the masked ones in band_min.cu.
#include "band_dispatch.cuh"
#include "band_fast.cuh"

namespace bpg {

struct MinFullTag {
    template <int L, int C, int T>
    static const void *get() { return (const void *)band_min_kernel<L, C, T, true>; }
};

const void *band_min_full_kernel(Layout lay, int T) { return pick_kernel<MinFullTag>(lay, T); }

}  // namespace bpg
