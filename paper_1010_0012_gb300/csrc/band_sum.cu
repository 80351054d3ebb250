// Instantiations of the linear sum-product O(mM) kernel (Eq. 7).
#include "band_dispatch.cuh"
#include "band_fast.cuh"

namespace bpg {

struct SumTag {
    template <int L, int C, int T>
    static const void *get() { return (const void *)band_sum_kernel<L, C, T, false>; }
};

cudaError_t launch_band_sum(const BandArgsF &a, Layout lay, int blocks, cudaStream_t s) {
    return launch_fast<SumTag>(a, lay, blocks, s);
}

bool band_fast_available(int Mp, Layout lay, int T) {
    return lay.L * 4 * lay.C == Mp && pick_kernel<SumTag>(lay, T) != nullptr;
}

}  // namespace bpg
