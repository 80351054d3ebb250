// Instantiations of the min-sum O(mM) kernel (Eq. 11 in energies).
#include "band_dispatch.cuh"
#include "band_fast.cuh"

namespace bpg {

struct MinTag {
    template <int L, int C, int T>
    static const void *get() { return (const void *)band_min_kernel<L, C, T>; }
};

cudaError_t launch_band_min(const BandArgsI &a, Layout lay, int blocks, cudaStream_t s) {
    return launch_fast<MinTag>(a, lay, blocks, s);
}

}  // namespace bpg
