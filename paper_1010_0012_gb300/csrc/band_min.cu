// Instantiations of the min-sum O(mM) kernel (Eq. 11 in energies).
#include <algorithm>

#include "band_dispatch.cuh"
#include "band_fast.cuh"

namespace bpg {

struct MinTag {
    template <int L, int C, int T>
    static const void *get() { return (const void *)band_min_kernel<L, C, T>; }
};

const void *band_min_full_kernel(Layout lay, int T);   // band_min_full.cu

// M == Mp: the variant without padded-label masks, launched on the grid of
// the masked variant.  Without the masks the wider bands need fewer
// registers (T = 4, two chunks per lane: 80 instead of 110), and the third
// resident block that would allow made the HBM stream slower (0.90 against
// 1.00 of HBM at M = 128); the masked variant's occupancy is the measured one.
cudaError_t launch_band_min(const BandArgsI &a, Layout lay, int blocks, cudaStream_t s) {
    if (a.d.M != a.d.Mp) return launch_fast<MinTag>(a, lay, blocks, s);
    if (lay.L * 4 * lay.C != a.d.Mp) return cudaErrorInvalidValue;
    const void *full = band_min_full_kernel(lay, a.T), *masked = pick_kernel<MinTag>(lay, a.T);
    if (!full || !masked) return cudaErrorInvalidValue;
    const int per_block = kBlock / lay.L;
    const long long need = (slots_of(a.d, a.parity) + per_block - 1) / per_block;
    if (blocks <= 0) blocks = device_sm_count() * std::min(blocks_per_sm(full), blocks_per_sm(masked));
    if (blocks > need) blocks = (int)need;
    if (blocks < 1) blocks = 1;
    void *args[] = {const_cast<BandArgsI *>(&a)};
    return cudaLaunchKernel(full, dim3(blocks), dim3(kBlock), args, 0, s);
}

}  // namespace bpg
