// Instantiations of the log-domain sum-product O(mM) kernel (Eq. 7 on
// log-messages).
#include "band_dispatch.cuh"
#include "band_fast.cuh"

namespace bpg {

struct LogTag {
    template <int L, int C, int T>
    static const void *get() { return (const void *)band_sum_kernel<L, C, T, true>; }
};

// M == Mp (every power-of-two label count): the form without label masks
struct LogFullTag {
    template <int L, int C, int T>
    static const void *get() { return (const void *)band_sum_kernel<L, C, T, true, true>; }
};

cudaError_t launch_band_log(const BandArgsLogF &a, Layout lay, int blocks, cudaStream_t s) {
    return a.d.M == a.d.Mp ? launch_fast<LogFullTag>(a, lay, blocks, s) : launch_fast<LogTag>(a, lay, blocks, s);
}

}  // namespace bpg
