// Register-pattern sparse-compatibility kernels, sum-product (Eq. 7, FP32): one instantiation
// per compiled (KM, LM) pair (kept apart from the other mode so the two
// translation units compile in parallel).
#include "sparse_reg.cuh"

namespace bpg {

cudaError_t launch_sparse_reg_sum(const SparseRegArgs &a, int KM, int LM, cudaStream_t s) {
    switch (KM * 1000 + LM) {
        case 1016: return sr::launch_reg<1, 16, false, false>(a, s);
        case 1048: return sr::launch_reg<1, 48, false, false>(a, s);
        case 2008: return sr::launch_reg<2, 8, false, false>(a, s);
        case 2012: return sr::launch_reg<2, 12, false, false>(a, s);
        case 2024: return sr::launch_reg<2, 24, false, false>(a, s);
        case 4006: return sr::launch_reg<4, 6, false, false>(a, s);
        case 4009: return sr::launch_reg<4, 9, false, false>(a, s);
        case 4012: return sr::launch_reg<4, 12, false, false>(a, s);
        case 8004: return sr::launch_reg<8, 4, false, false>(a, s);
        case 8006: return sr::launch_reg<8, 6, false, false>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bpg
