// Register-pattern sparse-compatibility kernels, min-sum (Eq. 11, int32): one instantiation
// per compiled (KM, LM) pair (kept apart from the other mode so the two
// translation units compile in parallel).
#include "sparse_reg.cuh"

namespace bpg {

cudaError_t launch_sparse_reg_min(const SparseRegArgs &a, int KM, int LM, cudaStream_t s) {
    switch (KM * 1000 + LM) {
        case 1016: return sr::launch_reg<1, 16, true, false>(a, s);
        case 1048: return sr::launch_reg<1, 48, true, false>(a, s);
        case 2008: return sr::launch_reg<2, 8, true, false>(a, s);
        case 2012: return sr::launch_reg<2, 12, true, false>(a, s);
        case 2024: return sr::launch_reg<2, 24, true, false>(a, s);
        case 4006: return sr::launch_reg<4, 6, true, false>(a, s);
        case 4009: return sr::launch_reg<4, 9, true, false>(a, s);
        case 4012: return sr::launch_reg<4, 12, true, false>(a, s);
        case 8004: return sr::launch_reg<8, 4, true, false>(a, s);
        case 8006: return sr::launch_reg<8, 6, true, false>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bpg
