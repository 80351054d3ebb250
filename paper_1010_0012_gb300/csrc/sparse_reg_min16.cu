// Register-pattern sparse-compatibility kernels, min-sum (Eq. 11) on 16-bit
// label pairs (Ebar <= kP16MaxEbar): one instantiation per compiled (KM, LM)
// pair, in a translation unit of its own so it compiles in parallel.
#include "sparse_reg.cuh"

namespace bpg {

cudaError_t launch_sparse_reg_min16(const SparseRegArgs &a, int KM, int LM, cudaStream_t s) {
    switch (KM * 1000 + LM) {
        case 1016: return sr::launch_reg<1, 16, true, true>(a, s);
        case 1048: return sr::launch_reg<1, 48, true, true>(a, s);
        case 2008: return sr::launch_reg<2, 8, true, true>(a, s);
        case 2012: return sr::launch_reg<2, 12, true, true>(a, s);
        case 2024: return sr::launch_reg<2, 24, true, true>(a, s);
        case 4006: return sr::launch_reg<4, 6, true, true>(a, s);
        case 4009: return sr::launch_reg<4, 9, true, true>(a, s);
        case 4012: return sr::launch_reg<4, 12, true, true>(a, s);
        case 8004: return sr::launch_reg<8, 4, true, true>(a, s);
        case 8006: return sr::launch_reg<8, 6, true, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bpg
