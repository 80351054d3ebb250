// Launch interface of the sparse-compatibility kernels.  Internal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"

namespace bpg {

// The pattern, interleaved by receiver label: entry i of x_j (the shared-
// memory slot of its sender label x_i, and the value bits) sits at
// ell[i * M + x_j], i < len[x_j].
//
// Slot of label x in the kernels' per-warp h arrays: a rotation by x / 4
// inside each group of four labels.
inline int sp_label_slot(int x) { return (x & ~3) | ((x + (x >> 2)) & 3); }
struct SparseArgsF {
    const float *g;
    const float *in;
    float *out;
    GridDims d;
    int parity;
    const int32_t *len;      // device [M]: compatible sender labels per receiver label
    const int2 *ell;         // device [max len][M]: (slot of x_i, bits of f(x_i, x_j) - fbar)
    float fbar;
};

struct SparseArgsI {
    const int32_t *eu;
    const int32_t *in;
    int32_t *out;
    GridDims d;
    int parity;
    const int32_t *len;
    const int2 *ell;         // (slot of x_i, E(x_i, x_j))
    int32_t ebar;
};

cudaError_t launch_sparse_sum(const SparseArgsF &a, cudaStream_t s);
cudaError_t launch_sparse_min(const SparseArgsI &a, cudaStream_t s);

}  // namespace bpg
