// Launch interface of the sparse-compatibility kernels.  Internal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"

namespace bpg {

struct SparseArgsF {
    const float *g;
    const float *in;
    float *out;
    GridDims d;
    int parity;
    const int32_t *rowptr;   // device [M + 1], over receiver labels x_j
    const int32_t *cols;     // device [nnz], sender labels x_i
    const float *w;          // device [nnz], f(x_i, x_j) - fbar
    int nnz;
    float fbar;
};

struct SparseArgsI {
    const int32_t *eu;
    const int32_t *in;
    int32_t *out;
    GridDims d;
    int parity;
    const int32_t *rowptr;
    const int32_t *cols;
    const int32_t *e;        // device [nnz], E(x_i, x_j)
    int nnz;
    int32_t ebar;
};

cudaError_t launch_sparse_sum(const SparseArgsF &a, cudaStream_t s);
cudaError_t launch_sparse_min(const SparseArgsI &a, cudaStream_t s);
size_t sparse_smem_bytes(int M, int Mp, int nnz);

}  // namespace bpg
