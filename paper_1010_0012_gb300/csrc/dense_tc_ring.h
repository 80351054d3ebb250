// Launch interface of the tensor-core O(M^2) kernels for Mp = 256
// (dense_tc_ring.cu), where a whole 128-row A tile no longer fits beside F^T
// in shared memory and the pipeline moves 64-label K-blocks instead.  Internal.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "bp_internal.h"

namespace bpg {

// packed form: A = [rows][256] BF16 h rows (tensor map, box 128 x 64), B = F^T
// (tensor map, box 256 x 64); out [rows][256] FP32, each row normalised
cudaError_t launch_gemm_ring256(const CUtensorMap &map_a, const CUtensorMap &map_b, float *out, long long rows,
                                int *status, cudaStream_t s);

// fused form: h formed on chip from g and the incoming planes ([..][256])
cudaError_t launch_fused_ring256(const CUtensorMap &map_b, const float *g, const float *in, float *out,
                                 const GridDims &d, int *status, cudaStream_t s);

}  // namespace bpg
