// Launch interface of the reverse-mode kernels (band_adjoint.cu).  Internal.
#pragma once

#include <cuda_runtime.h>

#include "bp_internal.h"

namespace bpg {

struct AdjArgs {
    const float *logg;      // [H][W][Mp] log g
    const float *ell;       // [4][H][W][Mp] log-messages entering iteration t
    const float *lam_next;  // [4][H][W][Mp] dL/d(messages after iteration t)
    float *lam;             // [4][H][W][Mp] dL/d(messages entering iteration t)
    float *dlogg;           // [H][W][Mp] dL/d log g, accumulated
    float *partial;         // [blocks][2T + 2] per-block sums of dL/df(d) and dL/dfbar
    const float2 *stats;    // [H][W][4] (C, S^) of each message of iteration t, from the recorded forward
    GridDims d;
    int T;
    float w[2 * kTMaxFast + 1];   // f(d) - fbar
    float fbar;
};

int adjoint_blocks(const GridDims &d, Layout lay, int T);
cudaError_t launch_band_log_adjoint(const AdjArgs &a, Layout lay, int blocks, cudaStream_t s);
cudaError_t launch_beliefs_log_adjoint(const float *logg, const float *ell, const float *dlogb, GridDims d,
                                       float *lam, float *dlogg, cudaStream_t s);
cudaError_t launch_reduce_partials_f64(const float *partial, long long rows, int np, double *out, cudaStream_t s);

}  // namespace bpg
