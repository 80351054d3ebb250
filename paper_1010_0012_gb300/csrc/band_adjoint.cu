// Reverse mode of the log-domain O(mM) sum-product update: launches, the
// reverse of the beliefs and the FP64 reduction.  The kernel itself is in
// band_adjoint.cuh; the label-mask-free instantiations (M == Mp) compile in
// band_adjoint_full.cu.
#include <cuda_runtime.h>

#include "band_adjoint.cuh"

namespace bpg {

const void *adjoint_kernel_full(Layout lay, int T);   // band_adjoint_full.cu

static const void *adjoint_kernel(const GridDims &d, Layout lay, int T) {
    return d.M == d.Mp ? adjoint_kernel_full(lay, T) : pick_kernel<AdjTagT<false>>(lay, T);
}

int adjoint_blocks(const GridDims &d, Layout lay, int T) {
    const void *fn = adjoint_kernel(d, lay, T);
    if (!fn) return 0;
    const int per_block = kBlock / lay.L;
    const long long need = ((long long)d.W * d.H + per_block - 1) / per_block;
    long long b = (long long)device_sm_count() * blocks_per_sm(fn);
    if (b > need) b = need;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_band_log_adjoint(const AdjArgs &a, Layout lay, int blocks, cudaStream_t s) {
    const void *fn = adjoint_kernel(a.d, lay, a.T);
    if (!fn || lay.L * 4 * lay.C != a.d.Mp || blocks < 1) return cudaErrorInvalidValue;
    void *args[] = {const_cast<AdjArgs *>(&a)};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(kBlock), args, 0, s);
}

// ---- reverse of the beliefs (Eq. 3 in logs) ------------------------------------
// log b(x) = a(x) - logsumexp(a), a = log g + sum of incoming l; given
// dL/d log b, da = dlogb - softmax(a) sum_x dlogb.  da seeds dL/d log g and the
// adjoint of every incoming message of the final state.  One warp per node.
__global__ void beliefs_log_adjoint_kernel(const float *logg, const float *ell, const float *dlogb, GridDims d,
                                           float *lam, float *dlogg) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int W = d.W, H = d.H, M = d.M, Mp = d.Mp;
    for (long long node = warp; node < (long long)W * H; node += nwarps) {
        const int r = (int)(node / W), c = (int)(node - (long long)r * W);
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        float amax = -3.0e38f, D = 0.f;
        for (int x = lane; x < M; x += 32) {
            float av = logg[node * Mp + x];
            for (int s = 0; s < 4; ++s)
                if (has[s]) av += ell[s * d.plane + node * Mp + x];
            amax = fmaxf(amax, av);
            D += dlogb[node * M + x];
        }
        for (int o = 16; o > 0; o >>= 1) {
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            D += __shfl_xor_sync(0xffffffffu, D, o);
        }
        float Z = 0.f;
        for (int x = lane; x < M; x += 32) {
            float av = logg[node * Mp + x];
            for (int s = 0; s < 4; ++s)
                if (has[s]) av += ell[s * d.plane + node * Mp + x];
            Z += exp2f(av - amax);
        }
        for (int o = 16; o > 0; o >>= 1) Z += __shfl_xor_sync(0xffffffffu, Z, o);
        for (int x = lane; x < Mp; x += 32) {
            float da = 0.f;
            if (x < M) {
                float av = logg[node * Mp + x];
                for (int s = 0; s < 4; ++s)
                    if (has[s]) av += ell[s * d.plane + node * Mp + x];
                da = dlogb[node * M + x] - exp2f(av - amax) / Z * D;
            }
            dlogg[node * Mp + x] = da;
            for (int s = 0; s < 4; ++s)
                if (has[s]) lam[s * d.plane + node * Mp + x] = da;
        }
    }
}

cudaError_t launch_beliefs_log_adjoint(const float *logg, const float *ell, const float *dlogb, GridDims d,
                                       float *lam, float *dlogg, cudaStream_t s) {
    beliefs_log_adjoint_kernel<<<grid_for((long long)d.W * d.H * 32, 256), 256, 0, s>>>(logg, ell, dlogb, d, lam,
                                                                                       dlogg);
    return cudaGetLastError();
}

// ---- final reduction of the parameter gradients in FP64 ------------------------
// out[j] = sum over rows of partial[row][j], rows = iterations x blocks.
__global__ void reduce_partials_f64_kernel(const float *partial, long long rows, int np, double *out) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < rows; i += blockDim.x) acc += (double)partial[i * np + j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = red[0];
}

cudaError_t launch_reduce_partials_f64(const float *partial, long long rows, int np, double *out, cudaStream_t s) {
    reduce_partials_f64_kernel<<<np, 256, 0, s>>>(partial, rows, np, out);
    return cudaGetLastError();
}

}  // namespace bpg
