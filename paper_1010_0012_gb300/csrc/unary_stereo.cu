// Unary potential of the stereo model formed on the device from the image
// pair (Sec. 6): the right image R is the reference, and label x matches
// pixel (r, c) of R with pixel (r, c + x) of the left image L.  The matching
// cost is the truncated absolute difference
//   cost(r, c, x) = min(|R(r, c) - L(r, c + x)|, Tu),   Tu where c + x >= W,
// an integer in 0..Tu, and the unary is a caller-given table of that cost:
// g = table[cost] (float32, e.g. exp(-beta cost)) or E_u = table[cost]
// (int32).  The table travels by value in the kernel arguments, so the call
// needs no device buffer and no host synchronisation.
//
// One thread writes four consecutive labels of one node as one 16-byte store
// (Mp is a multiple of 4); padded labels (x >= M) get 0, as bp_set_unary
// gives them.  The writes are the whole traffic: W H Mp x 4 bytes, against
// 2 W H bytes of images read (mostly from L1: the threads of a node and of
// its row neighbours read the same bytes of L).
#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"

namespace bpg {
namespace {

template <typename V>
struct CostTable {
    V v[kMaxStereoCost + 1];
};

template <typename V, typename V4>
__global__ void __launch_bounds__(256) unary_stereo_kernel(const uint8_t *__restrict__ left,
                                                           const uint8_t *__restrict__ right, V *__restrict__ out,
                                                           int W, int H, int M, int Mp, int Tu,
                                                           const CostTable<V> table) {
    const int quads = Mp >> 2;
    const long long n = (long long)W * H * quads;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long node = i / quads;
        const int x0 = (int)(i - node * quads) * 4;
        const int r = (int)(node / W), c = (int)(node - (long long)r * W);
        const int ref = right[(long long)r * W + c];
        const uint8_t *row = left + (long long)r * W;
        V o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + j;
            int cost = Tu;
            if (c + x < W) cost = min(abs(ref - (int)row[c + x]), Tu);
            o[j] = x < M ? table.v[cost] : V(0);
        }
        V4 w;
        w.x = o[0]; w.y = o[1]; w.z = o[2]; w.w = o[3];
        reinterpret_cast<V4 *>(out)[i] = w;
    }
}

}  // namespace

cudaError_t launch_unary_stereo_f32(const uint8_t *left, const uint8_t *right, float *out, int W, int H, int M,
                                    int Mp, int Tu, const float *host_table, cudaStream_t s) {
    if (Tu < 0 || Tu > kMaxStereoCost || (Mp & 3)) return cudaErrorInvalidValue;
    CostTable<float> t{};
    for (int k = 0; k <= Tu; ++k) t.v[k] = host_table[k];
    const long long n = (long long)W * H * (Mp >> 2);
    unary_stereo_kernel<float, float4><<<grid_for(n, 256), 256, 0, s>>>(left, right, out, W, H, M, Mp, Tu, t);
    return cudaGetLastError();
}

cudaError_t launch_unary_stereo_i32(const uint8_t *left, const uint8_t *right, int32_t *out, int W, int H, int M,
                                    int Mp, int Tu, const int32_t *host_table, cudaStream_t s) {
    if (Tu < 0 || Tu > kMaxStereoCost || (Mp & 3)) return cudaErrorInvalidValue;
    CostTable<int32_t> t{};
    for (int k = 0; k <= Tu; ++k) t.v[k] = host_table[k];
    const long long n = (long long)W * H * (Mp >> 2);
    unary_stereo_kernel<int32_t, int4><<<grid_for(n, 256), 256, 0, s>>>(left, right, out, W, H, M, Mp, Tu, t);
    return cudaGetLastError();
}

}  // namespace bpg
