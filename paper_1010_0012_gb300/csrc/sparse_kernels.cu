// O(nnz) message updates for a general sparse-compatibility potential
// (Sec. 4: "the neighborhood structure may be more complicated"; Sec. 7:
// robust potentials that are not functions of x_i - x_j).
//
// The potential is given per receiver label x_j as a list of compatible
// sender labels x_i with values f(x_i, x_j) (CSR over x_j); every other pair
// has the constant fbar.  Then Eq. 7 reads
//   m(x_j) = sum_{x_i in Nbd(x_j)} [f(x_i, x_j) - fbar] h(x_i) + fbar sum_x h(x)
// and Eq. 11 (energies, E <= Ebar)
//   m(x_j) = min( min_{x_i in Nbd(x_j)} [E(x_i, x_j) + h(x_i)], Ebar + min_x h(x) ).
//
// One warp per node: the warp forms the four h vectors in its shared-memory
// slice, reduces S (or min h) with shuffles, and every lane produces the
// outputs x_j = lane, lane + 32, ...  The pattern (column, weight) pairs sit in
// the block's shared memory; each pair is read once for the four directions.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"
#include "bp_sparse.h"

namespace bpg {
namespace {

constexpr int kSpBlock = 256;
constexpr int kSpWarps = kSpBlock / 32;
constexpr int32_t kBigE = 1 << 30;

__device__ __forceinline__ bool sp_slot(int slot, int nslots, int W, int parity, int &r, int &c) {
    if (slot >= nslots) return false;
    if (parity < 0) {
        r = slot / W;
        c = slot - r * W;
        return true;
    }
    const int Wh = (W + 1) >> 1;
    r = slot / Wh;
    c = 2 * (slot - r * Wh) + ((r + parity) & 1);
    return c < W;
}

__device__ __forceinline__ long long sp_dst(int t, int r, int c, int W, long long plane, int Mp) {
    const int dr = (t == 2) ? -1 : (t == 3) ? 1 : 0;
    const int dc = (t == 0) ? -1 : (t == 1) ? 1 : 0;
    return (t ^ 1) * plane + ((long long)(r + dr) * W + (c + dc)) * Mp;
}

__global__ void __launch_bounds__(kSpBlock) sparse_sum_kernel(const SparseArgsF a) {
    extern __shared__ uint8_t sm[];
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    int *rowptr = (int *)sm;                                   // [M + 1]
    int2 *ent = (int2 *)(sm + (((M + 1) * 4 + 15) & ~15));     // [nnz] (column, weight bits)
    float *hs = (float *)((uint8_t *)ent + a.nnz * 8);         // [warps][4][Mp]
    for (int i = threadIdx.x; i <= M; i += kSpBlock) rowptr[i] = a.rowptr[i];
    for (int i = threadIdx.x; i < a.nnz; i += kSpBlock) ent[i] = make_int2(a.cols[i], __float_as_int(a.w[i]));
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *h = hs + warp * 4 * Mp;
    const int nslots = a.parity < 0 ? W * H : ((W + 1) >> 1) * H;
    const int gw = blockIdx.x * kSpWarps + warp, nw = gridDim.x * kSpWarps;
    for (int slot = gw; slot < nslots; slot += nw) {
        int r = 0, c = 0;
        if (!sp_slot(slot, nslots, W, a.parity, r, c)) continue;   // uniform across the warp
        const long long node = (long long)r * W + c;
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        float S[4] = {0.f, 0.f, 0.f, 0.f};
        for (int x = lane; x < Mp; x += 32) {
            const long long o = node * Mp + x;
            float m[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) m[s] = has[s] ? a.in[s * a.d.plane + o] : 1.f;
            const float gv = x < M ? a.g[o] : 0.f;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                float p = gv;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (s != t) p *= m[s];
                h[t * Mp + x] = p;
                S[t] += p;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S[t] += __shfl_xor_sync(0xffffffffu, S[t], o);
        __syncwarp();
        float Z[4] = {0.f, 0.f, 0.f, 0.f};
        float u[4][16];   // Mp <= 512: at most 16 labels per lane
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int xj = lane + 32 * k;
            if (k * 32 >= Mp) break;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            if (xj < M) {
                for (int p = rowptr[xj]; p < rowptr[xj + 1]; ++p) {
                    const int2 e = ent[p];
                    const float wv = __int_as_float(e.y);
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[t] = fmaf(wv, h[t * Mp + e.x], acc[t]);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    acc[t] = fmaf(a.fbar, S[t], acc[t]);
                    Z[t] += acc[t];
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) u[t][k] = acc[t];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) Z[t] += __shfl_xor_sync(0xffffffffu, Z[t], o);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            const float inv = 1.f / Z[t];
            float *dst = a.out + sp_dst(t, r, c, W, a.d.plane, Mp);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int xj = lane + 32 * k;
                if (k * 32 >= Mp) break;
                if (xj < Mp) dst[xj] = xj < M ? u[t][k] * inv : 0.f;
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kSpBlock) sparse_min_kernel(const SparseArgsI a) {
    extern __shared__ uint8_t sm[];
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    int *rowptr = (int *)sm;
    int2 *ent = (int2 *)(sm + (((M + 1) * 4 + 15) & ~15));
    int32_t *hs = (int32_t *)((uint8_t *)ent + a.nnz * 8);
    for (int i = threadIdx.x; i <= M; i += kSpBlock) rowptr[i] = a.rowptr[i];
    for (int i = threadIdx.x; i < a.nnz; i += kSpBlock) ent[i] = make_int2(a.cols[i], a.e[i]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *h = hs + warp * 4 * Mp;
    const int nslots = a.parity < 0 ? W * H : ((W + 1) >> 1) * H;
    const int gw = blockIdx.x * kSpWarps + warp, nw = gridDim.x * kSpWarps;
    for (int slot = gw; slot < nslots; slot += nw) {
        int r = 0, c = 0;
        if (!sp_slot(slot, nslots, W, a.parity, r, c)) continue;
        const long long node = (long long)r * W + c;
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        int32_t hmin[4] = {kBigE, kBigE, kBigE, kBigE};
        for (int x = lane; x < Mp; x += 32) {
            const long long o = node * Mp + x;
            int32_t m[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) m[s] = has[s] ? a.in[s * a.d.plane + o] : 0;
            const int32_t ev = a.eu[o];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                int32_t p = ev;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (s != t) p += m[s];
                p = x < M ? p : kBigE;
                h[t * Mp + x] = p;
                hmin[t] = min(hmin[t], p);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hmin[t] = min(hmin[t], __shfl_xor_sync(0xffffffffu, hmin[t], o));
        __syncwarp();
        int32_t umin[4] = {kBigE, kBigE, kBigE, kBigE};
        int32_t u[4][16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int xj = lane + 32 * k;
            if (k * 32 >= Mp) break;
            int32_t b[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) b[t] = a.ebar + hmin[t];
            if (xj < M) {
                for (int p = rowptr[xj]; p < rowptr[xj + 1]; ++p) {
                    const int2 e = ent[p];
#pragma unroll
                    for (int t = 0; t < 4; ++t) b[t] = min(b[t], e.y + h[t * Mp + e.x]);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) umin[t] = min(umin[t], b[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) u[t][k] = b[t];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) umin[t] = min(umin[t], __shfl_xor_sync(0xffffffffu, umin[t], o));
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            int32_t *dst = a.out + sp_dst(t, r, c, W, a.d.plane, Mp);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int xj = lane + 32 * k;
                if (k * 32 >= Mp) break;
                if (xj < Mp) dst[xj] = xj < M ? u[t][k] - umin[t] : 0;
            }
        }
        __syncwarp();
    }
}

size_t sparse_smem(int M, int Mp, int nnz, int elem) {
    return (size_t)(((M + 1) * 4 + 15) & ~15) + (size_t)nnz * 8 + (size_t)kSpWarps * 4 * Mp * elem;
}

int sparse_blocks(const GridDims &d, int parity, const void *fn, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSpBlock, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long slots = parity < 0 ? (long long)d.W * d.H : (long long)((d.W + 1) / 2) * d.H;
    long long b = (long long)device_sm_count() * per_sm;
    const long long need = (slots + kSpWarps - 1) / kSpWarps;
    if (b > need) b = need;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_sparse_sum(const SparseArgsF &a, cudaStream_t s) {
    const size_t smem = sparse_smem(a.d.M, a.d.Mp, a.nnz, 4);
    cudaError_t e = cudaFuncSetAttribute(sparse_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sparse_sum_kernel<<<sparse_blocks(a.d, a.parity, (const void *)sparse_sum_kernel, smem), kSpBlock, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sparse_min(const SparseArgsI &a, cudaStream_t s) {
    const size_t smem = sparse_smem(a.d.M, a.d.Mp, a.nnz, 4);
    cudaError_t e = cudaFuncSetAttribute(sparse_min_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sparse_min_kernel<<<sparse_blocks(a.d, a.parity, (const void *)sparse_min_kernel, smem), kSpBlock, smem, s>>>(a);
    return cudaGetLastError();
}

size_t sparse_smem_bytes(int M, int Mp, int nnz) { return sparse_smem(M, Mp, nnz, 4); }

}  // namespace bpg
