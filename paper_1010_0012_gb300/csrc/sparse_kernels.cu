// O(nnz) message updates for a general sparse-compatibility potential
// (Sec. 4: "the neighborhood structure may be more complicated"; Sec. 7:
// robust potentials that are not functions of x_i - x_j).
//
// The potential is given per receiver label x_j as a list of compatible
// sender labels x_i with values f(x_i, x_j); every other pair has the
// constant fbar.  Then Eq. 7 reads
//   m(x_j) = sum_{x_i in Nbd(x_j)} [f(x_i, x_j) - fbar] h(x_i) + fbar sum_x h(x)
// and Eq. 11 (energies, E <= Ebar)
//   m(x_j) = min( min_{x_i in Nbd(x_j)} [E(x_i, x_j) + h(x_i)], Ebar + min_x h(x) ).
//
// One warp per node.  Phase 1: lane l forms h for labels 4l .. 4l+3 of every
// 128-label chunk from 16-byte loads of g and the four incoming messages, and
// writes, per label, the four directions' h as one 16-byte vector into the
// warp's shared-memory slice; S (or min h) per direction by shuffles.
// Phase 2: lane l produces the receiver labels x_j = l, l + 32, ...; each
// pattern entry (x_i, value) of x_j costs one 16-byte shared-memory gather of
// h(x_i) for all four directions, and the lane walks the lists of its labels
// side by side (entry i of every label, then entry i + 1).  The pattern is
// stored interleaved by receiver label (entry i of x_j at i * M + x_j:
// consecutive lanes read consecutive words) and read through L1, where it
// stays: every warp of every node reads the same few kilobytes.
//
// Shared-memory banks.  Label x lives in slot sp_label_slot(x) (bp_sparse.h),
// a rotation inside each group of four labels that makes the phase-1 stores
// of a quarter-warp hit eight different 16-byte bank groups.  Where the
// pattern fits, the register-pattern kernels (sparse_reg.cuh) run instead.  The pattern
// holds slots, not labels, and the host orders each receiver label's entries
// so that the eight lanes of a quarter-warp gather from different bank groups
// at each step as far as a matching allows (the order of the terms of a sum
// or a minimum is free).
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

__device__ __forceinline__ float4 ld4_nc(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ int4 ld4_nc(const int32_t *p) { return __ldg(reinterpret_cast<const int4 *>(p)); }
__device__ __forceinline__ float comp(const float4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ int32_t comp(const int4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

// KM = receiver labels per lane (Mp <= 32 KM)
template <int KM>
__global__ void __launch_bounds__(kSpBlock) sparse_sum_kernel(const SparseArgsF a) {
    extern __shared__ float4 sp_h4[];                // [warps][Mp]: h of directions 0..3 per label
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    const long long plane = a.d.plane;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *h4 = sp_h4 + warp * Mp;
    int len[KM], len_max = 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int xj = lane + 32 * k;
        len[k] = xj < M ? a.len[xj] : 0;
        len_max = max(len_max, len[k]);
    }
    const int nslots = a.parity < 0 ? W * H : ((W + 1) >> 1) * H;
    const int gw = blockIdx.x * kSpWarps + warp, nw = gridDim.x * kSpWarps;
    for (int slot = gw; slot < nslots; slot += nw) {
        int r = 0, c = 0;
        if (!sp_slot(slot, nslots, W, a.parity, r, c)) continue;   // uniform across the warp
        const long long node = (long long)r * W + c;
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        float S[4] = {0.f, 0.f, 0.f, 0.f};
        for (int x0 = 4 * lane; x0 < Mp; x0 += 128) {
            const long long o = node * Mp + x0;
            const float4 gv = ld4_nc(a.g + o);
            float4 m[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) m[s] = has[s] ? ld4_nc(a.in + s * plane + o) : make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float g = x0 + j < M ? comp(gv, j) : 0.f;
                const float m0 = comp(m[0], j), m1 = comp(m[1], j), m2 = comp(m[2], j), m3 = comp(m[3], j);
                const float g01 = g * m0 * m1, g23 = g * m2 * m3;
                const float4 hv = make_float4(g23 * m1, g23 * m0, g01 * m3, g01 * m2);
                h4[x0 + ((j + lane + (lane >> 2)) & 3)] = hv;   // slot of label x0 + j (sp_label_slot)
                S[0] += hv.x; S[1] += hv.y; S[2] += hv.z; S[3] += hv.w;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S[t] += __shfl_xor_sync(0xffffffffu, S[t], o);
        __syncwarp();
        float Z[4] = {0.f, 0.f, 0.f, 0.f};
        float4 u[KM];
#pragma unroll
        for (int k = 0; k < KM; ++k) u[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        // entry index outside, receiver labels inside: KM independent
        // load -> gather -> FMA chains in flight per lane
        for (int i = 0; i < len_max; ++i) {
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                if (i < len[k]) {
                    const int2 e = __ldg(a.ell + i * M + lane + 32 * k);
                    const float wv = __int_as_float(e.y);
                    const float4 hv = h4[e.x];
                    u[k].x = fmaf(wv, hv.x, u[k].x);
                    u[k].y = fmaf(wv, hv.y, u[k].y);
                    u[k].z = fmaf(wv, hv.z, u[k].z);
                    u[k].w = fmaf(wv, hv.w, u[k].w);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int xj = lane + 32 * k;
            float4 &acc = u[k];
            if (xj < M) {
                acc.x = fmaf(a.fbar, S[0], acc.x);
                acc.y = fmaf(a.fbar, S[1], acc.y);
                acc.z = fmaf(a.fbar, S[2], acc.z);
                acc.w = fmaf(a.fbar, S[3], acc.w);
                Z[0] += acc.x; Z[1] += acc.y; Z[2] += acc.z; Z[3] += acc.w;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) Z[t] += __shfl_xor_sync(0xffffffffu, Z[t], o);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            const float inv = 1.f / Z[t];
            float *dst = a.out + sp_dst(t, r, c, W, plane, Mp);
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int xj = lane + 32 * k;
                if (xj < Mp) dst[xj] = xj < M ? comp(u[k], t) * inv : 0.f;
            }
        }
        __syncwarp();   // the slice is rewritten by the warp's next node
    }
}

template <int KM>
__global__ void __launch_bounds__(kSpBlock) sparse_min_kernel(const SparseArgsI a) {
    extern __shared__ int4 sp_e4[];                  // [warps][Mp]: h of directions 0..3 per label
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    const long long plane = a.d.plane;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int4 *h4 = sp_e4 + warp * Mp;
    int len[KM], len_max = 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int xj = lane + 32 * k;
        len[k] = xj < M ? a.len[xj] : 0;
        len_max = max(len_max, len[k]);
    }
    const int nslots = a.parity < 0 ? W * H : ((W + 1) >> 1) * H;
    const int gw = blockIdx.x * kSpWarps + warp, nw = gridDim.x * kSpWarps;
    for (int slot = gw; slot < nslots; slot += nw) {
        int r = 0, c = 0;
        if (!sp_slot(slot, nslots, W, a.parity, r, c)) continue;
        const long long node = (long long)r * W + c;
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        int32_t hmin[4] = {kBigE, kBigE, kBigE, kBigE};
        for (int x0 = 4 * lane; x0 < Mp; x0 += 128) {
            const long long o = node * Mp + x0;
            const int4 ev = ld4_nc(a.eu + o);
            int4 m[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) m[s] = has[s] ? ld4_nc(a.in + s * plane + o) : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int32_t m0 = comp(m[0], j), m1 = comp(m[1], j), m2 = comp(m[2], j), m3 = comp(m[3], j);
                // padded labels (never a pattern column) stay out of the minima
                const int32_t tot = x0 + j < M ? comp(ev, j) + m0 + m1 + m2 + m3 : kBigE;
                const int4 hv = make_int4(tot - m0, tot - m1, tot - m2, tot - m3);
                h4[x0 + ((j + lane + (lane >> 2)) & 3)] = hv;   // slot of label x0 + j (sp_label_slot)
                hmin[0] = min(hmin[0], hv.x);
                hmin[1] = min(hmin[1], hv.y);
                hmin[2] = min(hmin[2], hv.z);
                hmin[3] = min(hmin[3], hv.w);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) hmin[t] = min(hmin[t], __shfl_xor_sync(0xffffffffu, hmin[t], o));
        __syncwarp();
        int32_t umin[4] = {kBigE, kBigE, kBigE, kBigE};
        int4 u[KM];
#pragma unroll
        for (int k = 0; k < KM; ++k) u[k] = make_int4(a.ebar + hmin[0], a.ebar + hmin[1], a.ebar + hmin[2], a.ebar + hmin[3]);
        for (int i = 0; i < len_max; ++i) {
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                if (i < len[k]) {
                    const int2 e = __ldg(a.ell + i * M + lane + 32 * k);
                    const int4 hv = h4[e.x];
                    u[k].x = __viaddmin_s32(e.y, hv.x, u[k].x);
                    u[k].y = __viaddmin_s32(e.y, hv.y, u[k].y);
                    u[k].z = __viaddmin_s32(e.y, hv.z, u[k].z);
                    u[k].w = __viaddmin_s32(e.y, hv.w, u[k].w);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int xj = lane + 32 * k;
            const int4 &b = u[k];
            if (xj < M) {
                umin[0] = min(umin[0], b.x);
                umin[1] = min(umin[1], b.y);
                umin[2] = min(umin[2], b.z);
                umin[3] = min(umin[3], b.w);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) umin[t] = min(umin[t], __shfl_xor_sync(0xffffffffu, umin[t], o));
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            int32_t *dst = a.out + sp_dst(t, r, c, W, plane, Mp);
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int xj = lane + 32 * k;
                if (xj < Mp) dst[xj] = xj < M ? comp(u[k], t) - umin[t] : 0;
            }
        }
        __syncwarp();
    }
}

template <typename Fn>
int sparse_blocks(const GridDims &d, int parity, Fn fn, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSpBlock, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long slots = parity < 0 ? (long long)d.W * d.H : (long long)((d.W + 1) / 2) * d.H;
    long long b = (long long)device_sm_count() * per_sm;
    const long long need = (slots + kSpWarps - 1) / kSpWarps;
    if (b > need) b = need;
    return (int)(b < 1 ? 1 : b);
}

template <typename Args, typename Kern>
cudaError_t launch_sp(Kern kern, const Args &a, cudaStream_t s) {
    const size_t smem = (size_t)kSpWarps * a.d.Mp * 16;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<sparse_blocks(a.d, a.parity, kern, smem), kSpBlock, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sparse_sum(const SparseArgsF &a, cudaStream_t s) {
    switch ((a.d.Mp + 31) / 32) {
        case 0: case 1: return launch_sp(sparse_sum_kernel<1>, a, s);
        case 2: return launch_sp(sparse_sum_kernel<2>, a, s);
        case 3: case 4: return launch_sp(sparse_sum_kernel<4>, a, s);
        case 5: case 6: case 7: case 8: return launch_sp(sparse_sum_kernel<8>, a, s);
        default: return a.d.Mp <= 512 ? launch_sp(sparse_sum_kernel<16>, a, s) : cudaErrorInvalidValue;
    }
}

cudaError_t launch_sparse_min(const SparseArgsI &a, cudaStream_t s) {
    switch ((a.d.Mp + 31) / 32) {
        case 0: case 1: return launch_sp(sparse_min_kernel<1>, a, s);
        case 2: return launch_sp(sparse_min_kernel<2>, a, s);
        case 3: case 4: return launch_sp(sparse_min_kernel<4>, a, s);
        case 5: case 6: case 7: case 8: return launch_sp(sparse_min_kernel<8>, a, s);
        default: return a.d.Mp <= 512 ? launch_sp(sparse_min_kernel<16>, a, s) : cudaErrorInvalidValue;
    }
}

}  // namespace bpg
