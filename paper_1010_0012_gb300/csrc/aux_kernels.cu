// Shared-memory O(mM) kernels for any band width, the dense O(M^2) CUDA-core
// baselines, beliefs / MAP, and the layout helpers (padding, fills).
#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"

namespace bpg {

namespace {

constexpr int kGenBlock = 256;
constexpr int kGenWarps = kGenBlock / 32;
constexpr int32_t kBig = 1 << 30;

// SM count per device ordinal (a process may drive several devices)
int g_sm_count[kMaxDevices] = {};

// Sum (or min) of four per-thread values over the block; every thread gets
// the result.  `red` holds kGenWarps * 4 entries.
template <bool MIN, typename E>
__device__ __forceinline__ void block_reduce4(E (&v)[4], E *red) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const E x = __shfl_xor_sync(0xffffffffu, v[t], o);
            v[t] = MIN ? (x < v[t] ? x : v[t]) : v[t] + x;
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int t = 0; t < 4; ++t) red[warp * 4 + t] = v[t];
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        E acc = red[t];
        for (int k = 1; k < kGenWarps; ++k) {
            const E x = red[k * 4 + t];
            acc = MIN ? (x < acc ? x : acc) : acc + x;
        }
        v[t] = acc;
    }
}

__device__ __forceinline__ void node_of(int slot, int W, int parity, int &r, int &c) {
    if (parity < 0) {
        r = slot / W;
        c = slot - r * W;
    } else {
        const int Wh = (W + 1) >> 1;
        r = slot / Wh;
        c = 2 * (slot - r * Wh) + ((r + parity) & 1);
    }
}

__device__ __forceinline__ long long dst_offset(int t, int r, int c, int W, long long plane, int Mp) {
    const int dr = (t == 2) ? -1 : (t == 3) ? 1 : 0;
    const int dc = (t == 0) ? -1 : (t == 1) ? 1 : 0;
    return (t ^ 1) * plane + ((long long)(r + dr) * W + (c + dc)) * Mp;
}

// One block per node.  DENSE: the full sum of Eq. 2 with the M x M table;
// otherwise the band form Eq. 7 with any T.
template <bool DENSE>
__global__ void __launch_bounds__(kGenBlock)
sum_generic_kernel(const float *g, const float *in, float *out, GridDims d, int parity, int T,
                   const float *wtab, float fbar) {
    extern __shared__ float sm[];
    const int Mp = d.Mp, M = d.M, W = d.W, H = d.H;
    float *hs = sm;              // [4][Mp]
    float *us = sm + 4 * Mp;     // [4][Mp]
    float *red = sm + 8 * Mp;    // [kGenWarps * 4]
    const int nslots = parity < 0 ? W * H : ((W + 1) >> 1) * H;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        int r, c;
        node_of(slot, W, parity, r, c);
        if (c >= W) continue;   // uniform across the block
        const long long node = (long long)r * W + c;
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        float s4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int x = threadIdx.x; x < Mp; x += kGenBlock) {
            const long long o = node * Mp + x;
            float m[4];
            for (int s = 0; s < 4; ++s) m[s] = has[s] ? in[s * d.plane + o] : 1.f;
            const float gv = x < M ? g[o] : 0.f;
            for (int t = 0; t < 4; ++t) {
                float p = gv;
                for (int s = 0; s < 4; ++s)
                    if (s != t) p *= m[s];
                hs[t * Mp + x] = p;
                s4[t] += p;
            }
        }
        block_reduce4<false>(s4, red);   // S_t (contains the barrier after hs writes)
        float z4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int xj = threadIdx.x; xj < M; xj += kGenBlock) {
            for (int t = 0; t < 4; ++t) {
                float acc = 0.f;
                if (DENSE) {
                    for (int xi = 0; xi < M; ++xi) acc = fmaf(wtab[(long long)xi * M + xj], hs[t * Mp + xi], acc);
                } else {
                    const int lo = max(-T, -xj), hi = min(T, M - 1 - xj);
                    for (int dd = lo; dd <= hi; ++dd) acc = fmaf(wtab[dd + T], hs[t * Mp + xj + dd], acc);
                    acc = fmaf(fbar, s4[t], acc);
                }
                us[t * Mp + xj] = acc;
                z4[t] += acc;
            }
        }
        block_reduce4<false>(z4, red);
        for (int x = threadIdx.x; x < Mp; x += kGenBlock)
            for (int t = 0; t < 4; ++t)
                if (has[t]) out[dst_offset(t, r, c, W, d.plane, Mp) + x] = x < M ? us[t * Mp + x] / z4[t] : 0.f;
        __syncthreads();
    }
}

template <bool DENSE>
__global__ void __launch_bounds__(kGenBlock)
min_generic_kernel(const int32_t *e, const int32_t *in, int32_t *out, GridDims d, int parity, int T,
                   const int32_t *wtab, int32_t ebar) {
    extern __shared__ int32_t smi[];
    const int Mp = d.Mp, M = d.M, W = d.W, H = d.H;
    int32_t *hs = smi;
    int32_t *us = smi + 4 * Mp;
    int32_t *red = smi + 8 * Mp;
    const int nslots = parity < 0 ? W * H : ((W + 1) >> 1) * H;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        int r, c;
        node_of(slot, W, parity, r, c);
        if (c >= W) continue;
        const long long node = (long long)r * W + c;
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        int32_t h4[4] = {kBig, kBig, kBig, kBig};
        for (int x = threadIdx.x; x < Mp; x += kGenBlock) {
            const long long o = node * Mp + x;
            int32_t m[4];
            for (int s = 0; s < 4; ++s) m[s] = has[s] ? in[s * d.plane + o] : 0;
            const int32_t ev = e[o];
            for (int t = 0; t < 4; ++t) {
                int32_t p = ev;
                for (int s = 0; s < 4; ++s)
                    if (s != t) p += m[s];
                p = x < M ? p : kBig;
                hs[t * Mp + x] = p;
                h4[t] = min(h4[t], p);
            }
        }
        block_reduce4<true>(h4, red);
        int32_t z4[4] = {kBig, kBig, kBig, kBig};
        for (int xj = threadIdx.x; xj < M; xj += kGenBlock) {
            for (int t = 0; t < 4; ++t) {
                int32_t b = kBig;
                if (DENSE) {
                    for (int xi = 0; xi < M; ++xi) b = min(b, wtab[(long long)xi * M + xj] + hs[t * Mp + xi]);
                } else {
                    const int lo = max(-T, -xj), hi = min(T, M - 1 - xj);
                    for (int dd = lo; dd <= hi; ++dd) b = min(b, wtab[dd + T] + hs[t * Mp + xj + dd]);
                    b = min(b, ebar + h4[t]);
                }
                us[t * Mp + xj] = b;
                z4[t] = min(z4[t], b);
            }
        }
        block_reduce4<true>(z4, red);
        for (int x = threadIdx.x; x < Mp; x += kGenBlock)
            for (int t = 0; t < 4; ++t)
                if (has[t]) out[dst_offset(t, r, c, W, d.plane, Mp) + x] = x < M ? us[t * Mp + x] - z4[t] : 0;
        __syncthreads();
    }
}

// ---- beliefs (Eq. 3) and MAP: one warp per node -----------------------------
__global__ void beliefs_f32_kernel(const float *g, const float *planes, GridDims d, int log_domain,
                                   float *out, int32_t *map) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int W = d.W, H = d.H, M = d.M, Mp = d.Mp;
    for (long long node = warp; node < (long long)W * H; node += nwarps) {
        const int r = (int)(node / W), c = (int)(node - (long long)r * W);
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        // pass 1: maximum of the (log) product, for the log-domain normaliser
        float amax = -3.0e38f;
        if (log_domain) {
            for (int x = lane; x < M; x += 32) {
                float a = g[node * Mp + x];
                for (int s = 0; s < 4; ++s)
                    if (has[s]) a += planes[s * d.plane + node * Mp + x];
                amax = fmaxf(amax, a);
            }
            for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
        float Z = 0.f;
        for (int x = lane; x < M; x += 32) {
            float b;
            if (log_domain) {
                float a = g[node * Mp + x];
                for (int s = 0; s < 4; ++s)
                    if (has[s]) a += planes[s * d.plane + node * Mp + x];
                b = exp2f(a - amax);
            } else {
                b = g[node * Mp + x];
                for (int s = 0; s < 4; ++s)
                    if (has[s]) b *= planes[s * d.plane + node * Mp + x];
            }
            Z += b;
        }
        for (int o = 16; o > 0; o >>= 1) Z += __shfl_xor_sync(0xffffffffu, Z, o);
        const float logZ = log_domain ? amax + log2f(Z) : 0.f;   // base 2
        float best = -3.0e38f;
        int besti = 0x7fffffff;
        for (int x = lane; x < M; x += 32) {
            float b;
            if (log_domain) {
                float a = g[node * Mp + x];
                for (int s = 0; s < 4; ++s)
                    if (has[s]) a += planes[s * d.plane + node * Mp + x];
                b = (a - logZ) * 0.693147180559945309f;   // natural log-belief
            } else {
                b = g[node * Mp + x];
                for (int s = 0; s < 4; ++s)
                    if (has[s]) b *= planes[s * d.plane + node * Mp + x];
                b = b / Z;
            }
            out[node * M + x] = b;
            if (b > best) { best = b; besti = x; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
            if (ob > best || (ob == best && oi < besti)) { best = ob; besti = oi; }
        }
        if (map && lane == 0) map[node] = besti;
    }
}

__global__ void beliefs_i32_kernel(const int32_t *e, const int32_t *planes, GridDims d, int32_t *out,
                                   int32_t *map) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int W = d.W, H = d.H, M = d.M, Mp = d.Mp;
    for (long long node = warp; node < (long long)W * H; node += nwarps) {
        const int r = (int)(node / W), c = (int)(node - (long long)r * W);
        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        int32_t best = 0x7fffffff;
        int besti = 0x7fffffff;
        for (int x = lane; x < M; x += 32) {
            int32_t b = e[node * Mp + x];
            for (int s = 0; s < 4; ++s)
                if (has[s]) b += planes[s * d.plane + node * Mp + x];
            out[node * M + x] = b;
            if (b < best) { best = b; besti = x; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
            if (ob < best || (ob == best && oi < besti)) { best = ob; besti = oi; }
        }
        if (map && lane == 0) map[node] = besti;
    }
}

// ---- layout helpers ----------------------------------------------------------
// transform of one value: 0 copy, 1 log, 2 exp, 3 natural log -> base-2 log
__device__ __forceinline__ float pad_transform(float v, int lg) {
    if (lg == 1) return logf(v);
    if (lg == 2) return expf(v);
    if (lg == 3) return v * 1.44269504088896341f;
    return v;
}

__global__ void pad_f32_kernel(const float *src, float *dst, long long nodes, int M, int Mp, int lg) {
    const long long n = nodes * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long node = i / Mp;
        const int x = (int)(i - node * Mp);
        dst[i] = x < M ? pad_transform(src[node * M + x], lg) : 0.f;
    }
}

// M == Mp and 16-byte aligned buffers: the same values, 16 bytes per thread
// and step, no index division
__global__ void pad_f32_vec_kernel(const float4 *src, float4 *dst, long long n4, int lg) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = src[i];
        dst[i] = make_float4(pad_transform(v.x, lg), pad_transform(v.y, lg), pad_transform(v.z, lg),
                             pad_transform(v.w, lg));
    }
}

// log g into the handle in one read: base-2 log g (transform 3) and g
// (transform 2), each value as the two single passes compute it
__global__ void log_unary_kernel(const float *src, float *dst_log2, float *dst_lin, long long nodes, int M, int Mp) {
    const long long n = nodes * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long node = i / Mp;
        const int x = (int)(i - node * Mp);
        const float v = x < M ? src[node * M + x] : 0.f;
        dst_log2[i] = x < M ? pad_transform(v, 3) : 0.f;
        dst_lin[i] = x < M ? pad_transform(v, 2) : 0.f;
    }
}

__global__ void log_unary_vec_kernel(const float4 *src, float4 *dst_log2, float4 *dst_lin, long long n4) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = src[i];
        dst_log2[i] = make_float4(pad_transform(v.x, 3), pad_transform(v.y, 3), pad_transform(v.z, 3),
                                  pad_transform(v.w, 3));
        dst_lin[i] = make_float4(pad_transform(v.x, 2), pad_transform(v.y, 2), pad_transform(v.z, 2),
                                 pad_transform(v.w, 2));
    }
}

__global__ void pad_i32_kernel(const int32_t *src, int32_t *dst, long long nodes, int M, int Mp) {
    const long long n = nodes * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long node = i / Mp;
        const int x = (int)(i - node * Mp);
        dst[i] = x < M ? src[node * M + x] : 0;
    }
}

__global__ void unpad_kernel(const int32_t *src, int32_t *dst, long long rows, int M, int Mp) {
    const long long n = rows * M;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long row = i / M;
        const int x = (int)(i - row * M);
        dst[i] = src[row * Mp + x];
    }
}

template <typename E>
__global__ void fill_kernel(E *planes, long long rows, int M, int Mp, E value) {
    const long long n = rows * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mp);
        planes[i] = x < M ? value : E(0);
    }
}

}  // namespace

int grid_for(long long n, int block) {
    long long b = (n + block - 1) / block;
    const long long cap = (long long)device_sm_count() * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int *slot = dev < kMaxDevices ? &g_sm_count[dev] : nullptr;
    if (slot && *slot > 0) return *slot;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    if (slot) *slot = n;
    return n;
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    return dev;
}

int padded_labels(int M) {
    if (M <= 512) {
        int Mp = 4;
        while (Mp < M) Mp <<= 1;
        return Mp;
    }
    return (M + 3) & ~3;
}

int layouts_for(int Mp, Layout *out, int max_out) {
    static const Layout all[] = {{1, 1}, {2, 1}, {4, 1}, {2, 2}, {8, 1}, {4, 2}, {16, 1},
                                 {8, 2}, {32, 1}, {16, 2}, {32, 2}, {16, 4}, {32, 4}};
    int n = 0;
    // default first: two 4-label chunks per lane where compiled (measured on
    // GB300: 8 labels per lane keep enough loads in flight to reach 0.95-0.99 of
    // HBM at M = 32..128, against 0.89-0.96 with 4), then the rest by C
    for (int pref : {2, 1, 4})
        for (const Layout &l : all) {
            if (l.L * 4 * l.C != Mp || l.C != pref) continue;
            if (n < max_out) out[n] = l;
            ++n;
        }
    return n;
}

static size_t generic_smem(int Mp) { return (size_t)(8 * Mp + kGenWarps * 4) * 4; }

static int generic_blocks(const GridDims &d, int parity) {
    const long long slots = parity < 0 ? (long long)d.W * d.H : (long long)((d.W + 1) / 2) * d.H;
    long long b = (long long)device_sm_count() * 8;
    if (b > slots) b = slots;
    return (int)(b < 1 ? 1 : b);
}

static cudaError_t set_generic_smem(const void *fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_band_sum_generic(const BandArgsGenericF &a, cudaStream_t s) {
    const size_t sm = generic_smem(a.d.Mp);
    cudaError_t e = set_generic_smem((const void *)sum_generic_kernel<false>, sm);
    if (e != cudaSuccess) return e;
    sum_generic_kernel<false><<<generic_blocks(a.d, a.parity), kGenBlock, sm, s>>>(
        a.g, a.in, a.out, a.d, a.parity, a.T, a.w, a.fbar);
    return cudaGetLastError();
}

cudaError_t launch_band_min_generic(const BandArgsGenericI &a, cudaStream_t s) {
    const size_t sm = generic_smem(a.d.Mp);
    cudaError_t e = set_generic_smem((const void *)min_generic_kernel<false>, sm);
    if (e != cudaSuccess) return e;
    min_generic_kernel<false><<<generic_blocks(a.d, a.parity), kGenBlock, sm, s>>>(
        a.e, a.in, a.out, a.d, a.parity, a.T, a.w, a.ebar);
    return cudaGetLastError();
}

cudaError_t launch_dense_sum(const DenseArgsF &a, cudaStream_t s) {
    const size_t sm = generic_smem(a.d.Mp);
    cudaError_t e = set_generic_smem((const void *)sum_generic_kernel<true>, sm);
    if (e != cudaSuccess) return e;
    sum_generic_kernel<true><<<generic_blocks(a.d, -1), kGenBlock, sm, s>>>(a.g, a.in, a.out, a.d, -1, 0,
                                                                           a.F, 0.f);
    return cudaGetLastError();
}

cudaError_t launch_dense_min(const DenseArgsI &a, cudaStream_t s) {
    const size_t sm = generic_smem(a.d.Mp);
    cudaError_t e = set_generic_smem((const void *)min_generic_kernel<true>, sm);
    if (e != cudaSuccess) return e;
    min_generic_kernel<true><<<generic_blocks(a.d, -1), kGenBlock, sm, s>>>(a.e, a.in, a.out, a.d, -1, 0,
                                                                           a.V, 0);
    return cudaGetLastError();
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

cudaError_t launch_pad_copy_f32(const float *src, float *dst, long long nodes, int M, int Mp, int log_transform,
                                cudaStream_t s) {
    const long long n = nodes * Mp;
    if (M == Mp && (n & 3) == 0 && aligned16(src) && aligned16(dst))
        pad_f32_vec_kernel<<<grid_for(n / 4, 256), 256, 0, s>>>((const float4 *)src, (float4 *)dst, n / 4,
                                                                 log_transform);
    else
        pad_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst, nodes, M, Mp, log_transform);
    return cudaGetLastError();
}

cudaError_t launch_log_unary(const float *src, float *dst_log2, float *dst_lin, long long nodes, int M, int Mp,
                             cudaStream_t s) {
    const long long n = nodes * Mp;
    if (M == Mp && (n & 3) == 0 && aligned16(src) && aligned16(dst_log2) && aligned16(dst_lin))
        log_unary_vec_kernel<<<grid_for(n / 4, 256), 256, 0, s>>>((const float4 *)src, (float4 *)dst_log2,
                                                                   (float4 *)dst_lin, n / 4);
    else
        log_unary_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, dst_log2, dst_lin, nodes, M, Mp);
    return cudaGetLastError();
}

cudaError_t launch_pad_copy_i32(const int32_t *src, int32_t *dst, long long nodes, int M, int Mp, cudaStream_t s) {
    pad_i32_kernel<<<grid_for(nodes * Mp, 256), 256, 0, s>>>(src, dst, nodes, M, Mp);
    return cudaGetLastError();
}

cudaError_t launch_unpad_copy(const void *src, void *dst, long long rows, int M, int Mp, cudaStream_t s) {
    unpad_kernel<<<grid_for(rows * M, 256), 256, 0, s>>>((const int32_t *)src, (int32_t *)dst, rows, M, Mp);
    return cudaGetLastError();
}

cudaError_t launch_fill_messages_f32(float *planes, long long rows, int M, int Mp, float value, cudaStream_t s) {
    fill_kernel<float><<<grid_for(rows * Mp, 256), 256, 0, s>>>(planes, rows, M, Mp, value);
    return cudaGetLastError();
}

cudaError_t launch_fill_messages_i32(int32_t *planes, long long rows, int M, int Mp, int32_t value,
                                     cudaStream_t s) {
    fill_kernel<int32_t><<<grid_for(rows * Mp, 256), 256, 0, s>>>(planes, rows, M, Mp, value);
    return cudaGetLastError();
}

cudaError_t launch_beliefs_f32(const float *g, const float *planes, GridDims d, int log_domain, float *out,
                               int32_t *map, cudaStream_t s) {
    beliefs_f32_kernel<<<grid_for((long long)d.W * d.H * 32, 256), 256, 0, s>>>(g, planes, d, log_domain, out, map);
    return cudaGetLastError();
}

cudaError_t launch_beliefs_i32(const int32_t *e, const int32_t *planes, GridDims d, int32_t *out, int32_t *map,
                               cudaStream_t s) {
    beliefs_i32_kernel<<<grid_for((long long)d.W * d.H * 32, 256), 256, 0, s>>>(e, planes, d, out, map);
    return cudaGetLastError();
}

}  // namespace bpg

// ---- linear <-> log conversions ------------------------------------------------
// The log domain of the library is base 2 throughout (messages, log g, the
// recorded states): the log-domain kernels then take h from one hardware 2^x
// of an exact argument and store one hardware log2.  Natural logs appear only
// at the boundary (bp_set_unary_log, log-beliefs, gradients).
namespace bpg {
namespace {
__global__ void convert_kernel(float *p, long long rows, int M, int Mp, int to_log) {
    const long long n = rows * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mp);
        p[i] = x < M ? (to_log ? log2f(p[i]) : exp2f(p[i])) : 0.f;
    }
}
__global__ void log_copy_kernel(const float *g, float *lg, long long nodes, int M, int Mp) {
    const long long n = nodes * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mp);
        lg[i] = x < M ? log2f(g[i]) : 0.f;
    }
}
// Message planes [4][H][W][Mp] -> [4][H][W][M]; slots without a neighbour
// (never read by any update) come out as 0, the log domain (base 2) as linear.
__global__ void unpad_messages_kernel(const int32_t *src, int32_t *dst, int W, int H, int M, int Mp, int exp2_log) {
    const long long n = 4LL * W * H * M;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long row = i / M;
        const int x = (int)(i - row * M);
        const int pl = (int)(row / ((long long)W * H));
        const long long node = row - (long long)pl * W * H;
        const int r = (int)(node / W), c = (int)(node - (long long)r * W);
        const bool has = pl == 0 ? c > 0 : pl == 1 ? c < W - 1 : pl == 2 ? r > 0 : r < H - 1;
        int32_t v = 0;
        if (has) {
            v = src[row * Mp + x];
            if (exp2_log) v = __float_as_int(exp2f(__int_as_float(v)));
        }
        dst[i] = v;
    }
}

__global__ void convert_dense_kernel(float *p, long long n, int to_log) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = to_log ? log2f(p[i]) : exp2f(p[i]);
}
}  // namespace

cudaError_t launch_domain_convert(float *planes, long long rows, int M, int Mp, int to_log, cudaStream_t s) {
    convert_kernel<<<grid_for(rows * Mp, 256), 256, 0, s>>>(planes, rows, M, Mp, to_log);
    return cudaGetLastError();
}
cudaError_t launch_domain_convert_copy(const float *g, float *logg, long long nodes, int M, int Mp, cudaStream_t s) {
    log_copy_kernel<<<grid_for(nodes * Mp, 256), 256, 0, s>>>(g, logg, nodes, M, Mp);
    return cudaGetLastError();
}
cudaError_t launch_unpad_messages(const void *src, void *dst, int W, int H, int M, int Mp, int exp2_log,
                                  cudaStream_t s) {
    unpad_messages_kernel<<<grid_for(4LL * W * H * M, 256), 256, 0, s>>>((const int32_t *)src, (int32_t *)dst, W, H,
                                                                         M, Mp, exp2_log);
    return cudaGetLastError();
}
cudaError_t launch_domain_convert_dense(float *p, long long n, int to_log, cudaStream_t s) {
    convert_dense_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n, to_log);
    return cudaGetLastError();
}
}  // namespace bpg
