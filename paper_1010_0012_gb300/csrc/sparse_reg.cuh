// O(nnz) message updates for a general sparse-compatibility potential with the
// pattern held in registers (Sec. 4: Nbd(x_j) of any shape; Sec. 7: robust
// potentials that are not functions of x_i - x_j).  Same mathematics as the
// list kernel (sparse_kernels.cu):
//   m(x_j) = sum_{x_i in Nbd(x_j)} [f(x_i, x_j) - fbar] h(x_i) + fbar sum_x h(x)      (Eq. 7)
//   m(x_j) = min( min_{x_i in Nbd(x_j)} [E(x_i, x_j) + h(x_i)], Ebar + min_x h(x) )   (Eq. 11)
//
// The pattern is the same at every node, so each lane loads its share once
// per launch into registers: lane l of 32-label block k owns one receiver
// label (chosen by the host, see sparse_reg_plan.cu) and, for each step
// c < LM, one entry (byte offset of the sender label's h slot, value) or a
// hole.  The host schedules the entries so that at every step the eight lanes
// of a quarter-warp gather from distinct 16-byte bank groups: each gather is
// one shared-memory wavefront per quarter-warp.
//
// One warp per node.  The node's unary and four incoming vectors arrive by
// bulk copies (cp.async.bulk, completion counted on an mbarrier) into one of
// two per-warp staging buffers: the next node's copies are in flight while the
// current node is computed.  Phase 1 forms h of the four directions per label
// (Eq. 5) from the staging buffer into the warp's h slice, slot
// sr_slot(x) = (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7): the eight lanes of
// a quarter-warp store to eight bank groups.  Phase 2 walks the register
// pattern; the outgoing vectors are normalised in registers and stored
// straight into the neighbours' planes (one 128-byte line per store).
//
// Every wait on the mbarrier is bounded by the global timer; on time-out the
// kernel records status 301, waits (bounded) for its copies still in flight
// and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"
#include "bp_sparse.h"

namespace bpg {
namespace sr {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s
constexpr int32_t kBigE = 1 << 30;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}

// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// slot -> node of a synchronous iteration (parity < 0) or of a red-black half-step
__device__ __forceinline__ bool slot_node(int slot, int nslots, int W, int parity, int &r, int &c) {
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

__device__ __forceinline__ int next_slot(int s, int nslots, int nw, int W, int parity) {
    int r, c;
    while (s < nslots && !slot_node(s, nslots, W, parity, r, c)) s += nw;
    return s;
}

__device__ __forceinline__ long long dst_offset(int t, int r, int c, int W, long long plane, int Mp) {
    const int dr = (t == 2) ? -1 : (t == 3) ? 1 : 0;
    const int dc = (t == 0) ? -1 : (t == 1) ? 1 : 0;
    return (t ^ 1) * plane + ((long long)(r + dr) * W + (c + dc)) * Mp;
}

template <bool MIN>
struct Types;
template <>
struct Types<false> {
    using T = float;
    using V = float4;
};
template <>
struct Types<true> {
    using T = int32_t;
    using V = int4;
};

__device__ __forceinline__ float comp(const float4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ int32_t comp(const int4 &v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

// per-warp shared memory: two staging buffers of 5 vectors, the h slice
// (16 bytes per slot, at least 32 slots), two mbarriers
__host__ __device__ inline size_t warp_smem_bytes(int Mp) {
    const int hslots = Mp < 32 ? 32 : Mp;
    return (size_t)2 * 5 * Mp * 4 + (size_t)hslots * 16 + 16;
}

template <int KM, int LM, bool MIN>
__global__ void __launch_bounds__(kBlock, 2) sparse_reg_kernel(const SparseRegArgs a) {
    using T = typename Types<MIN>::T;
    using V = typename Types<MIN>::V;
    extern __shared__ __align__(128) unsigned char sr_raw[];
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    const long long plane = a.d.plane;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hslots = Mp < 32 ? 32 : Mp;
    const uint32_t vbytes = (uint32_t)Mp * 4;
    unsigned char *wb = sr_raw + (size_t)warp * warp_smem_bytes(Mp);
    T *stage[2] = {(T *)wb, (T *)wb + 5 * Mp};
    V *h4 = (V *)(wb + (size_t)10 * vbytes);
    uint64_t *bar = (uint64_t *)(wb + (size_t)10 * vbytes + (size_t)hslots * 16);

    // this lane's share of the pattern, once per launch
    T wv[KM * LM];
    uint32_t so[(KM * LM + 1) / 2];
    uint32_t labp[(KM + 1) / 2];   // receiver label of block k in half k % 2 of word k / 2; 0xFFFF: none
#pragma unroll
    for (int i = 0; i < (KM * LM + 1) / 2; ++i) so[i] = 0;
#pragma unroll
    for (int i = 0; i < (KM + 1) / 2; ++i) labp[i] = 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int lk = a.lab[k * 32 + lane];
        labp[k >> 1] |= (uint32_t)(lk < 0 ? 0xFFFF : lk) << ((k & 1) * 16);
#pragma unroll
        for (int c = 0; c < LM; ++c) {
            const int i = k * LM + c;
            const int2 e = a.ent[(size_t)i * 32 + lane];
            if constexpr (MIN)
                wv[i] = e.y;
            else
                wv[i] = __int_as_float(e.y);
            so[i >> 1] |= ((uint32_t)e.x & 0xFFFFu) << ((i & 1) * 16);
        }
    }

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();

    const int nslots = a.parity < 0 ? W * H : ((W + 1) >> 1) * H;
    const int nw = gridDim.x * kWarps;
    auto issue = [&](int rr, int cc, int st) {   // lane 0: node (rr, cc)'s unary and incoming vectors into stage st
        const long long o = ((long long)rr * W + cc) * Mp;
        mbar_expect_tx(&bar[st], 5 * vbytes);
        bulk_g2s(stage[st], (const T *)a.u + o, vbytes, &bar[st]);
#pragma unroll
        for (int t = 0; t < 4; ++t) bulk_g2s(stage[st] + (1 + t) * Mp, (const T *)a.in + t * plane + o, vbytes, &bar[st]);
    };

    int cur = next_slot(blockIdx.x * kWarps + warp, nslots, nw, W, a.parity);
    int r = 0, c = 0;
    slot_node(cur, nslots, W, a.parity, r, c);
    uint32_t ph = 0, pending = 0;
    int st = 0;
    if (cur < nslots) {
        if (lane == 0) issue(r, c, 0);
        pending = 1;
    }
    bool ok = true;
    while (cur < nslots) {
        const int nxt = next_slot(cur + nw, nslots, nw, W, a.parity);
        int rn = 0, cn = 0;
        slot_node(nxt, nslots, W, a.parity, rn, cn);
        if (nxt < nslots) {
            // stage st ^ 1 was read by the previous node's phase 1; those reads
            // have returned (their values were consumed) and the warp has
            // synchronised since, so the copies may overwrite it
            __syncwarp();
            if (lane == 0) issue(rn, cn, st ^ 1);
            pending |= 1u << (st ^ 1);
        }
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], (ph >> st) & 1u));
        if (!ok) break;
        ph ^= 1u << st;
        pending &= ~(1u << st);

        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        const T *sg = stage[st];

        // phase 1: h of the four directions per label (Eq. 5), outer terms
        T S[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) S[t] = MIN ? (T)kBigE : (T)0;
        for (int x0 = 4 * lane; x0 < Mp; x0 += 128) {
            const V gv = *(const V *)(sg + x0);
            V m[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if constexpr (MIN)
                    m[t] = has[t] ? *(const V *)(sg + (1 + t) * Mp + x0) : make_int4(0, 0, 0, 0);
                else
                    m[t] = has[t] ? *(const V *)(sg + (1 + t) * Mp + x0) : make_float4(1.f, 1.f, 1.f, 1.f);
            }
            const int sbase = (x0 & ~31) | (lane & 7);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const T m0 = comp(m[0], j), m1 = comp(m[1], j), m2 = comp(m[2], j), m3 = comp(m[3], j);
                V hv;
                if constexpr (MIN) {
                    // padded labels (never a pattern column) stay out of the minima
                    const int32_t tot = x0 + j < M ? comp(gv, j) + m0 + m1 + m2 + m3 : kBigE;
                    hv = make_int4(tot - m0, tot - m1, tot - m2, tot - m3);
                    S[0] = min(S[0], hv.x);
                    S[1] = min(S[1], hv.y);
                    S[2] = min(S[2], hv.z);
                    S[3] = min(S[3], hv.w);
                } else {
                    const float g = x0 + j < M ? comp(gv, j) : 0.f;
                    const float g01 = g * m0 * m1, g23 = g * m2 * m3;
                    hv = make_float4(g23 * m1, g23 * m0, g01 * m3, g01 * m2);
                    S[0] += hv.x;
                    S[1] += hv.y;
                    S[2] += hv.z;
                    S[3] += hv.w;
                }
                h4[sbase + (j << 3)] = hv;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if constexpr (MIN) {
                S[t] = __reduce_min_sync(0xffffffffu, S[t]);
            } else {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) S[t] += __shfl_xor_sync(0xffffffffu, S[t], o);
            }
        }
        __syncwarp();

        // phase 2: the band of every receiver label this lane owns, from the
        // register pattern; step c outside, so KM independent chains
        V u[KM];
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if constexpr (MIN)
                u[k] = make_int4(a.ebar + S[0], a.ebar + S[1], a.ebar + S[2], a.ebar + S[3]);
            else
                u[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const unsigned char *hb = (const unsigned char *)h4;
#pragma unroll
        for (int c2 = 0; c2 < LM; ++c2) {
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int i = k * LM + c2;
                // a hole reads slot 0 with a value that changes nothing (0 in
                // a sum, 2^29 in a minimum): no branch, so the gathers can be
                // issued ahead of their use
                const uint32_t off = (so[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
                {
                    const V hv = *(const V *)(hb + off);
                    if constexpr (MIN) {
                        u[k].x = __viaddmin_s32(wv[i], hv.x, u[k].x);
                        u[k].y = __viaddmin_s32(wv[i], hv.y, u[k].y);
                        u[k].z = __viaddmin_s32(wv[i], hv.z, u[k].z);
                        u[k].w = __viaddmin_s32(wv[i], hv.w, u[k].w);
                    } else {
                        u[k].x = fmaf(wv[i], hv.x, u[k].x);
                        u[k].y = fmaf(wv[i], hv.y, u[k].y);
                        u[k].z = fmaf(wv[i], hv.z, u[k].z);
                        u[k].w = fmaf(wv[i], hv.w, u[k].w);
                    }
                }
            }
        }

        // combine, normalise (sum: divide by the total; min-sum: subtract the
        // minimum), store into the neighbours' planes
        T Z[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) Z[t] = MIN ? (T)kBigE : (T)0;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const int lk = (labp[k >> 1] >> ((k & 1) * 16)) & 0xFFFF;
            if (lk < M) {
                if constexpr (MIN) {
                    Z[0] = min(Z[0], u[k].x);
                    Z[1] = min(Z[1], u[k].y);
                    Z[2] = min(Z[2], u[k].z);
                    Z[3] = min(Z[3], u[k].w);
                } else {
                    u[k].x = fmaf(a.fbar, S[0], u[k].x);
                    u[k].y = fmaf(a.fbar, S[1], u[k].y);
                    u[k].z = fmaf(a.fbar, S[2], u[k].z);
                    u[k].w = fmaf(a.fbar, S[3], u[k].w);
                    Z[0] += u[k].x;
                    Z[1] += u[k].y;
                    Z[2] += u[k].z;
                    Z[3] += u[k].w;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if constexpr (MIN) {
                Z[t] = __reduce_min_sync(0xffffffffu, Z[t]);
            } else {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) Z[t] += __shfl_xor_sync(0xffffffffu, Z[t], o);
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            T *dst = (T *)a.out + dst_offset(t, r, c, W, plane, Mp);
            if constexpr (MIN) {
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int lk = (labp[k >> 1] >> ((k & 1) * 16)) & 0xFFFF;
                    if (lk != 0xFFFF) dst[lk] = lk < M ? comp(u[k], t) - Z[t] : 0;
                }
            } else {
                const float inv = __frcp_rn(Z[t]);   // the correctly rounded 1 / Z
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int lk = (labp[k >> 1] >> ((k & 1) * 16)) & 0xFFFF;
                    if (lk != 0xFFFF) dst[lk] = lk < M ? comp(u[k], t) * inv : 0.f;
                }
            }
        }
        __syncwarp();   // the h slice is rewritten by the warp's next node
        st ^= 1;
        cur = nxt;
        r = rn;
        c = cn;
    }
    if (!ok) {
        if (lane == 0) atomicExch(a.status, 301);
        // copies still in flight land in this warp's staging buffers: wait
        // for them (bounded) before the block's shared memory goes away
        for (int s2 = 0; s2 < 2; ++s2)
            if (pending & (1u << s2)) mbar_wait_bounded(&bar[s2], (ph >> s2) & 1u);
    }
}

template <int KM, int LM, bool MIN>
cudaError_t launch_reg(const SparseRegArgs &a, cudaStream_t s) {
    auto kern = sparse_reg_kernel<KM, LM, MIN>;
    const size_t smem = (size_t)kWarps * warp_smem_bytes(a.d.Mp);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long slots = a.parity < 0 ? (long long)a.d.W * a.d.H : (long long)((a.d.W + 1) / 2) * a.d.H;
    long long b = (long long)device_sm_count() * per_sm;
    const long long need = (slots + kWarps - 1) / kWarps;
    if (b > need) b = need;
    kern<<<(int)(b < 1 ? 1 : b), kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sr
}  // namespace bpg
