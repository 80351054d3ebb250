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

constexpr int kBlock = 32;             // one warp per block: every shared address is a block constant
constexpr int kMinBlocks = 16;         // resident blocks per SM the registers must allow (128 each)
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

// Walks the nodes of a launch with a stride of `nw` slots.  Slots are the
// nodes in row-major order (synchronous iteration, parity < 0), or of a
// red-black half-step the row-major slots ch of the nodes with
// (r + c) % 2 == parity, c = 2 ch + ((r + parity) & 1).  A step adds the
// stride without a division.
struct NodeWalk {
    int r, ch, dq, dr, row, W, H, parity;
    __device__ __forceinline__ void init(int slot, int nw, int W_, int H_, int parity_) {
        W = W_;
        H = H_;
        parity = parity_;
        row = parity < 0 ? W : (W + 1) >> 1;
        r = slot / row;
        ch = slot - r * row;
        dq = nw / row;
        dr = nw - dq * row;
        settle();
    }
    __device__ __forceinline__ int col() const { return parity < 0 ? ch : 2 * ch + ((r + parity) & 1); }
    __device__ __forceinline__ bool live() const { return r < H; }
    __device__ __forceinline__ void step() {
        ch += dr;
        r += dq;
        if (ch >= row) {
            ch -= row;
            ++r;
        }
    }
    // the last slot of a row of odd width has no node of one parity
    __device__ __forceinline__ void settle() {
        while (r < H && col() >= W) step();
    }
    __device__ __forceinline__ void next() {
        step();
        settle();
    }
};

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

// Sum of four values over the warp, returned to every lane: two exchange
// rounds leave each lane one direction's partial (bits 4 and 3 of the lane),
// three more rounds finish it, four reads broadcast the totals.
__device__ __forceinline__ void warp_sum4(float (&v)[4], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    float k0 = b4 ? v[2] : v[0], k1 = b4 ? v[3] : v[1];
    k0 += __shfl_xor_sync(0xffffffffu, b4 ? v[0] : v[2], 16);
    k1 += __shfl_xor_sync(0xffffffffu, b4 ? v[1] : v[3], 16);
    float k = b3 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, b3 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    v[0] = __shfl_sync(0xffffffffu, k, 0);
    v[1] = __shfl_sync(0xffffffffu, k, 8);
    v[2] = __shfl_sync(0xffffffffu, k, 16);
    v[3] = __shfl_sync(0xffffffffu, k, 24);
}

// Phase 1 for one node: h of the four directions per label (Eq. 5) from the
// staged unary and incoming vectors into the h slice, and the outer terms S
// (sum of h, or its minimum) per direction, this lane's part.  FAST: every
// neighbour present and M == Mp (no masks, no selects).
template <bool MIN, bool FAST>
__device__ __forceinline__ void form_h(const typename Types<MIN>::T *sg, typename Types<MIN>::V *h4, int M, int Mp,
                                       int lane, const bool (&has)[4], typename Types<MIN>::T (&S)[4]) {
    using T = typename Types<MIN>::T;
    using V = typename Types<MIN>::V;
    for (int x0 = 4 * lane; x0 < Mp; x0 += 128) {
        const V gv = *(const V *)(sg + x0);
        V m[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const V in = *(const V *)(sg + (1 + t) * Mp + x0);
            if constexpr (FAST) {
                m[t] = in;
            } else {
                if constexpr (MIN)
                    m[t] = has[t] ? in : make_int4(0, 0, 0, 0);
                else
                    m[t] = has[t] ? in : make_float4(1.f, 1.f, 1.f, 1.f);
            }
        }
        const int sbase = (x0 & ~31) | (lane & 7);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T m0 = comp(m[0], j), m1 = comp(m[1], j), m2 = comp(m[2], j), m3 = comp(m[3], j);
            V hv;
            if constexpr (MIN) {
                // padded labels (never a pattern column) stay out of the minima
                const int32_t tot = (FAST || x0 + j < M) ? comp(gv, j) + m0 + m1 + m2 + m3 : kBigE;
                hv = make_int4(tot - m0, tot - m1, tot - m2, tot - m3);
                S[0] = min(S[0], hv.x);
                S[1] = min(S[1], hv.y);
                S[2] = min(S[2], hv.z);
                S[3] = min(S[3], hv.w);
            } else {
                const float g = (FAST || x0 + j < M) ? comp(gv, j) : 0.f;
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
}

template <int KM, int LM, bool MIN>
__global__ void __launch_bounds__(kBlock, kMinBlocks) sparse_reg_kernel(const SparseRegArgs a) {
    using T = typename Types<MIN>::T;
    using V = typename Types<MIN>::V;
    extern __shared__ __align__(128) unsigned char sr_raw[];
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    const long long plane = a.d.plane;
    const int lane = threadIdx.x;
    const int hslots = Mp < 32 ? 32 : Mp;
    const uint32_t vbytes = (uint32_t)Mp * 4;
    T *stage[2] = {(T *)sr_raw, (T *)sr_raw + 5 * Mp};
    V *h4 = (V *)(sr_raw + (size_t)10 * vbytes);
    uint64_t *bar = (uint64_t *)(sr_raw + (size_t)10 * vbytes + (size_t)hslots * 16);

    // this lane's share of the pattern, once per launch
    T wv[KM * LM];
    uint32_t so[(KM * LM + 1) / 2];
    uint32_t labp[(KM + 1) / 2];   // receiver label of block k in half k % 2 of word k / 2; 0xFFFF: none
    uint32_t real = 0;             // bit k: the label of block k is a label (< M)
#pragma unroll
    for (int i = 0; i < (KM * LM + 1) / 2; ++i) so[i] = 0;
#pragma unroll
    for (int i = 0; i < (KM + 1) / 2; ++i) labp[i] = 0;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const int lk = a.lab[k * 32 + lane];
        labp[k >> 1] |= (uint32_t)(lk < 0 ? 0xFFFF : lk) << ((k & 1) * 16);
        if (lk >= 0 && lk < M) real |= 1u << k;
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
    const bool all_lanes_labelled = Mp >= 32;   // else some lanes own no label

    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // lane 0: node (rr, cc)'s unary and incoming vectors into stage st
    auto issue = [&](int rr, int cc, int st) {
        const long long o = ((long long)rr * W + cc) * Mp;
        mbar_expect_tx(&bar[st], 5 * vbytes);
        bulk_g2s(stage[st], (const T *)a.u + o, vbytes, &bar[st]);
#pragma unroll
        for (int t = 0; t < 4; ++t) bulk_g2s(stage[st] + (1 + t) * Mp, (const T *)a.in + t * plane + o, vbytes, &bar[st]);
    };

    NodeWalk cur;
    cur.init(blockIdx.x, gridDim.x, W, H, a.parity);
    uint32_t ph = 0, pending = 0;
    int st = 0;
    if (cur.live()) {
        if (lane == 0) issue(cur.r, cur.col(), 0);
        pending = 1;
    }
    bool ok = true;
    while (cur.live()) {
        const int r = cur.r, c = cur.col();
        NodeWalk nxt = cur;
        nxt.next();
        if (nxt.live()) {
            // stage st ^ 1 was read by the previous node's phase 1; those reads
            // have returned (their values were consumed) and the warp has
            // synchronised since, so the copies may overwrite it
            __syncwarp();
            if (lane == 0) issue(nxt.r, nxt.col(), st ^ 1);
            pending |= 1u << (st ^ 1);
        }
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], (ph >> st) & 1u));
        if (!ok) break;
        ph ^= 1u << st;
        pending &= ~(1u << st);

        const bool has[4] = {c > 0, c < W - 1, r > 0, r < H - 1};
        T S[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) S[t] = MIN ? (T)kBigE : (T)0;
        if (M == Mp && has[0] && has[1] && has[2] && has[3])
            form_h<MIN, true>(stage[st], h4, M, Mp, lane, has, S);
        else
            form_h<MIN, false>(stage[st], h4, M, Mp, lane, has, S);
        if constexpr (MIN) {
#pragma unroll
            for (int t = 0; t < 4; ++t) S[t] = __reduce_min_sync(0xffffffffu, S[t]);
        } else {
            warp_sum4(S, lane);
        }
        __syncwarp();

        // phase 2: the band of every receiver label this lane owns, from the
        // register pattern; step c outside, so KM independent chains.  A hole
        // reads a slot another lane reads with a value that changes nothing
        // (0 in a sum, 2^29 in a minimum): no branch.
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
                const uint32_t off = (so[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
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

        // combine, normalise (sum: divide by the total; min-sum: subtract the
        // minimum), store into the neighbours' planes
        T Z[4];
        if constexpr (MIN) {
#pragma unroll
            for (int t = 0; t < 4; ++t) Z[t] = kBigE;
#pragma unroll
            for (int k = 0; k < KM; ++k)
                if (real & (1u << k)) {
                    Z[0] = min(Z[0], u[k].x);
                    Z[1] = min(Z[1], u[k].y);
                    Z[2] = min(Z[2], u[k].z);
                    Z[3] = min(Z[3], u[k].w);
                }
#pragma unroll
            for (int t = 0; t < 4; ++t) Z[t] = __reduce_min_sync(0xffffffffu, Z[t]);
        } else {
            // a padded label has no entries: its u stays 0 and adds nothing
#pragma unroll
            for (int k = 0; k < KM; ++k)
                if (real & (1u << k)) {
                    u[k].x = fmaf(a.fbar, S[0], u[k].x);
                    u[k].y = fmaf(a.fbar, S[1], u[k].y);
                    u[k].z = fmaf(a.fbar, S[2], u[k].z);
                    u[k].w = fmaf(a.fbar, S[3], u[k].w);
                }
#pragma unroll
            for (int t = 0; t < 4; ++t) Z[t] = 0.f;
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                Z[0] += u[k].x;
                Z[1] += u[k].y;
                Z[2] += u[k].z;
                Z[3] += u[k].w;
            }
            warp_sum4(Z, lane);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            T *dst = (T *)a.out + dst_offset(t, r, c, W, plane, Mp);
            T scale;
            if constexpr (MIN)
                scale = Z[t];
            else
                scale = __frcp_rn(Z[t]);   // the correctly rounded 1 / Z
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int lk = (labp[k >> 1] >> ((k & 1) * 16)) & 0xFFFF;
                if (all_lanes_labelled || lk != 0xFFFF) {
                    if constexpr (MIN)
                        dst[lk] = (real & (1u << k)) ? comp(u[k], t) - scale : 0;
                    else
                        dst[lk] = comp(u[k], t) * scale;   // padded labels: 0
                }
            }
        }
        __syncwarp();   // the h slice is rewritten by the warp's next node
        st ^= 1;
        cur = nxt;
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
    const size_t smem = warp_smem_bytes(a.d.Mp);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long slots = a.parity < 0 ? (long long)a.d.W * a.d.H : (long long)((a.d.W + 1) / 2) * a.d.H;
    long long b = (long long)device_sm_count() * per_sm;
    if (b > slots) b = slots;
    kern<<<(int)(b < 1 ? 1 : b), kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sr
}  // namespace bpg
