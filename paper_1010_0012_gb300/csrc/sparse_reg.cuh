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
// One warp per block works through units of NPW consecutive node slots (one
// node, or two for min-sum up to 128 labels: then the pattern registers, the
// slot-offset extraction, the walk, the wait and the reductions serve two
// nodes, and every step has twice the independent gathers).  A unit's unary
// and four incoming vectors per node arrive by bulk copies (cp.async.bulk,
// completion counted on an mbarrier) into one of two per-warp staging
// buffers: the next unit's copies are in flight while the current unit is
// computed.  Phase 1 forms h of the four directions per label (Eq. 5) from
// the staging buffer into the node's h slice, slot
// (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7): the eight lanes of a
// quarter-warp store to eight bank groups.  Phase 2 walks the register
// pattern; the outgoing vectors are normalised in registers and stored
// straight into the neighbours' planes (one 128-byte line per store).
//
// Min-sum has a 16-bit form (P16) for Ebar <= kP16MaxEbar.  With
// hmin = min_x h(x) and energies in [0, Ebar], a term E + h(x_i) of Eq. 11 can
// beat the flat term Ebar + hmin only if h(x_i) - hmin <= Ebar, so
// m(x_j) - hmin = min( min_{x_i} [E + h'(x_i)], Ebar ) exactly, with
// h' = min(h - hmin, Ebar + 1).  Every operand lies in [0, 2 Ebar + 2]: the
// four directions' h' go into one 8-byte slot as two 16-bit pairs,
// (x & ~63) | ((x & 3) << 4) | ((x >> 2) & 15), gathered by the sixteen lanes
// of a half-warp from distinct 8-byte bank groups, and each step is two
// 16-bit-pair add-min instructions instead of four.  The shift by hmin cancels
// in the normalisation, so the output equals the 32-bit kernel's.
//
// Every wait on the mbarrier is bounded by the global timer; on time-out the
// kernel records status 301, waits (bounded) for its copies still in flight
// and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "bp_internal.h"
#include "bp_sparse.h"

namespace bpg {
namespace sr {

constexpr int kBlock = 32;             // one warp per block: every shared address is a block constant
constexpr int kMinBlocks = 16;         // resident blocks per SM the registers must allow (128 each), one node per warp
constexpr int kMinBlocks2 = 12;        // the same with two nodes per warp (168 registers each)
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

// Walks the nodes of a launch with a stride of nw slots (the grid size).
// Slots are the nodes in row-major order (synchronous iteration, parity < 0),
// or of a red-black half-step the row-major slots ch of the nodes with
// (r + c) % 2 == parity, c = 2 ch + ((r + parity) & 1).  A step adds the
// stride without a division: the slots per row and the stride in rows and
// slots (SparseWalk) are kernel parameters, so only the position lives in
// registers.
inline SparseWalk make_walk(int nw, int W, int parity) {
    SparseWalk w;
    w.row = parity < 0 ? W : (W + 1) >> 1;
    w.dq = nw / w.row;
    w.dr = nw - w.dq * w.row;
    return w;
}

struct NodeWalk {
    int r, ch;
    __device__ __forceinline__ void init(int slot, const SparseWalk &w, int parity) {
        r = slot / w.row;
        ch = slot - r * w.row;
    }
    __device__ __forceinline__ int col(int parity) const { return parity < 0 ? ch : 2 * ch + ((r + parity) & 1); }
    __device__ __forceinline__ bool live(int H) const { return r < H; }
    __device__ __forceinline__ void step(const SparseWalk &w) {
        ch += w.dr;
        r += w.dq;
        if (ch >= w.row) {
            ch -= w.row;
            ++r;
        }
    }
    // the last slot of a row of odd width has no node of one parity
    __device__ __forceinline__ void settle(const SparseWalk &w, int parity, int W, int H) {
        while (r < H && col(parity) >= W) step(w);
    }
    __device__ __forceinline__ void next(const SparseWalk &w, int parity, int W, int H) {
        step(w);
        settle(w, parity, W, H);
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

// bytes of the h slice: 16-byte slots, at least 32; or (P16) 8-byte slots, a
// multiple of 64
__host__ __device__ inline int hslice_bytes(int Mp, bool p16) {
    return p16 ? ((Mp + 63) & ~63) * 8 : (Mp < 32 ? 32 : Mp) * 16;
}

// per-warp shared memory for units of npw nodes: ns staging buffers of
// 5 npw vectors, npw h slices, ns mbarriers
__host__ __device__ inline size_t warp_smem_bytes(int Mp, bool p16, int npw, int ns) {
    return (size_t)ns * npw * 5 * Mp * 4 + (size_t)npw * hslice_bytes(Mp, p16) + (size_t)8 * ns;
}

// Sum of four values over the warp: two exchange rounds leave each lane one
// direction's partial (bits 4 and 3 of the lane), three more rounds finish
// it.  Lane l returns the total of value (l >> 3) & 3; the caller broadcasts
// it (or its reciprocal) from lane 8 t.
__device__ __forceinline__ float warp_sum4_own(const float (&v)[4], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8;
    float k0 = b4 ? v[2] : v[0], k1 = b4 ? v[3] : v[1];
    k0 += __shfl_xor_sync(0xffffffffu, b4 ? v[0] : v[2], 16);
    k1 += __shfl_xor_sync(0xffffffffu, b4 ? v[1] : v[3], 16);
    float k = b3 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, b3 ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
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

// Phase 1 of the 16-bit min-sum form for one node: h of the four directions
// (Eq. 5) in 32 bits for the NC chunks of four labels this lane holds, the
// per-direction minima over the warp (returned in S), then
// h' = min(h - S, Ebar + 1) packed as (t0 | t1 << 16, t2 | t3 << 16).
template <int NC, bool FAST>
__device__ __forceinline__ void form_h16(const int32_t *sg, uint2 *h2, int M, int Mp, int lane,
                                         const bool (&has)[4], int32_t cap, int32_t (&S)[4]) {
    int4 hv[NC][4];
#pragma unroll
    for (int n = 0; n < NC; ++n) {
        const int x0 = 4 * lane + 128 * n;
        if (x0 >= Mp) continue;
        const int4 gv = *(const int4 *)(sg + x0);
        int4 m[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int4 in = *(const int4 *)(sg + (1 + t) * Mp + x0);
            m[t] = (FAST || has[t]) ? in : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int32_t m0 = comp(m[0], j), m1 = comp(m[1], j), m2 = comp(m[2], j), m3 = comp(m[3], j);
            const int32_t tot = (FAST || x0 + j < M) ? comp(gv, j) + m0 + m1 + m2 + m3 : kBigE;
            hv[n][j] = make_int4(tot - m0, tot - m1, tot - m2, tot - m3);
            S[0] = min(S[0], hv[n][j].x);
            S[1] = min(S[1], hv[n][j].y);
            S[2] = min(S[2], hv[n][j].z);
            S[3] = min(S[3], hv[n][j].w);
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) S[t] = __reduce_min_sync(0xffffffffu, S[t]);
#pragma unroll
    for (int n = 0; n < NC; ++n) {
        const int x0 = 4 * lane + 128 * n;
        if (x0 >= Mp) continue;
        const int sbase = (x0 & ~63) | (lane & 15);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t d0 = (uint32_t)min(hv[n][j].x - S[0], cap), d1 = (uint32_t)min(hv[n][j].y - S[1], cap);
            const uint32_t d2 = (uint32_t)min(hv[n][j].z - S[2], cap), d3 = (uint32_t)min(hv[n][j].w - S[3], cap);
            h2[sbase + (j << 4)] = make_uint2(d0 | (d1 << 16), d2 | (d3 << 16));
        }
    }
}

// Sum of eight values over the warp (two nodes' four directions), with the
// exchange tree of warp_sum4 (xor 16, 8, 4, 2, 1): after the tree lane l holds
// the total of value (l >> 2) & 7.  Returns that total; the caller broadcasts
// it (or its reciprocal) from lane 4 j.
__device__ __forceinline__ float warp_sum8_own(const float (&v)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float k[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        k[i] = b4 ? v[i + 4] : v[i];
        k[i] += __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 4], 16);
    }
    float q[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        q[i] = b3 ? k[i + 2] : k[i];
        q[i] += __shfl_xor_sync(0xffffffffu, b3 ? k[i] : k[i + 2], 8);
    }
    float s = b2 ? q[1] : q[0];
    s += __shfl_xor_sync(0xffffffffu, b2 ? q[0] : q[1], 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    return s;
}

// Positions of the NPW consecutive slots of a unit: the walker holds the first
// slot's (r, ch); slot n of the unit is ch + n, wrapping to the next row.
template <int NPW>
struct Unit {
    int r[NPW], c[NPW];
    bool v[NPW];   // the slot is a node of this launch
    __device__ __forceinline__ void of(const NodeWalk &w, const SparseWalk &sw, int parity, int W, int H) {
#pragma unroll
        for (int n = 0; n < NPW; ++n) {
            int rr = w.r, ch = w.ch + n;
            if (ch >= sw.row) {
                ch -= sw.row;
                ++rr;
            }
            const int cc = parity < 0 ? ch : 2 * ch + ((rr + parity) & 1);
            r[n] = rr;
            c[n] = cc;
            v[n] = rr < H && cc < W;
        }
    }
};

// One warp per block computes the NPW nodes of one unit at a time.  With
// NPW = 2 the pattern registers, the slot-offset extraction, the walk, the
// wait and the reductions are shared by two nodes, and every step has twice
// the independent gathers.
template <int KM, int LM, bool MIN, bool P16, int NPW, int NS>
__global__ void __launch_bounds__(kBlock, NPW == 2 ? kMinBlocks2 : kMinBlocks) sparse_reg_kernel(const SparseRegArgs a) {
    static_assert(MIN || !P16, "the 16-bit form is min-sum only");
    static_assert(NPW == 1 || NPW == 2, "one or two nodes per unit");
    static_assert(NS >= 2 && NS <= 4, "two to four stages");
    using T = typename Types<MIN>::T;
    using V = typename Types<MIN>::V;
    using W32 = typename std::conditional<P16, uint32_t, T>::type;   // a register weight
    constexpr int NC = (KM * 32 + 127) / 128;                        // chunks of four labels per lane
    constexpr int kSlice = P16 ? ((KM * 32 + 63) & ~63) * 8 : KM * 32 * 16;   // bytes of one node's h slice
    extern __shared__ __align__(128) unsigned char sr_raw[];
    const int M = a.d.M, Mp = a.d.Mp, W = a.d.W, H = a.d.H;
    const long long plane = a.d.plane;
    const int lane = threadIdx.x;
    const uint32_t vbytes = (uint32_t)Mp * 4;
    T *const stage0 = (T *)sr_raw;                                   // stage s at stage0 + s NPW 5 Mp
    unsigned char *hb = sr_raw + (size_t)NS * NPW * 5 * vbytes;       // node n's slice at hb + n kSlice
    uint64_t *bar = (uint64_t *)(hb + NPW * kSlice);

    // this lane's share of the pattern, once per launch.  FP32 / int32: a
    // weight register per entry, two 16-bit slot offsets per register.
    // 16-bit form: one register per entry, the offset in the low half and E
    // in the high half (E < 2^15).
    constexpr int kSO = P16 ? KM * LM : (KM * LM + 1) / 2;
    W32 wv[P16 ? 1 : KM * LM];
    uint32_t so[kSO];
    uint32_t labp[(KM + 1) / 2];   // receiver label of block k in half k % 2 of word k / 2; 0xFFFF: none
    uint32_t real = 0;             // bit k: the label of block k is a label (< M)
#pragma unroll
    for (int i = 0; i < kSO; ++i) so[i] = 0;
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
            if constexpr (P16) {
                so[i] = ((uint32_t)e.x & 0xFFFFu) | ((uint32_t)e.y & 0xFFFF0000u);
            } else {
                if constexpr (MIN)
                    wv[i] = e.y;
                else
                    wv[i] = __int_as_float(e.y);
                so[i >> 1] |= ((uint32_t)e.x & 0xFFFFu) << ((i & 1) * 16);
            }
        }
    }
    const bool all_lanes_labelled = Mp >= 32;   // else some lanes own no label

    if (lane == 0) {
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2) mbar_init(&bar[s2], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // lane 0: the unit's nodes' unary and incoming vectors into stage st (a
    // unit without nodes arrives with no bytes: the phase completes at once)
    auto issue = [&](const Unit<NPW> &un, int st) {
        uint32_t bytes = 0;
#pragma unroll
        for (int n = 0; n < NPW; ++n) bytes += un.v[n] ? 5 * vbytes : 0;
        mbar_expect_tx(&bar[st], bytes);
#pragma unroll
        for (int n = 0; n < NPW; ++n) {
            if (!un.v[n]) continue;
            const long long o = ((long long)un.r[n] * W + un.c[n]) * Mp;
            T *dst = stage0 + (st * NPW + n) * 5 * Mp;
            bulk_g2s(dst, (const T *)a.u + o, vbytes, &bar[st]);
#pragma unroll
            for (int t = 0; t < 4; ++t) bulk_g2s(dst + (1 + t) * Mp, (const T *)a.in + t * plane + o, vbytes, &bar[st]);
        }
    };

    // a ring of NS stages: unit i is staged in stage i % NS, and while unit
    // i is computed the copies of units i + 1 .. i + NS - 1 are in flight
    NodeWalk cur, ahead;
    cur.init(NPW * blockIdx.x, a.walk, a.parity);
    ahead = cur;
    uint32_t ph = 0, pending = 0;
#pragma unroll
    for (int s2 = 0; s2 < NS - 1; ++s2) {
        if (!ahead.live(H)) break;
        Unit<NPW> un;
        un.of(ahead, a.walk, a.parity, W, H);
        if (lane == 0) issue(un, s2);
        pending |= 1u << s2;
        ahead.step(a.walk);
    }
    int st = 0;
    bool ok = true;
    while (cur.live(H)) {
        Unit<NPW> un;
        un.of(cur, a.walk, a.parity, W, H);
        if (ahead.live(H)) {
            // the stage before st was read by the previous unit's phase 1;
            // those reads have returned (their values were consumed) and the
            // warp has synchronised since, so the copies may overwrite it
            const int is = st == 0 ? NS - 1 : st - 1;
            Unit<NPW> un2;
            un2.of(ahead, a.walk, a.parity, W, H);
            __syncwarp();
            if (lane == 0) issue(un2, is);
            pending |= 1u << is;
            ahead.step(a.walk);
        }
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], (ph >> st) & 1u));
        if (!ok) break;
        ph ^= 1u << st;
        pending &= ~(1u << st);

        bool has[NPW][4];
        bool fast = M == Mp;
#pragma unroll
        for (int n = 0; n < NPW; ++n) {
            has[n][0] = un.c[n] > 0;
            has[n][1] = un.c[n] < W - 1;
            has[n][2] = un.r[n] > 0;
            has[n][3] = un.r[n] < H - 1;
            fast = fast && un.v[n] && has[n][0] && has[n][1] && has[n][2] && has[n][3];
        }
        T S[NPW][4];
#pragma unroll
        for (int n = 0; n < NPW; ++n)
#pragma unroll
            for (int t = 0; t < 4; ++t) S[n][t] = MIN ? (T)kBigE : (T)0;

        // phase 1: h of every node of the unit into its slice, and the outer
        // terms S per node and direction
        if constexpr (P16) {
#pragma unroll
            for (int n = 0; n < NPW; ++n) {
                if (!un.v[n]) continue;
                const int32_t *sg = (const int32_t *)stage0 + (st * NPW + n) * 5 * Mp;
                uint2 *h2 = (uint2 *)(hb + n * kSlice);
                if (fast)
                    form_h16<NC, true>(sg, h2, M, Mp, lane, has[n], a.ebar + 1, S[n]);
                else
                    form_h16<NC, false>(sg, h2, M, Mp, lane, has[n], a.ebar + 1, S[n]);
            }
        } else {
#pragma unroll
            for (int n = 0; n < NPW; ++n) {
                if (!un.v[n]) continue;
                const T *sg = stage0 + (st * NPW + n) * 5 * Mp;
                V *h4 = (V *)(hb + n * kSlice);
                if (fast)
                    form_h<MIN, true>(sg, h4, M, Mp, lane, has[n], S[n]);
                else
                    form_h<MIN, false>(sg, h4, M, Mp, lane, has[n], S[n]);
            }
            if constexpr (MIN) {
#pragma unroll
                for (int n = 0; n < NPW; ++n)
#pragma unroll
                    for (int t = 0; t < 4; ++t) S[n][t] = __reduce_min_sync(0xffffffffu, S[n][t]);
            } else {
                float own;
                if constexpr (NPW == 1)
                    own = warp_sum4_own(S[0], lane);
                else
                    own = warp_sum8_own({S[0][0], S[0][1], S[0][2], S[0][3], S[1][0], S[1][1], S[1][2], S[1][3]},
                                        lane);
#pragma unroll
                for (int n = 0; n < NPW; ++n)
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        S[n][t] = __shfl_sync(0xffffffffu, own, NPW == 1 ? 8 * t : 4 * (4 * n + t));
            }
        }
        __syncwarp();

        // phase 2: the band of every receiver label this lane owns, from the
        // register pattern; step c outside, so KM x NPW independent chains.
        // A hole reads a slot another lane reads with a value that changes
        // nothing (0 in a sum, 2^29 or Ebar + 1 in a minimum): no branch.
        // Then combine, normalise (sum: multiply by the correctly rounded
        // 1 / total; min-sum: subtract the minimum) and store into the
        // neighbours' planes, one 128-byte line per store.
        if constexpr (P16) {
            // 16-bit pairs: u01 holds directions 0 and 1, u23 directions 2
            // and 3, starting at the flat term Ebar (h' has minimum 0)
            uint32_t u01[NPW][KM], u23[NPW][KM];
            const uint32_t flat = (uint32_t)a.ebar | ((uint32_t)a.ebar << 16);
#pragma unroll
            for (int n = 0; n < NPW; ++n)
#pragma unroll
                for (int k = 0; k < KM; ++k) u01[n][k] = u23[n][k] = flat;
#pragma unroll
            for (int c2 = 0; c2 < LM; ++c2) {
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int i = k * LM + c2;
                    const uint32_t off = so[i] & 0xFFFFu;
                    const uint32_t w2 = __byte_perm(so[i], 0u, 0x3232);   // E in both halves
#pragma unroll
                    for (int n = 0; n < NPW; ++n) {
                        const uint2 hv = *(const uint2 *)(hb + n * kSlice + off);
                        u01[n][k] = __viaddmin_s16x2(w2, hv.x, u01[n][k]);
                        u23[n][k] = __viaddmin_s16x2(w2, hv.y, u23[n][k]);
                    }
                }
            }
            // the shift by min h cancels in the normalisation
#pragma unroll
            for (int n = 0; n < NPW; ++n) {
                if (!un.v[n]) continue;
                int32_t Z[4] = {kBigE, kBigE, kBigE, kBigE};
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (real & (1u << k)) {
                        Z[0] = min(Z[0], (int32_t)(u01[n][k] & 0xFFFFu));
                        Z[1] = min(Z[1], (int32_t)(u01[n][k] >> 16));
                        Z[2] = min(Z[2], (int32_t)(u23[n][k] & 0xFFFFu));
                        Z[3] = min(Z[3], (int32_t)(u23[n][k] >> 16));
                    }
#pragma unroll
                for (int t = 0; t < 4; ++t) Z[t] = __reduce_min_sync(0xffffffffu, Z[t]);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (!has[n][t]) continue;
                    int32_t *dst = (int32_t *)a.out + dst_offset(t, un.r[n], un.c[n], W, plane, Mp);
#pragma unroll
                    for (int k = 0; k < KM; ++k) {
                        const int lk = (labp[k >> 1] >> ((k & 1) * 16)) & 0xFFFF;
                        const uint32_t pr = t < 2 ? u01[n][k] : u23[n][k];
                        const int32_t v = (int32_t)((t & 1) ? pr >> 16 : pr & 0xFFFFu);
                        if (all_lanes_labelled || lk != 0xFFFF) dst[lk] = (real & (1u << k)) ? v - Z[t] : 0;
                    }
                }
            }
        } else {
            V u[NPW][KM];
#pragma unroll
            for (int n = 0; n < NPW; ++n)
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if constexpr (MIN)
                        u[n][k] = make_int4(a.ebar + S[n][0], a.ebar + S[n][1], a.ebar + S[n][2], a.ebar + S[n][3]);
                    else
                        u[n][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
            for (int c2 = 0; c2 < LM; ++c2) {
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int i = k * LM + c2;
                    const uint32_t off = (so[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
#pragma unroll
                    for (int n = 0; n < NPW; ++n) {
                        const V hv = *(const V *)(hb + n * kSlice + off);
                        if constexpr (MIN) {
                            u[n][k].x = __viaddmin_s32(wv[i], hv.x, u[n][k].x);
                            u[n][k].y = __viaddmin_s32(wv[i], hv.y, u[n][k].y);
                            u[n][k].z = __viaddmin_s32(wv[i], hv.z, u[n][k].z);
                            u[n][k].w = __viaddmin_s32(wv[i], hv.w, u[n][k].w);
                        } else {
                            u[n][k].x = fmaf(wv[i], hv.x, u[n][k].x);
                            u[n][k].y = fmaf(wv[i], hv.y, u[n][k].y);
                            u[n][k].z = fmaf(wv[i], hv.z, u[n][k].z);
                            u[n][k].w = fmaf(wv[i], hv.w, u[n][k].w);
                        }
                    }
                }
            }
            T scale[NPW][4];
            if constexpr (MIN) {
#pragma unroll
                for (int n = 0; n < NPW; ++n) {
#pragma unroll
                    for (int t = 0; t < 4; ++t) scale[n][t] = kBigE;
#pragma unroll
                    for (int k = 0; k < KM; ++k)
                        if (real & (1u << k)) {
                            scale[n][0] = min(scale[n][0], u[n][k].x);
                            scale[n][1] = min(scale[n][1], u[n][k].y);
                            scale[n][2] = min(scale[n][2], u[n][k].z);
                            scale[n][3] = min(scale[n][3], u[n][k].w);
                        }
#pragma unroll
                    for (int t = 0; t < 4; ++t) scale[n][t] = __reduce_min_sync(0xffffffffu, scale[n][t]);
                }
            } else {
                // a padded label has no entries: its u stays 0 and adds nothing
                float Z[NPW][4];
#pragma unroll
                for (int n = 0; n < NPW; ++n) {
#pragma unroll
                    for (int k = 0; k < KM; ++k)
                        if (real & (1u << k)) {
                            u[n][k].x = fmaf(a.fbar, S[n][0], u[n][k].x);
                            u[n][k].y = fmaf(a.fbar, S[n][1], u[n][k].y);
                            u[n][k].z = fmaf(a.fbar, S[n][2], u[n][k].z);
                            u[n][k].w = fmaf(a.fbar, S[n][3], u[n][k].w);
                        }
#pragma unroll
                    for (int t = 0; t < 4; ++t) Z[n][t] = 0.f;
#pragma unroll
                    for (int k = 0; k < KM; ++k) {
                        Z[n][0] += u[n][k].x;
                        Z[n][1] += u[n][k].y;
                        Z[n][2] += u[n][k].z;
                        Z[n][3] += u[n][k].w;
                    }
                }
                // each lane takes the correctly rounded reciprocal of the one
                // total it holds; the reciprocals are broadcast
                float own;
                if constexpr (NPW == 1)
                    own = warp_sum4_own(Z[0], lane);
                else
                    own = warp_sum8_own({Z[0][0], Z[0][1], Z[0][2], Z[0][3], Z[1][0], Z[1][1], Z[1][2], Z[1][3]},
                                        lane);
                const float rz = __frcp_rn(own);
#pragma unroll
                for (int n = 0; n < NPW; ++n)
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        scale[n][t] = __shfl_sync(0xffffffffu, rz, NPW == 1 ? 8 * t : 4 * (4 * n + t));
            }
#pragma unroll
            for (int n = 0; n < NPW; ++n) {
                if (!un.v[n]) continue;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (!has[n][t]) continue;
                    T *dst = (T *)a.out + dst_offset(t, un.r[n], un.c[n], W, plane, Mp);
#pragma unroll
                    for (int k = 0; k < KM; ++k) {
                        const int lk = (labp[k >> 1] >> ((k & 1) * 16)) & 0xFFFF;
                        if (all_lanes_labelled || lk != 0xFFFF) {
                            if constexpr (MIN)
                                dst[lk] = (real & (1u << k)) ? comp(u[n][k], t) - scale[n][t] : 0;
                            else
                                dst[lk] = comp(u[n][k], t) * scale[n][t];   // padded labels: 0
                        }
                    }
                }
            }
        }
        __syncwarp();   // the h slices are rewritten by the warp's next unit
        st = st + 1 == NS ? 0 : st + 1;
        cur.step(a.walk);
    }
    if (!ok) {
        if (lane == 0) atomicExch(a.status, 301);
        // copies still in flight land in this warp's staging buffers: wait
        // for them (bounded) before the block's shared memory goes away
        for (int s2 = 0; s2 < NS; ++s2)
            if (pending & (1u << s2)) mbar_wait_bounded(&bar[s2], (ph >> s2) & 1u);
    }
}

// Nodes per unit: two for min-sum up to 128 labels, one for sum-product and
// at 256 labels (measured on the 1280 x 720, M = 128 workload: min-sum runs
// faster with two, sum-product as fast with one; at 256 the staging buffers
// and slices of two nodes leave room for too few warps).  Two stages: a third
// speeds up the copies alone but not the kernel, whose shared-memory gathers
// (16 or 8 bytes per entry) then bound it.
template <int KM, bool MIN>
constexpr int units_of() {
    return MIN && KM <= 4 ? 2 : 1;
}

template <int KM, int LM, bool MIN, bool P16>
cudaError_t launch_reg(const SparseRegArgs &args, cudaStream_t s) {
    constexpr int NPW = units_of<KM, MIN>(), NS = 2;
    auto kern = sparse_reg_kernel<KM, LM, MIN, P16, NPW, NS>;
    const size_t smem = warp_smem_bytes(args.d.Mp, P16, NPW, NS);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    SparseRegArgs a = args;
    const long long slots = a.parity < 0 ? (long long)a.d.W * a.d.H : (long long)((a.d.W + 1) / 2) * a.d.H;
    const long long units = (slots + NPW - 1) / NPW;
    long long b = (long long)device_sm_count() * per_sm;
    if (b > units) b = units;
    if (b < 1) b = 1;
    a.walk = make_walk((int)b * NPW, a.d.W, a.parity);
    kern<<<(int)b, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sr
}  // namespace bpg
