// O(mM) message update kernels, register/shuffle form (band half-width T <= 8).
//
// One group of L lanes handles one node; lane q of the group holds the V = 4C
// consecutive labels [qV, qV + V) of every vector of that node.  Per node the
// group reads the unary and the four incoming messages once (5 x Mp words),
// forms the four products h of Eq. 5 in registers, and writes the four outgoing
// messages (4 x Mp words) straight into the neighbours' incoming planes:
//
//   sum-product (Eq. 7):
//     S      = sum_x h(x)                        (group shuffle reduction)
//     B(x_j) = sum_{|d| <= T} [f(d) - fbar] h(x_j + d)   (band; halo via shuffles)
//     u(x_j) = B(x_j) + fbar S,  m(x_j) = u(x_j) / sum_x u(x)
//   min-sum (Eq. 11 in energies):
//     Hmin   = min_x h(x)
//     u(x_j) = min( min_{|d| <= T} [E(d) + h(x_j + d)], Ebar + Hmin ),  m = u - min_x u
//
// The band is clipped to the labels [0, M) (a label outside has no h).  The
// normaliser sum_x u(x) of Eq. 7 is obtained without a second pass over u:
//   sum_{x_j} B(x_j) = sum_{x_i} h(x_i) c(x_i),  c(x_i) = sum of f(d) - fbar over
//   the d that keep x_j = x_i - d inside [0, M),
// so sum_x u = sum_x h(x) (c(x) + M fbar), reduced together with S.
//
// The log-domain form keeps messages and log g as base-2 logs: h is
// 2^(log2 g + sum of log2-messages - their maximum), one hardware ex2 of an
// exact argument, and the stored message is the hardware log2 of m (absolute
// error about 2^-22).  The results are the linear form's within about 1e-6.

#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"

namespace bpg {

#define BPG_FULL 0xffffffffu
constexpr int32_t kIntBig = 1 << 30;   // "no label" energy, far above any message
constexpr float kLogNone = -1.0e30f;   // "no label" log-value

// ---------------------------------------------------------------- vectors ----
template <int V>
__device__ __forceinline__ void ld_vec(float (&v)[V], const float *p) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + i);
        v[4 * i + 0] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
}
template <int V>
__device__ __forceinline__ void ld_vec(int32_t (&v)[V], const int32_t *p) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i) {
        const int4 t = __ldg(reinterpret_cast<const int4 *>(p) + i);
        v[4 * i + 0] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
}
template <int V>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[V]) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i)
        reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
template <int V>
__device__ __forceinline__ void st_vec(int32_t *p, const int32_t (&v)[V]) {
#pragma unroll
    for (int i = 0; i < V / 4; ++i)
        reinterpret_cast<int4 *>(p)[i] = make_int4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
template <int V, typename T>
__device__ __forceinline__ void fill_vec(T (&v)[V], T x) {
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = x;
}

// minimum of a register vector, three-input DPX minimum where it pairs up
template <int V>
__device__ __forceinline__ int32_t min_vec(const int32_t (&v)[V]) {
    int32_t r = v[0];
#pragma unroll
    for (int k = 1; k + 1 < V; k += 2) r = __vimin3_s32(r, v[k], v[k + 1]);
    if (V % 2 == 0) r = min(r, v[V - 1]);
    return r;
}

// 2^x by the hardware approximation (ex2.approx.ftz: about 2 ulp; results
// below 2^-126 flush to 0).  The log-domain kernels work in base 2, so the
// max-shifted argument is exact and this is the whole exp.
__device__ __forceinline__ float exp2_hw(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------- group reductions ----
template <int L>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(BPG_FULL, v, o);
    return v;
}
template <int L>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(BPG_FULL, v, o));
    return v;
}
template <int L>
__device__ __forceinline__ int32_t group_min(int32_t v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(BPG_FULL, v, o));
    return v;
}

// Band window: win[T + j] = h(qV + j) for j in [-T, V + T), taken from the
// neighbouring lanes of the group; labels outside [0, L*V) get `none`.
template <int L, int V, int T, typename E>
__device__ __forceinline__ void band_window(E (&win)[V + 2 * T], const E (&h)[V], int q, E none) {
#pragma unroll
    for (int k = 0; k < V; ++k) win[T + k] = h[k];
#pragma unroll
    for (int j = 1; j <= T; ++j) {               // label offset -j
        const int delta = (j + V - 1) / V;       // source lane q - delta
        const int idx = delta * V - j;           // its register
        E v = none;
        if (L > 1) {
            v = __shfl_up_sync(BPG_FULL, h[idx], delta, L);
            if (q < delta) v = none;
        }
        win[T - j] = v;
    }
#pragma unroll
    for (int j = 0; j < T; ++j) {                // label offset V + j
        const int delta = (V + j) / V;           // source lane q + delta
        const int idx = V + j - delta * V;
        E v = none;
        if (L > 1) {
            v = __shfl_down_sync(BPG_FULL, h[idx], delta, L);
            if (q + delta >= L) v = none;
        }
        win[T + V + j] = v;
    }
}

// Node of slot `slot` for a synchronous sweep (parity < 0) or a red-black
// half-step (nodes with (r + c) % 2 == parity).  Returns false past the end.
__device__ __forceinline__ bool slot_node(int slot, int nslots, int W, int parity, int &r, int &c) {
    r = 0;
    c = 0;
    if (slot >= nslots) return false;
    if (parity < 0) {
        r = slot / W;
        c = slot - r * W;
        return true;
    }
    const int Wh = (W + 1) >> 1;
    r = slot / Wh;
    c = 2 * (slot - r * Wh) + ((r + parity) & 1);
    if (c >= W) { c = 0; return false; }
    return true;
}

__device__ __forceinline__ int num_slots(int W, int H, int parity) {
    return parity < 0 ? W * H : ((W + 1) >> 1) * H;
}

// Outgoing direction t: 0 to the left neighbour (stored in its plane 1),
// 1 to the right (plane 0), 2 up (plane 3), 3 down (plane 2).  Eq. 5 leaves
// out the message that came from that neighbour, i.e. incoming plane t.
__device__ __forceinline__ long long out_offset(int t, int r, int c, int W, long long plane, int Mp) {
    const int dst_plane = t ^ 1;
    const int dr = (t == 2) ? -1 : (t == 3) ? 1 : 0;
    const int dc = (t == 0) ? -1 : (t == 1) ? 1 : 0;
    return dst_plane * plane + ((long long)(r + dr) * W + (c + dc)) * Mp;
}

// Message loads: read-only ("nc") when the messages were written by an earlier
// launch; coherent at L2 ("cg") inside a persistent launch whose other blocks
// wrote them.
template <bool COH, int V>
__device__ __forceinline__ void ld_msg(float (&v)[V], const float *p) {
    if (COH) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            const float4 t = __ldcg(reinterpret_cast<const float4 *>(p) + i);
            v[4 * i + 0] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else {
        ld_vec<V>(v, p);
    }
}
template <bool COH, int V>
__device__ __forceinline__ void ld_msg(int32_t (&v)[V], const int32_t *p) {
    if (COH) {
#pragma unroll
        for (int i = 0; i < V / 4; ++i) {
            const int4 t = __ldcg(reinterpret_cast<const int4 *>(p) + i);
            v[4 * i + 0] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else {
        ld_vec<V>(v, p);
    }
}

// ----------------------------------------------- sum-product (linear/log) ----
// One lane's share of the update of one node: the constants of the band
// (weights, normaliser weights) are set once per grid, node() runs per node.
// LOG = false: linear messages, g is the unary.  LOG = true: log-messages,
// g holds log g; h is formed as exp(log h - max log h), which leaves the
// normalised result unchanged.
// FULL: every padded label is a label (M == Mp), so the label masks vanish
template <int L, int C, int T, bool LOG, bool COH, bool FULL = false>
struct SumBand {
    static constexpr int V = 4 * C;
    float w[2 * T + 1];
    float fbar;
    float cz[V];
    bool lab_ok[V];
    int q;

    __device__ __forceinline__ void setup(const float *wsrc, float fb, int M, int lane_q) {
        q = lane_q;
        fbar = fb;
#pragma unroll
        for (int i = 0; i < 2 * T + 1; ++i) w[i] = wsrc[i];
        // per-label normaliser weights c(x) + M fbar (0 on padded labels)
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int x = q * V + k;
            float cx = 0.f;
#pragma unroll
            for (int d = -T; d <= T; ++d)
                if (x - d >= 0 && x - d < M) cx += w[d + T];
            lab_ok[k] = x < M;
            cz[k] = lab_ok[k] ? cx + (float)M * fbar : 0.f;
        }
    }

    __device__ __forceinline__ void node(const float *g, const float *in, float *out, int W, int H, int Mp,
                                         long long plane, int r, int c, bool valid,
                                         float2 *stats = nullptr) const {
        const long long off = ((long long)r * W + c) * Mp + q * V;
        const bool has[4] = {valid && c > 0, valid && c < W - 1, valid && r > 0, valid && r < H - 1};
        const float absent = LOG ? 0.f : 1.f;

        float gv[V], m[4][V];
        if (valid) ld_vec<V>(gv, g + off); else fill_vec<V>(gv, 0.f);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (has[s]) ld_msg<COH, V>(m[s], in + s * plane + off);
            else fill_vec<V>(m[s], absent);
        }

#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float h[V];
            float amax = 0.f;   // log mode: the max shift of h
            if (!LOG) {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    // product of the unary and the three messages other than m[t]
                    const float p01 = (t == 0) ? m[1][k] : (t == 1) ? m[0][k] : m[0][k] * m[1][k];
                    const float p23 = (t == 2) ? m[3][k] : (t == 3) ? m[2][k] : m[2][k] * m[3][k];
                    h[k] = gv[k] * p01 * p23;
                }
            } else {
                amax = kLogNone;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    float s = gv[k];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (u != t) s += m[u][k];
                    h[k] = (FULL || lab_ok[k]) ? s : kLogNone;
                    amax = fmaxf(amax, h[k]);
                }
                amax = group_max<L>(amax);
#pragma unroll
                for (int k = 0; k < V; ++k) h[k] = (FULL || lab_ok[k]) ? exp2_hw(h[k] - amax) : 0.f;
            }

            float S = 0.f, Z = 0.f;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                S += h[k];
                Z = fmaf(h[k], cz[k], Z);
            }
            S = group_sum<L>(S);
            Z = group_sum<L>(Z);

            float win[V + 2 * T];
            band_window<L, V, T, float>(win, h, q, 0.f);
            const float inv = 1.f / Z;
            const float base_term = fbar * S * inv;
            if constexpr (LOG) {
                // the scale of this message for the adjoint, [node][direction]:
                // h / Z = 2^(a - C), C = shift + log2 Z; lane t of the group
                // writes direction t (a node's four pairs fill one 32-byte sector)
                if (stats && valid && q == (t & (L - 1)))
                    stats[((long long)r * W + c) * 4 + t] = make_float2(amax + __log2f(Z), S * inv);
            }
            float o[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int d = -T; d <= T; ++d) acc = fmaf(w[d + T], win[T + k + d], acc);
                const float mv = fmaf(acc, inv, base_term);
                o[k] = (FULL || lab_ok[k]) ? (LOG ? __log2f(mv) : mv) : 0.f;
            }
            if (has[t]) st_vec<V>(out + out_offset(t, r, c, W, plane, Mp) + q * V, o);
        }
    }
};

template <bool LOG>
struct SumArgsOf {
    using type = BandArgsF;
};
template <>
struct SumArgsOf<true> {
    using type = BandArgsLogF;
};

template <int L, int C, int T, bool LOG, bool FULL = false>
__global__ void __launch_bounds__(kBlock) band_sum_kernel(const typename SumArgsOf<LOG>::type a) {
    constexpr int GPB = kBlock / L;
    const int grp = threadIdx.x / L;
    SumBand<L, C, T, LOG, false, FULL> band;
    band.setup(a.w, a.fbar, a.d.M, threadIdx.x & (L - 1));
    const int W = a.d.W;
    const int nslots = num_slots(W, a.d.H, a.parity);
    for (int base = blockIdx.x * GPB; base < nslots; base += gridDim.x * GPB) {
        int r, c;
        const bool valid = slot_node(base + grp, nslots, W, a.parity, r, c);
        if constexpr (LOG)
            band.node(a.g, a.in, a.out, W, a.d.H, a.d.Mp, a.d.plane, r, c, valid, a.stats);
        else
            band.node(a.g, a.in, a.out, W, a.d.H, a.d.Mp, a.d.plane, r, c, valid);
    }
}

// ------------------------------------------------------------- min-sum ------
// When E(0) is the smallest entry of the table (every truncated potential),
// min_x u(x) = E(0) + min_x h(x) exactly: the pair (x*, x*) with h(x*) minimal
// is in the band, every band term is >= E(0) + min h, and Ebar >= E(0).  The
// second reduction is then skipped (`zero_min`).
// FULL: M == Mp, every padded label is a label and the label masks vanish
template <int L, int C, int T, bool COH, bool FULL = false>
struct MinBand {
    static constexpr int V = 4 * C;
    static constexpr int VP = V / 2;            // label pairs per lane (packed form)
    static constexpr int TP = (T + 1) / 2;      // halo pairs on each side
    int32_t w[2 * T + 1];
    int32_t ebar;
    bool lab_ok[V];
    bool zero_min;
    int q;
    // packed form: E'(d) = E(d) - Emin in both halves, Ebar' = Ebar - Emin
    bool p16;
    uint32_t wp[2 * T + 1];
    uint32_t keep[VP];                          // 0xffff per half that holds a label < M
    int32_t ebar16;

    __device__ __forceinline__ void setup(const int32_t *wsrc, int32_t eb, int M, int lane_q, bool zmin = false,
                                          bool packed = false) {
        q = lane_q;
        ebar = eb;
        zero_min = zmin;
        int32_t emin = eb;
#pragma unroll
        for (int i = 0; i < 2 * T + 1; ++i) {
            w[i] = wsrc[i];
            emin = min(emin, w[i]);
        }
#pragma unroll
        for (int k = 0; k < V; ++k) lab_ok[k] = q * V + k < M;
        p16 = packed;
        ebar16 = eb - emin;
#pragma unroll
        for (int i = 0; i < 2 * T + 1; ++i) wp[i] = (uint32_t)(w[i] - emin) * 0x10001u;
#pragma unroll
        for (int k = 0; k < VP; ++k) keep[k] = (lab_ok[2 * k] ? 0xffffu : 0u) | (lab_ok[2 * k + 1] ? 0xffff0000u : 0u);
    }

    // Eq. 11 on 16-bit label pairs, exact when Ebar - Emin <= 16000 (the host
    // decides).  With h' = min(h - Hmin, Ebar' + 1) and E' = E - Emin,
    //   u'(x) = min(Ebar', min_d E'(d) + h'(x + d))
    // equals u(x) - Hmin - Emin: a clamped term is > Ebar' >= u'(x) either way,
    // so the clamp never changes the minimum, and every value stays below
    // 2 Ebar' + 2 <= 32002.  Two labels per DPX add-min instead of one.
    __device__ __forceinline__ void band_packed(const int32_t (&h)[V], int32_t hmin, int32_t (&u)[V]) const {
        const int32_t cap = hmin + ebar16 + 1;
        uint32_t hp[VP];
#pragma unroll
        for (int k = 0; k < VP; ++k) {
            const uint32_t lo = (uint32_t)(min(h[2 * k], cap) - hmin);
            const uint32_t hi = (uint32_t)(min(h[2 * k + 1], cap) - hmin);
            hp[k] = lo | (hi << 16);
        }
        const uint32_t none = (uint32_t)(ebar16 + 1) * 0x10001u;
        uint32_t win[VP + 2 * TP];                 // pairs of labels qV - 2TP + 2j, + 1
        band_window<L, VP, TP, uint32_t>(win, hp, q, none);
        uint32_t odd[VP + 2 * TP - 1];             // pairs starting one label later
#pragma unroll
        for (int j = 0; j + 1 < VP + 2 * TP; ++j) odd[j] = __byte_perm(win[j], win[j + 1], 0x5432);
        const uint32_t flat = (uint32_t)ebar16 * 0x10001u;
        uint32_t acc[VP];
#pragma unroll
        for (int k = 0; k < VP; ++k) {
            uint32_t a = flat;
#pragma unroll
            for (int d = -T; d <= T; ++d) {
                const int r = 2 * k + d + 2 * TP;  // window position of label pair (2k + d, 2k + d + 1)
                const uint32_t term = (r & 1) ? odd[(r - 1) / 2] : win[r / 2];
                a = __viaddmin_s16x2(wp[d + T], term, a);
            }
            acc[k] = FULL ? a : (a & keep[k]) | (flat & ~keep[k]);   // labels >= M: Ebar', never below the minimum
        }
        int32_t umin;
        if (zero_min) {
            umin = (int32_t)(wp[T] & 0xffffu);
        } else {
            uint32_t m2 = acc[0];
#pragma unroll
            for (int k = 1; k < VP; ++k) m2 = __vimin_s16x2_relu(m2, acc[k]);   // halves are >= 0
            umin = group_min<L>(min((int32_t)(m2 & 0xffffu), (int32_t)(m2 >> 16)));
        }
        const uint32_t sub = (uint32_t)umin * 0x10001u;
#pragma unroll
        for (int k = 0; k < VP; ++k) {
            const uint32_t o = FULL ? acc[k] - sub : (acc[k] - sub) & keep[k];   // no borrow: every half >= umin
            u[2 * k] = (int32_t)(o & 0xffffu);
            u[2 * k + 1] = (int32_t)(o >> 16);
        }
    }

    // Eq. 11 on int32 labels: one DPX add-min per band term
    __device__ __forceinline__ void band_int(const int32_t (&h)[V], int32_t hmin, int32_t (&u)[V]) const {
        int32_t win[V + 2 * T];
        band_window<L, V, T, int32_t>(win, h, q, kIntBig);
        const int32_t flat = ebar + hmin;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            int32_t b = flat;
#pragma unroll
            for (int d = -T; d <= T; ++d) b = __viaddmin_s32(w[d + T], win[T + k + d], b);
            u[k] = (FULL || lab_ok[k]) ? b : kIntBig;
        }
        const int32_t umin = zero_min ? w[T] + hmin : group_min<L>(min_vec<V>(u));
#pragma unroll
        for (int k = 0; k < V; ++k) u[k] = (FULL || lab_ok[k]) ? u[k] - umin : 0;
    }

    __device__ __forceinline__ void node(const int32_t *e, const int32_t *in, int32_t *out, int W, int H, int Mp,
                                         long long plane, int r, int c, bool valid) const {
        const long long off = ((long long)r * W + c) * Mp + q * V;
        const bool has[4] = {valid && c > 0, valid && c < W - 1, valid && r > 0, valid && r < H - 1};

        int32_t ev[V], m[4][V];
        if (valid) ld_vec<V>(ev, e + off); else fill_vec<V, int32_t>(ev, 0);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (has[s]) ld_msg<COH, V>(m[s], in + s * plane + off);
            else fill_vec<V, int32_t>(m[s], 0);
        }
        // E_u + all four messages once per label (labels >= M: kIntBig); the
        // h of direction t is that total minus the message from side t
        int32_t tot[V];
#pragma unroll
        for (int k = 0; k < V; ++k) tot[k] = (FULL || lab_ok[k]) ? ev[k] + m[0][k] + m[1][k] + m[2][k] + m[3][k] : kIntBig;

#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int32_t h[V];
#pragma unroll
            for (int k = 0; k < V; ++k) h[k] = tot[k] - m[t][k];
            int32_t hmin = min_vec<V>(h);
            hmin = group_min<L>(hmin);

            int32_t u[V];
            // the packed form pays from T = 3 on; narrower bands keep the
            // int32 form only (and its register count)
            if constexpr (T >= 3) {
                if (p16) band_packed(h, hmin, u);
                else band_int(h, hmin, u);
            } else {
                band_int(h, hmin, u);
            }
            if (has[t]) st_vec<V>(out + out_offset(t, r, c, W, plane, Mp) + q * V, u);
        }
    }
};

template <int L, int C, int T, bool FULL = false>
__global__ void __launch_bounds__(kBlock) band_min_kernel(const BandArgsI a) {
    constexpr int GPB = kBlock / L;
    const int grp = threadIdx.x / L;
    MinBand<L, C, T, false, FULL> band;
    band.setup(a.w, a.ebar, a.d.M, threadIdx.x & (L - 1), a.zero_min != 0, a.packed16 != 0);
    const int W = a.d.W;
    const int nslots = num_slots(W, a.d.H, a.parity);
    for (int base = blockIdx.x * GPB; base < nslots; base += gridDim.x * GPB) {
        int r, c;
        const bool valid = slot_node(base + grp, nslots, W, a.parity, r, c);
        band.node(a.e, a.in, a.out, W, a.d.H, a.d.Mp, a.d.plane, r, c, valid);
    }
}

}  // namespace bpg
