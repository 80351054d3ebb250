// Reverse mode of the log-domain O(mM) sum-product update.
//
// Forward, for the message from node i to its neighbour j (Eq. 5, Eq. 7, with
// the log-domain shift A = max_x a(x), which leaves the result unchanged):
//   a(x)   = log g_i(x) + sum_{k != j} l_ki(x),   h(x) = exp(a(x) - A)
//   S      = sum_x h(x),  B(x_j) = sum_{|d|<=T} w(d) h(x_j + d),  w(d) = f(d) - fbar
//   u(x_j) = B(x_j) + fbar S,  Z = sum_x u(x),  l_ij(x_j) = log u(x_j) - log Z
// Reverse, given delta(x_j) = dL/dl_ij(x_j):
//   nu(x_j)   = delta(x_j) / u(x_j) - (sum_x delta(x)) / Z            (= dL/du)
//   dh(x_i)   = sum_{|e|<=T} w(-e) nu(x_i + e) + fbar sum_x nu(x)      (band transposed: O(mM))
//   da(x_i)   = dh(x_i) h(x_i)   -> dL/d log g_i and dL/d l_ki for every k != j
//   dw(d)    += sum_{x_j} nu(x_j) h(x_j + d)                           (= dL/df(d))
//   dfbar    += S sum_x nu(x) - sum_d dw(d)   (fbar enters u directly and through w)
// In terms of the normalised h^ = h / Z, S^ = S / Z, u^ = u / Z and
// nu^ = Z nu = delta / u^ - sum delta, every line keeps its form:
//   da = h^ (sum_e w(-e) nu^(x + e) + fbar sum nu^),  dw(d) += sum nu^ h^(x_j + d),
//   dfbar += S^ sum nu^ - sum_d dw(d).
// The recorded forward stores per message C = A + log2 Z and S^ (the stats
// planes), so h^ = 2^(a - C) comes without the max, S and Z reductions of
// the forward; only sum delta and sum nu^ are reduced here.
// The states and log g are base-2 logs (the library's log domain): h^ and the
// belief softmax are computed with 2^x exactly as the forward kernel does,
// while every adjoint (delta, nu, da, dL/d log g) is a derivative with
// respect to natural logs, the units of the caller's log g and log-beliefs.
// delta / u^ uses the hardware approximate division (2 ulp; u^ > 0 is normal).
//
// One kernel launch reverses one synchronous iteration for every node; the
// per-block sums of dw and dfbar go to a scratch row per (iteration, block),
// reduced over all edges and iterations in FP64 at the end.
#pragma once

#include <cuda_runtime.h>

#include "band_dispatch.cuh"
#include "band_fast.cuh"
#include "bp_adjoint.h"

namespace bpg {

// scale of an absent message: 2^(a - kNoScale) = 0
constexpr float kNoScale = 3.0e38f;

// One chunk per lane and T <= 4 (kEarly): the kernel is held to 80 registers
// so that three blocks (24 warps) share an SM, and every load of a node is
// issued at once; the extra warps hide the latency (72 -> 61 us at 256x256,
// M = 64, T = 3, for a few bytes of spill).  Wider layouts and bands would
// spill heavily: they keep the compiler's register choice and load each
// direction's adjoint where it is used.
template <int C, int T>
__host__ __device__ constexpr bool adjoint_early() { return C == 1 && T <= 4; }

// FULL: M == Mp, every padded label is a label and the label masks vanish
template <int L, int C, int T, bool kEarly, bool FULL>
__device__ __forceinline__ void adjoint_body(const AdjArgs &a) {
    constexpr int V = 4 * C;
    constexpr int GPB = kBlock / L;
    constexpr int NP = 2 * T + 2;      // dw(-T..T), dfbar
    const int q = threadIdx.x & (L - 1);
    const int grp = threadIdx.x / L;
    const int W = a.d.W, H = a.d.H, M = a.d.M, Mp = a.d.Mp;
    const long long plane = a.d.plane;

    float w[2 * T + 1];
#pragma unroll
    for (int i = 0; i < 2 * T + 1; ++i) w[i] = a.w[i];
    const float fbar = a.fbar;
    bool lab_ok[V];
#pragma unroll
    for (int k = 0; k < V; ++k) lab_ok[k] = q * V + k < M;

    float pacc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) pacc[i] = 0.f;

    const int nslots = W * H;
    for (int base = blockIdx.x * GPB; base < nslots; base += gridDim.x * GPB) {
        int r, c;
        const bool valid = slot_node(base + grp, nslots, W, -1, r, c);
        const long long off = ((long long)r * W + c) * Mp + q * V;
        const bool has[4] = {valid && c > 0, valid && c < W - 1, valid && r > 0, valid && r < H - 1};

        // with the 80-register bound (kEarly) every load of the node goes
        // first: the state, the adjoints of the four outgoing messages and
        // dL/d log g, one round trip instead of six
        constexpr int VE = kEarly ? V : 1;
        float gam[V], l[4][V], lam[4][VE], dgo[VE];
        if (valid) ld_vec<V>(gam, a.logg + off); else fill_vec<V>(gam, 0.f);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (has[s]) ld_vec<V>(l[s], a.ell + s * plane + off);
            else fill_vec<V>(l[s], 0.f);
        }
        if constexpr (kEarly) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (has[t]) ld_vec<V>(lam[t], a.lam_next + out_offset(t, r, c, W, plane, Mp) + q * V);
                else fill_vec<V>(lam[t], 0.f);
            }
            if (valid) ld_vec<V>(dgo, a.dlogg + off); else fill_vec<V>(dgo, 0.f);
        }
        // the forward's scale and S^ of each outgoing message (absent: h^ = 0)
        const float2 *sp = a.stats + ((long long)r * W + c) * 4;
        float dl[4][V], dg[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            dg[k] = 0.f;
#pragma unroll
            for (int s = 0; s < 4; ++s) dl[s][k] = 0.f;
        }

#pragma unroll
        for (int t = 0; t < 4; ++t) {
            // h^ of the message towards neighbour t, from the stored scale
            float Ct = kNoScale, St = 0.f;
            if (has[t]) {
                const float2 sv = __ldg(sp + t);
                Ct = sv.x;
                St = sv.y;
            }
            float h[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                float s = gam[k];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u != t) s += l[u][k];
                h[k] = (FULL || lab_ok[k]) ? exp2_hw(s - Ct) : 0.f;   // as the forward kernel
            }
            float win[V + 2 * T];
            band_window<L, V, T, float>(win, h, q, 0.f);

            // adjoint of the stored message
            float del[V];
            if constexpr (kEarly) {
#pragma unroll
                for (int k = 0; k < V; ++k) del[k] = lam[t][k % VE];
            } else {
                if (has[t]) ld_vec<V>(del, a.lam_next + out_offset(t, r, c, W, plane, Mp) + q * V);
                else fill_vec<V>(del, 0.f);
            }
            float nd = 0.f;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                del[k] = (FULL || lab_ok[k]) ? del[k] : 0.f;
                nd += del[k];
            }
            nd = group_sum<L>(nd);
            float nu[V];
            float nn = 0.f;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                float u = fbar * St;
#pragma unroll
                for (int d = -T; d <= T; ++d) u = fmaf(w[d + T], win[T + k + d], u);
                nu[k] = ((FULL || lab_ok[k]) && has[t]) ? __fdividef(del[k], u) - nd : 0.f;
                nn += nu[k];
            }
            nn = group_sum<L>(nn);

            // dh through the transposed band, then da = dh * h
            float nwin[V + 2 * T];
            band_window<L, V, T, float>(nwin, nu, q, 0.f);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                float dh = fbar * nn;
#pragma unroll
                for (int e = -T; e <= T; ++e) dh = fmaf(w[-e + T], nwin[T + k + e], dh);
                const float da = dh * h[k];
                dg[k] += da;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (s != t) dl[s][k] += da;
            }

            // parameter gradients
            float dsum = 0.f;
#pragma unroll
            for (int d = -T; d <= T; ++d) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < V; ++k) acc = fmaf(nu[k], win[T + k + d], acc);
                pacc[d + T] += acc;
                dsum += acc;
            }
            pacc[NP - 1] += (q == 0 ? nn * St : 0.f) - dsum;
        }

#pragma unroll
        for (int s = 0; s < 4; ++s)
            if (has[s]) st_vec<V>(a.lam + s * plane + off, dl[s]);
        if constexpr (kEarly) {
            if (valid) {
#pragma unroll
                for (int k = 0; k < V; ++k) dg[k] += dgo[k % VE];
                st_vec<V>(a.dlogg + off, dg);
            }
        } else if (valid) {
            float acc[V];
            ld_vec<V>(acc, a.dlogg + off);
#pragma unroll
            for (int k = 0; k < V; ++k) acc[k] += dg[k];
            st_vec<V>(a.dlogg + off, acc);
        }
    }

    // block sums of the parameter gradients -> scratch row of this block
    __shared__ float red[kBlock / 32][NP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        float v = pacc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(BPG_FULL, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        float v = 0.f;
        for (int k = 0; k < kBlock / 32; ++k) v += red[k][threadIdx.x];
        a.partial[(long long)blockIdx.x * NP + threadIdx.x] = v;
    }
}

template <int L, int C, int T, bool FULL>
__global__ void __launch_bounds__(kBlock) band_log_adjoint_kernel(const AdjArgs a) {
    adjoint_body<L, C, T, false, FULL>(a);
}

template <int L, int C, int T, bool FULL>
__global__ void __launch_bounds__(kBlock, 3) band_log_adjoint_kernel_3pm(const AdjArgs a) {
    adjoint_body<L, C, T, true, FULL>(a);
}

template <bool FULL>
struct AdjTagT {
    template <int L, int C, int T>
    static const void *get() {
        if constexpr (adjoint_early<C, T>()) return (const void *)band_log_adjoint_kernel_3pm<L, C, T, FULL>;
        else return (const void *)band_log_adjoint_kernel<L, C, T, FULL>;
    }
};

}  // namespace bpg
