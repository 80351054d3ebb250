// Persistent O(mM) kernel for a batch of independent MRFs of uneven size,
// label count and band width.
//
// One cooperative launch runs every iteration of every MRF.  The nodes of all
// MRFs are cut into work items (mrf, first node, node count) of roughly equal
// bytes, listed by (band half-width, label count) class.  Blocks take items
// in list order from one 64-bit ticket counter (ticket k = item k % n_items of
// step k / n_items), each block fetching its next ticket while it works on the
// current item, and run per item the per-node update (SumBand / MinBand)
// compiled for that MRF's padded label count and band half-width.  Taking the
// list in order keeps the whole grid inside one class at a time, so an SM
// runs one compiled variant at a time; taking it dynamically balances items
// whose cost differs with T.  A ticket past the current step is kept for the
// step it belongs to.  Between iterations all blocks meet at a grid barrier
// whose wait is bounded: on time-out the block records an error code in the
// status word and the kernel returns (the host reports BP_ERR_TIMEOUT).
// Messages written by other blocks are read with L2-coherent loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "band_fast.cuh"
#include "bp_batch_internal.h"

namespace bpg {

__device__ __forceinline__ unsigned long long batch_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-reversing grid barrier over `expected` arrivals.  Returns false (in
// every thread of the block) if the wait ran out.  Thread 0 of each block
// publishes the block's writes (bar.sync then a gpu-scope acq_rel fence),
// arrives on the counter, and the last arrival bumps the generation word the
// others poll.
__device__ __forceinline__ bool batch_grid_barrier(unsigned *count, unsigned *gen, unsigned expected,
                                                   unsigned long long limit_ns, int *status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned g;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        const unsigned arrived = atomicAdd(count, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(count, 0u);
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            atomicAdd(gen, 1u);
        } else {
            unsigned long long t0 = 0;
            for (unsigned spins = 0;; ++spins) {
                unsigned cur;
                asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(gen) : "memory");
                if (cur != g) break;
                if ((spins & 1023u) == 0) {
                    const unsigned long long now = batch_timer();
                    if (spins == 0) t0 = now;
                    else if (now - t0 > limit_ns) {
                        ok = 0;
                        atomicExch(status, 201);
                        break;
                    }
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
    return ok != 0;
}

// parity < 0: synchronous (read msg[src], write msg[src ^ 1]); parity 0/1:
// red-black half-step in place on msg[src], slots as in slot_node.
// FULL: every MRF of the batch has M == Mp (no padded-label masks)
template <int L, int C, int T, bool MIN, bool RB, bool FULL>
__device__ __forceinline__ void batch_item(const BatchMrf *__restrict__ m, int node0, int count, int src,
                                           int parity_rt) {
    const int parity = RB ? parity_rt : -1;
    constexpr int GPB = kBlock / L;
    const int grp = threadIdx.x / L;
    const int q = threadIdx.x & (L - 1);
    const int W = m->W, H = m->H, Mp = m->Mp;
    const long long plane = m->plane;
    const int nslots = num_slots(W, H, parity);
    const void *un = m->unary;
    const void *in = m->msg[src];
    void *out = parity < 0 ? m->msg[src ^ 1] : m->msg[src];
    if (MIN) {
        MinBand<L, C, T, true, FULL> b;
        b.setup(m->wi, m->ebar, m->M, q, m->zero_min != 0, m->packed16 != 0);
        for (int base = 0; base < count; base += GPB) {
            int r = 0, c = 0;
            bool valid = base + grp < count;
            if (RB) {
                valid = valid && slot_node(node0 + base + grp, nslots, W, parity, r, c);
            } else if (valid) {
                const int n = node0 + base + grp;
                r = n / W;
                c = n - r * W;
            }
            b.node((const int32_t *)un, (const int32_t *)in, (int32_t *)out, W, H, Mp, plane, r, c, valid);
        }
    } else {
        SumBand<L, C, T, false, true, FULL> b;
        b.setup(m->wf, m->fbar, m->M, q);
        for (int base = 0; base < count; base += GPB) {
            int r = 0, c = 0;
            bool valid = base + grp < count;
            if (RB) {
                valid = valid && slot_node(node0 + base + grp, nslots, W, parity, r, c);
            } else if (valid) {
                const int n = node0 + base + grp;
                r = n / W;
                c = n - r * W;
            }
            b.node((const float *)un, (const float *)in, (float *)out, W, H, Mp, plane, r, c, valid);
        }
    }
}

template <int L, int C, bool MIN, bool RB, bool FULL>
__device__ __forceinline__ void batch_item_t(const BatchMrf *__restrict__ m, int node0, int count, int src,
                                             int parity) {
    switch (m->T) {
        case 0: batch_item<L, C, 0, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 1: batch_item<L, C, 1, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 2: batch_item<L, C, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 3: batch_item<L, C, 3, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 4: batch_item<L, C, 4, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 5: batch_item<L, C, 5, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 6: batch_item<L, C, 6, MIN, RB, FULL>(m, node0, count, src, parity); break;
        case 7: batch_item<L, C, 7, MIN, RB, FULL>(m, node0, count, src, parity); break;
        default: batch_item<L, C, 8, MIN, RB, FULL>(m, node0, count, src, parity); break;
    }
}

// Family 1: the fewest labels per lane (C = 1 up to 128 labels);
// family 2: two 4-label chunks per lane.  Padded label counts 16..256.
template <int FAM, bool MIN, bool RB, bool FULL>
__device__ __forceinline__ void batch_dispatch(const BatchMrf *__restrict__ m, int node0, int count, int src,
                                               int parity) {
    if (FAM == 1) {
        switch (m->Mp) {
            case 16: batch_item_t<4, 1, MIN, RB, FULL>(m, node0, count, src, parity); break;
            case 32: batch_item_t<8, 1, MIN, RB, FULL>(m, node0, count, src, parity); break;
            case 64: batch_item_t<16, 1, MIN, RB, FULL>(m, node0, count, src, parity); break;
            case 128: batch_item_t<32, 1, MIN, RB, FULL>(m, node0, count, src, parity); break;
            default: batch_item_t<32, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
        }
    } else {
        switch (m->Mp) {
            case 16: batch_item_t<2, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
            case 32: batch_item_t<4, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
            case 64: batch_item_t<8, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
            case 128: batch_item_t<16, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
            default: batch_item_t<32, 2, MIN, RB, FULL>(m, node0, count, src, parity); break;
        }
    }
}

// FAM = 0: each item runs the family of its MRF's class (classes with
// different lane layouts in one launch)
template <int FAM, bool MIN, bool RB, bool FULL>
__device__ __forceinline__ void batch_dispatch_any(const BatchMrf *__restrict__ m, int node0, int count, int src,
                                                   int parity) {
    if constexpr (FAM == 0) {
        if (m->family == 2)
            batch_dispatch<2, MIN, RB, FULL>(m, node0, count, src, parity);
        else
            batch_dispatch<1, MIN, RB, FULL>(m, node0, count, src, parity);
    } else {
        batch_dispatch<FAM, MIN, RB, FULL>(m, node0, count, src, parity);
    }
}

// RB: the red-black form (two in-place half-steps per iteration), compiled
// separately so that the synchronous batch kernel keeps its registers.
template <int FAM, bool MIN, bool RB, bool FULL = false>
__global__ void __launch_bounds__(kBlock, 2) batch_kernel(const BatchArgs a) {
    __shared__ unsigned long long s_ticket[2];
    const int phases = RB ? 2 : 1;
    const int total = a.n_iters * phases;
    const unsigned long long n_items = (unsigned long long)a.n_items;
    // thread 0 writes slot `slot ^ 1` while the others read slot `slot`; a
    // slot is rewritten only after the __syncthreads that follows its read
    int slot = 0;
    if (threadIdx.x == 0) s_ticket[0] = atomicAdd(a.tickets, 1ull);
    __syncthreads();
    unsigned long long ticket = s_ticket[0];
    for (int step = 0; step < total; ++step) {
        const int parity = RB ? (step & 1) : -1;
        const int src = RB ? a.start_buf : ((a.start_buf + step) & 1);
        const unsigned long long first = (unsigned long long)step * n_items;
        while (ticket < first + n_items) {
            if (threadIdx.x == 0) s_ticket[slot ^ 1] = atomicAdd(a.tickets, 1ull);
            const BatchItem item = a.items[ticket - first];
            batch_dispatch_any<FAM, MIN, RB, FULL>(a.mrfs + item.mrf, item.node0, item.count, src, parity);
            __syncthreads();
            slot ^= 1;
            ticket = s_ticket[slot];
        }
        if (step + 1 < total) {
            if (!batch_grid_barrier(a.bar_count, a.bar_gen, gridDim.x + a.extra_arrivals, a.limit_ns, a.status))
                return;
        }
    }
}

}  // namespace bpg
