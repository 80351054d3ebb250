// Device-side descriptors and launch interface of the batched O(mM) kernel.
// Internal; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bp_internal.h"

namespace bpg {

struct BatchMrf {
    const void *unary;      // [H][W][Mp]
    void *msg[2];           // two [4][H][W][Mp] message states
    long long plane;        // H * W * Mp
    int W, H, M, Mp;
    int T;                  // effective band half-width (<= kTMaxFast)
    float wf[2 * kTMaxFast + 1];    // f(d) - fbar (sum-product)
    float fbar;
    int32_t wi[2 * kTMaxFast + 1];  // E(d) (min-sum)
    int32_t ebar;
    int zero_min;                   // 1 if E(0) is the table's minimum
    int packed16;                   // 1: min-sum band on 16-bit label pairs (see MinBand)
    int family;                     // lane layout of this MRF's (Mp, T) class: 1 or 2 chunks per lane
};

// A run of `count` consecutive slots of one MRF: nodes for a synchronous
// iteration, half-step slots (see slot_node) for the red-black schedule.
struct BatchItem {
    int mrf;
    int node0;
    int count;
};

struct BatchArgs {
    const BatchMrf *mrfs;
    const BatchItem *items;
    int n_items;
    int n_iters;
    int start_buf;              // synchronous: iteration t reads msg[(start_buf + t) & 1]
    int redblack;               // 1: two in-place half-steps per iteration on msg[start_buf]
    int full;                   // host-side choice: every MRF has M == Mp (kernel variant without label masks)
    unsigned *bar_count;        // grid barrier: arrivals, generation
    unsigned *bar_gen;
    unsigned long long *tickets;   // work counter, zero at launch: ticket k is item k % n_items of step k / n_items
    int extra_arrivals;         // 0; > 0 makes the barrier wait for blocks that never come
    unsigned long long limit_ns;
    int *status;
};

// Layout of the barrier / work-counter words (32 bytes, 8-byte aligned):
// [0] barrier arrivals, [2..3] the 64-bit ticket counter (both zeroed before
// every launch: kBatchZeroBytes from the start), [4] barrier generation.
constexpr int kBatchCtlWords = 8;
constexpr size_t kBatchZeroBytes = 16;
constexpr int kBatchTicketWord = 2;
constexpr int kBatchGenWord = 4;

// Launch one persistent cooperative batch kernel (family 1 or 2 for every MRF,
// or 0: each MRF's own family).
cudaError_t launch_batch(const BatchArgs &a, int family, bool min_sum, int blocks, cudaStream_t s);
// Largest co-resident grid for that kernel.
int batch_max_blocks(int family, bool min_sum);
// Groups per block (nodes in flight) of a family for a padded label count.
int batch_lanes_per_node(int family, int Mp);

}  // namespace bpg
