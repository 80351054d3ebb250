// Compile-time table of the O(mM) fast kernels: every (L, C) layout below for
// every band half-width T = 0..kTMaxFast, and a launcher that picks one.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "bp_internal.h"

namespace bpg {

// (lanes per node L, 4-label chunks per lane C); padded label count 4*L*C.
#define BPG_LAYOUT_LIST(X) \
    X(1, 1) X(2, 1) X(4, 1) X(2, 2) X(8, 1) X(4, 2) X(16, 1) X(8, 2) X(32, 1) X(16, 2) X(32, 2) X(16, 4) X(32, 4)

template <class Tag, int L, int C>
inline const void *pick_t(int T) {
    switch (T) {
        case 0: return Tag::template get<L, C, 0>();
        case 1: return Tag::template get<L, C, 1>();
        case 2: return Tag::template get<L, C, 2>();
        case 3: return Tag::template get<L, C, 3>();
        case 4: return Tag::template get<L, C, 4>();
        case 5: return Tag::template get<L, C, 5>();
        case 6: return Tag::template get<L, C, 6>();
        case 7: return Tag::template get<L, C, 7>();
        case 8: return Tag::template get<L, C, 8>();
        default: return nullptr;
    }
}

template <class Tag>
inline const void *pick_kernel(Layout lay, int T) {
#define BPG_X(l, c) \
    if (lay.L == l && lay.C == c) return pick_t<Tag, l, c>(T);
    BPG_LAYOUT_LIST(BPG_X)
#undef BPG_X
    return nullptr;
}

// Resident blocks per SM for a kernel (cached).
inline int blocks_per_sm(const void *fn) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kBlock, 0) != cudaSuccess || n < 1) n = 1;
    cache[fn] = n;
    return n;
}

inline int slots_of(const GridDims &d, int parity) {
    return parity < 0 ? d.W * d.H : ((d.W + 1) / 2) * d.H;
}

template <class Tag, class Args>
inline cudaError_t launch_fast(const Args &a, Layout lay, int blocks, cudaStream_t s) {
    if (lay.L * 4 * lay.C != a.d.Mp) return cudaErrorInvalidValue;
    const void *fn = pick_kernel<Tag>(lay, a.T);
    if (!fn) return cudaErrorInvalidValue;
    const int per_block = kBlock / lay.L;
    const long long need = (slots_of(a.d, a.parity) + per_block - 1) / per_block;
    if (blocks <= 0) blocks = device_sm_count() * blocks_per_sm(fn);
    if (blocks > need) blocks = (int)need;
    if (blocks < 1) blocks = 1;
    void *args[] = {const_cast<Args *>(&a)};
    return cudaLaunchKernel(fn, dim3(blocks), dim3(kBlock), args, 0, s);
}

}  // namespace bpg
