// Launch of the persistent batch kernel, min-sum int32.
#include "band_dispatch.cuh"
#include "bp_batch_internal.h"

namespace bpg {

const void *batch_min_kernel_f1();        // batch_min_f1.cu
const void *batch_min_kernel_f2();        // batch_min_f2.cu
const void *batch_min_kernel_f1_full();   // batch_min_f1_full.cu
const void *batch_min_kernel_f2_full();   // batch_min_f2_full.cu
const void *batch_min_kernel_rb();        // batch_min_rb.cu
const void *batch_min_kernel_mixed();     // batch_min_mixed.cu
const void *batch_min_kernel_mixed_full();   // batch_min_mixed_full.cu

// full: every MRF has M == Mp, the variant without padded-label masks (same
// launch bounds, so the same two resident blocks per SM)
static const void *batch_min_fn(int family, bool redblack = false, bool full = false) {
    if (redblack) return batch_min_kernel_rb();
    if (family == 0) return full ? batch_min_kernel_mixed_full() : batch_min_kernel_mixed();
    if (full) return family == 2 ? batch_min_kernel_f2_full() : batch_min_kernel_f1_full();
    return family == 2 ? batch_min_kernel_f2() : batch_min_kernel_f1();
}

cudaError_t launch_batch_min(const BatchArgs &a, int family, int blocks, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<BatchArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, batch_min_fn(family, a.redblack != 0, a.full != 0), args);
}

int batch_max_blocks_min(int family, bool redblack, bool full) {
    return device_sm_count() * blocks_per_sm(batch_min_fn(family, redblack, full));
}

}  // namespace bpg
