// Instantiations of the persistent batch kernel, min-sum int32.
#include "batch_kernels.cuh"
#include "band_dispatch.cuh"

namespace bpg {

static const void *batch_min_fn(int family, bool redblack = false) {
    if (redblack) return (const void *)batch_kernel<1, true, true>;
    return family == 2 ? (const void *)batch_kernel<2, true, false> : (const void *)batch_kernel<1, true, false>;
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
    return cudaLaunchKernelExC(&cfg, batch_min_fn(family, a.redblack != 0), args);
}

int batch_max_blocks_min(int family, bool redblack) {
    return device_sm_count() * blocks_per_sm(batch_min_fn(family, redblack));
}

}  // namespace bpg
