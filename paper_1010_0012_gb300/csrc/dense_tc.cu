// Dense O(M^2) sum-product baseline on the tensor cores.
#include <cuda_runtime.h>

#include "bp_ctx.h"

bp_status bpg_dense_tc_iterate(bp_ctx *h, int n_iters) {
    (void)n_iters;
    return bpg_fail(h, BP_ERR_UNSUPPORTED, "bp_iterate_dense: tensor-core baseline not available in this build");
}
