// Recorded log-domain forward and its adjoint (bp_backward).
#include <cuda_runtime.h>

#include "bp_ctx.h"

void bpg_free_extras(bp_ctx *h) {
    bpg_free_tc(h);
    for (void *p : h->ckpts)
        if (p) cudaFree(p);
    h->ckpts.clear();
    void *bufs[] = {h->seg_buf, h->adj[0], h->adj[1], h->dtab_partial, h->tc_a, h->tc_b, h->tc_z};
    for (void *p : bufs)
        if (p) cudaFree(p);
}

bp_status bpg_record_forward(bp_ctx *h, int n_iters) {
    (void)n_iters;
    return bpg_fail(h, BP_ERR_UNSUPPORTED, "bp_iterate: BP_RECORD is not available in this build");
}

extern "C" bp_status bp_backward(bp_handle h, const float *dev_dlogb, float *dev_dlogg, double *host_dtable,
                                 double *host_dfbar) {
    (void)dev_dlogb; (void)dev_dlogg; (void)host_dtable; (void)host_dfbar;
    if (!h) return BP_ERR_ARG;
    return bpg_fail(h, BP_ERR_UNSUPPORTED, "bp_backward is not available in this build");
}
