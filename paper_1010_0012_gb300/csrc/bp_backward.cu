// Recorded log-domain forward (checkpoints) and its reverse (bp_backward).
//
// Forward with BP_RECORD: the message state entering iterations 0, c, 2c, ...
// is kept as a checkpoint (c = checkpoint interval), and the last segment's
// states are kept whole.  Backward walks the segments from the last to the
// first: it recomputes the states of a segment from its checkpoint with the
// same forward kernel (so bit-identical to the recorded run; the last segment
// needs none), then applies the adjoint kernel once per iteration in
// reverse, accumulating dL/d log g and per-block sums of dL/df(d), dL/dfbar;
// those sums are reduced over all blocks and iterations in FP64.
#include <cuda_runtime.h>

#include <vector>

#include "trace.h"
#include "bp_adjoint.h"
#include "bp_ctx.h"

using namespace bpg;

void bpg_free_extras(bp_ctx *h) {
    bpg_free_tc(h);
    bpg_free_levels(h);
    for (void *p : h->ckpts)
        if (p) cudaFree(p);
    h->ckpts.clear();
    void *bufs[] = {h->seg_buf, h->adj[0], h->adj[1], h->dtab_partial, h->tc_a, h->tc_b, h->tc_z, h->dlogg_pad,
                    h->d_red, h->p_mrf, h->p_items[0], h->p_items[1], h->p_bar, h->ms_logu, h->stats_buf};
    for (void *p : bufs)
        if (p) cudaFree(p);
}

#define BK_CK(h, call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return bpg_cuda_fail((h), e_, #call);     \
    } while (0)

static BandArgsLogF log_args(bp_ctx *h, const void *in, void *out) {
    BandArgsLogF a{};
    a.g = h->log_unary;
    a.in = (const float *)in;
    a.out = (float *)out;
    a.d = h->dims;
    a.parity = -1;
    a.T = h->Teff;
    for (int i = 0; i < 2 * h->Teff + 1; ++i) a.w[i] = h->wf[i];
    a.fbar = h->fbarf;
    return a;
}

// The states of a segment after its checkpoint (c - 1 of them) live in one buffer.
static bp_status ensure_segment_buffer(bp_ctx *h, int c) {
    const int seg_states = c > 1 ? c - 1 : 1;
    if (h->seg_cap >= seg_states) return BP_OK;
    if (h->seg_buf) {
        cudaFree(h->seg_buf);
        h->seg_buf = nullptr;
    }
    h->seg_cap = 0;
    if (bp_status st = bpg_ensure_buffer(h, &h->seg_buf, bpg_state_bytes(h) * seg_states, "segment states")) return st;
    h->seg_cap = seg_states;
    return BP_OK;
}

// The recorded forward writes each checkpoint directly: the iteration that
// ends at t = c, 2c, ... stores its output in that checkpoint, and the next
// iteration reads it from there.  Only the state entering iteration 0 is
// copied.  The states of the last segment after its checkpoint go to the
// segment buffer, where the backward finds them without recomputing.
bp_status bpg_record_forward(bp_ctx *h, int n_iters) {
    const int c = h->ckpt_every;
    const int n_ck = (n_iters + c - 1) / c;
    const size_t sb = bpg_state_bytes(h);
    while ((int)h->ckpts.size() < n_ck) {
        void *p = nullptr;
        if (bp_status st = bpg_ensure_buffer(h, &p, sb, "checkpoint")) return st;
        h->ckpts.push_back(p);
    }
    if (bp_status st = ensure_segment_buffer(h, c)) return st;
    const size_t stats_per_iter = (size_t)4 * h->W * h->H;   // float2 per message, [H][W][4]
    const size_t stats_bytes = stats_per_iter * sizeof(float2) * (n_iters > 0 ? n_iters : 1);
    if (h->stats_cap < stats_bytes) {
        if (h->stats_buf) {
            cudaFree(h->stats_buf);
            h->stats_buf = nullptr;
        }
        h->stats_cap = 0;
        if (bp_status st = bpg_ensure_buffer(h, &h->stats_buf, stats_bytes, "forward scales")) return st;
        h->stats_cap = stats_bytes;
    }
    const int last_start = (n_ck - 1) * c;
    h->rec_layout = h->log_layout;
    void *state = h->msg[h->cur];
    if (n_iters > 0) BK_CK(h, cudaMemcpyAsync(h->ckpts[0], state, sb, cudaMemcpyDeviceToDevice, h->stream));
    for (int t = 0; t < n_iters; ++t) {
        const int t1 = t + 1;   // the state this iteration produces enters iteration t1
        void *out;
        if (t1 < n_iters && t1 % c == 0)
            out = h->ckpts[t1 / c];
        else if (t1 < n_iters && t1 > last_start)
            out = (char *)h->seg_buf + (size_t)(t1 - last_start - 1) * sb;
        else
            out = state == h->msg[0] ? h->msg[1] : h->msg[0];
        BandArgsLogF la = log_args(h, state, out);
        la.stats = (float2 *)h->stats_buf + (size_t)t * stats_per_iter;
        BK_CK(h, launch_band_log(la, h->rec_layout, h->blocks_override, h->stream));
        h->launches += 1;
        state = out;
    }
    h->cur = state == h->msg[0] ? 0 : 1;
    h->rec_iters = n_iters;
    h->rec_every = c;
    h->recorded = true;
    h->last_seg_kept = n_iters > 0;
    return BP_OK;
}

// The reverse pass of bp_backward / bp_backward_device.  dtable and dfbar
// are host memory (written after a synchronisation of the handle's stream) or,
// with device_out, device memory written by copies on that stream.
static bp_status backward_impl(bp_ctx *h, const char *name, const float *dev_dlogb, float *dev_dlogg,
                               double *dtable, double *dfbar, bool device_out) {
    if (!h) return bpg_fail(nullptr, BP_ERR_ARG, std::string(name) + ": NULL handle");
    h->err.clear();
    if (!dev_dlogb || !dev_dlogg || !dtable || !dfbar)
        return bpg_fail(h, BP_ERR_ARG, std::string(name) + ": NULL argument");
    if (!h->recorded || !h->msg_log)
        return bpg_fail(h, BP_ERR_STATE, std::string(name) + ": run bp_iterate with BP_SUM|BP_LOG|BP_RECORD first");
    if (!h->fast) return bpg_fail(h, BP_ERR_UNSUPPORTED, std::string(name) + ": needs T <= 8 and M <= 512");
    if (bp_status st = bpg_check_device(h)) return st;
    const int K = h->rec_iters, c = h->rec_every, Teff = h->Teff, NP = 2 * Teff + 2;
    const size_t sb = bpg_state_bytes(h);
    const long long nodes = (long long)h->W * h->H;
    const int blocks = adjoint_blocks(h->dims, h->adj_layout, Teff);
    if (blocks < 1) return bpg_fail(h, BP_ERR_UNSUPPORTED, std::string(name) + ": no adjoint kernel for this layout");
    if (bp_status st = ensure_segment_buffer(h, c)) return st;
    if (bp_status st = bpg_ensure_buffer(h, &h->adj[0], sb, "adjoint state")) return st;
    if (bp_status st = bpg_ensure_buffer(h, &h->adj[1], sb, "adjoint state")) return st;
    if (bp_status st = bpg_ensure_buffer(h, &h->dlogg_pad, (size_t)nodes * h->Mp * 4, "dlogg")) return st;
    const long long rows = (long long)K * blocks;
    const size_t pbytes = (size_t)(rows > 0 ? rows : 1) * NP * 4;
    if (h->dtab_cap < pbytes) {
        if (h->dtab_partial) { cudaFree(h->dtab_partial); h->dtab_partial = nullptr; }
        if (bp_status st = bpg_ensure_buffer(h, &h->dtab_partial, pbytes, "gradient partial sums")) return st;
        h->dtab_cap = pbytes;
    }
    if (bp_status st = bpg_ensure_buffer(h, &h->d_red, (2 * kTMaxFast + 2) * sizeof(double), "gradient sums"))
        return st;

    // reverse of the beliefs: seeds the adjoint of the final messages and dL/d log g
    BK_CK(h, launch_beliefs_log_adjoint(h->log_unary, (const float *)h->msg[h->cur], dev_dlogb, h->dims,
                                        (float *)h->adj[0], (float *)h->dlogg_pad, h->stream));
    h->launches += 1;
    int ca = 0;
    const int n_ck = (K + c - 1) / c;
    std::vector<void *> states(c);
    for (int seg = n_ck - 1; seg >= 0; --seg) {
        const int start = seg * c, end = std::min(K, start + c), len = end - start;
        states[0] = h->ckpts[seg];
        // the last segment's states are still in the segment buffer from the
        // recorded run (unless a previous backward has overwritten it)
        const bool kept = seg == n_ck - 1 && h->last_seg_kept;
        for (int j = 1; j < len; ++j) {
            states[j] = (char *)h->seg_buf + (size_t)(j - 1) * sb;
            if (kept) continue;
            BK_CK(h, launch_band_log(log_args(h, states[j - 1], states[j]), h->rec_layout, h->blocks_override,
                                     h->stream));
            h->launches += 1;
        }
        h->last_seg_kept = false;   // the next segment's recompute overwrites the buffer
        for (int t = end - 1; t >= start; --t) {
            AdjArgs a{};
            a.logg = h->log_unary;
            a.ell = (const float *)states[t - start];
            a.lam_next = (const float *)h->adj[ca];
            a.lam = (float *)h->adj[ca ^ 1];
            a.dlogg = (float *)h->dlogg_pad;
            a.partial = (float *)h->dtab_partial + (size_t)t * blocks * NP;
            a.stats = (const float2 *)h->stats_buf + (size_t)t * 4 * nodes;
            a.d = h->dims;
            a.T = Teff;
            for (int i = 0; i < 2 * Teff + 1; ++i) a.w[i] = h->wf[i];
            a.fbar = h->fbarf;
            BK_CK(h, launch_band_log_adjoint(a, h->adj_layout, blocks, h->stream));
            h->launches += 1;
            ca ^= 1;
        }
    }
    if (rows > 0) {
        BK_CK(h, launch_reduce_partials_f64((const float *)h->dtab_partial, rows, NP, (double *)h->d_red, h->stream));
        h->launches += 1;
    } else {
        BK_CK(h, cudaMemsetAsync(h->d_red, 0, NP * sizeof(double), h->stream));
    }
    BK_CK(h, launch_unpad_copy(h->dlogg_pad, dev_dlogg, nodes, h->M, h->Mp, h->stream));
    h->launches += 1;
    // d_red holds dL/df(d) for |d| <= Teff, then dL/dfbar; table entries with
    // |d| > Teff (T >= M) meet no label pair and get 0
    const int T = h->T;
    if (device_out) {
        if (T > Teff) BK_CK(h, cudaMemsetAsync(dtable, 0, (size_t)(2 * T + 1) * sizeof(double), h->stream));
        BK_CK(h, cudaMemcpyAsync(dtable + (T - Teff), h->d_red, (size_t)(2 * Teff + 1) * sizeof(double),
                                 cudaMemcpyDeviceToDevice, h->stream));
        BK_CK(h, cudaMemcpyAsync(dfbar, (const double *)h->d_red + (NP - 1), sizeof(double), cudaMemcpyDeviceToDevice,
                                 h->stream));
        return BP_OK;
    }
    std::vector<double> red(NP, 0.0);
    BK_CK(h, cudaMemcpyAsync(red.data(), h->d_red, NP * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (bp_status st = bp_sync(h)) return st;
    for (int d = -T; d <= T; ++d) dtable[d + T] = (d >= -Teff && d <= Teff) ? red[d + Teff] : 0.0;
    *dfbar = red[NP - 1];
    return BP_OK;
}

extern "C" bp_status bp_backward(bp_handle h, const float *dev_dlogb, float *dev_dlogg, double *host_dtable,
                                 double *host_dfbar) {
    BPG_TRACE("bp_backward");
    return backward_impl(h, "bp_backward", dev_dlogb, dev_dlogg, host_dtable, host_dfbar, false);
}

extern "C" bp_status bp_backward_device(bp_handle h, const float *dev_dlogb, float *dev_dlogg, double *dev_dtable,
                                        double *dev_dfbar) {
    BPG_TRACE("bp_backward_device");
    return backward_impl(h, "bp_backward_device", dev_dlogb, dev_dlogg, dev_dtable, dev_dfbar, true);
}
