// Coarse-to-fine (multi-scale) message passing of [2], run in tandem with the
// O(mM) update (Sec. 2, Sec. 6).
//
// Level l+1 has one node per 2 x 2 block of level l; its unary is the product
// of the block's unaries, scaled to maximum 1 per node and formed in logs
// (sum of energies for min-sum); every level uses the handle's pairwise
// potential.  BP runs on the coarsest level from uniform
// messages, then each finer level starts from the coarser level's final
// messages copied by direction (the message into (r, c) from side s starts as
// the one into (r/2, c/2) from side s; uniform where the coarse node has no
// neighbour on that side) and runs its own iterations.  Each coarse level is a
// child handle owned by the grid's handle, so every level runs on the same
// kernels as bp_iterate.
#include <cuda_runtime.h>

#include <vector>

#include "trace.h"
#include "bp_ctx.h"

namespace {

// One warp per coarse node.  The coarse unary is the product of the block's
// unaries up to a per-node scale (BP does not see that scale).  It is built in
// logs: lu_coarse(x) = sum over the block of lu_fine(x), minus its maximum over
// x, so lu <= 0 stays finite at every level and g = exp(lu) has maximum 1 --
// the product of 4^l pixel unaries would leave FP32's range.  `fine_log` is
// the finer level's log unary, or NULL on the first level (then log g of the
// grid's own unary is taken).
__global__ void coarsen_f32_kernel(const float *fine_g, const float *fine_log, float *coarse_g, float *coarse_log,
                                   int Wf, int Hf, int Wc, int Hc, int M, int Mp) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long node = warp; node < (long long)Wc * Hc; node += nwarps) {
        const int r = (int)(node / Wc), c = (int)(node - (long long)r * Wc);
        float mx = -3.0e38f;
        for (int x = lane; x < M; x += 32) {
            float sl = 0.f;
            for (int dr = 0; dr < 2; ++dr)
                for (int dc = 0; dc < 2; ++dc) {
                    const int fr = 2 * r + dr, fc = 2 * c + dc;
                    if (fr < Hf && fc < Wf) {
                        const long long o = ((long long)fr * Wf + fc) * Mp + x;
                        sl += fine_log ? fine_log[o] : logf(fine_g[o]);
                    }
                }
            coarse_log[node * Mp + x] = sl;
            mx = fmaxf(mx, sl);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        for (int x = lane; x < Mp; x += 32) {
            const float lv = x < M ? coarse_log[node * Mp + x] - mx : -3.0e38f;
            coarse_log[node * Mp + x] = x < M ? lv : 0.f;
            coarse_g[node * Mp + x] = x < M ? expf(lv) : 0.f;
        }
    }
}

__global__ void coarsen_i32_kernel(const int32_t *fine, int32_t *coarse, int Wf, int Hf, int Wc, int Hc, int M,
                                   int Mp) {
    const long long n = (long long)Wc * Hc * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long node = i / Mp;
        const int x = (int)(i - node * Mp);
        const int r = (int)(node / Wc), c = (int)(node - (long long)r * Wc);
        int32_t e = 0;
        if (x < M)
            for (int dr = 0; dr < 2; ++dr)
                for (int dc = 0; dc < 2; ++dc) {
                    const int fr = 2 * r + dr, fc = 2 * c + dc;
                    if (fr < Hf && fc < Wf) e += fine[((long long)fr * Wf + fc) * Mp + x];
                }
        coarse[i] = e;
    }
}

template <typename E>
__global__ void upsample_kernel(const E *coarse, E *fine, int Wc, int Hc, int Wf, int Hf, int M, int Mp, E fill) {
    const long long planef = (long long)Wf * Hf * Mp, planec = (long long)Wc * Hc * Mp;
    const long long n = 4 * planef;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i / planef);
        const long long rem = i - s * planef;
        const long long node = rem / Mp;
        const int x = (int)(rem - node * Mp);
        const int r = (int)(node / Wf), c = (int)(node - (long long)r * Wf);
        const int pr = r >> 1, pc = c >> 1;
        const bool parent_has = (s == 0) ? pc > 0 : (s == 1) ? pc < Wc - 1 : (s == 2) ? pr > 0 : pr < Hc - 1;
        E v = x < M ? fill : E(0);
        if (parent_has) v = coarse[s * planec + ((long long)pr * Wc + pc) * Mp + x];
        fine[i] = v;
    }
}

bp_status ms_ck(bp_ctx *h, cudaError_t e, const char *where) {
    return e == cudaSuccess ? BP_OK : bpg_cuda_fail(h, e, where);
}

}  // namespace

void bpg_free_levels(bp_ctx *h) {
    for (bp_ctx *c : h->levels) bp_destroy(c);
    h->levels.clear();
}

extern "C" bp_status bp_iterate_multiscale(bp_handle h, int n_levels, const int *host_iters, int mode,
                                           bp_schedule schedule) {
    BPG_TRACE("bp_iterate_multiscale");
    if (!h) return bpg_fail(nullptr, BP_ERR_ARG, "bp_iterate_multiscale: NULL handle");
    h->err.clear();
    if (n_levels < 1 || n_levels > 16 || !host_iters) return bpg_fail(h, BP_ERR_ARG, "bp_iterate_multiscale: bad levels");
    for (int k = 0; k < n_levels; ++k)
        if (host_iters[k] < 0) return bpg_fail(h, BP_ERR_ARG, "bp_iterate_multiscale: negative iteration count");
    if (mode != BP_SUM && mode != BP_MAX) return bpg_fail(h, BP_ERR_ARG, "bp_iterate_multiscale: mode BP_SUM or BP_MAX");
    if (!h->have_unary || !h->have_potential)
        return bpg_fail(h, BP_ERR_STATE, "bp_iterate_multiscale: set the unary and the potential first");
    if (bp_status st = bpg_check_device(h)) return st;
    // the level dimensions; rebuild the children when they change
    std::vector<int> Ws{h->W}, Hs{h->H};
    for (int l = 1; l < n_levels; ++l) {
        Ws.push_back((Ws.back() + 1) / 2);
        Hs.push_back((Hs.back() + 1) / 2);
    }
    bool rebuild = (int)h->levels.size() != n_levels - 1;
    for (int l = 1; l < n_levels && !rebuild; ++l)
        rebuild = h->levels[l - 1]->W != Ws[l] || h->levels[l - 1]->H != Hs[l];
    if (rebuild) {
        bpg_free_levels(h);
        for (int l = 1; l < n_levels; ++l) {
            bp_handle c = nullptr;
            bp_status st = bp_create(Ws[l], Hs[l], h->M, h->dtype, (void *)h->stream, &c);
            if (st) return bpg_fail(h, st, std::string("bp_iterate_multiscale: level handle: ") + bp_last_error(nullptr));
            h->levels.push_back(c);
        }
    }
    // potential and unary of every coarse level
    for (int l = 1; l < n_levels; ++l) {
        bp_ctx *c = h->levels[l - 1];
        bp_status st;
        if (h->sparse)
            st = bp_set_potential_sparse(c, h->sp_rowptr.data(), h->sp_cols.data(),
                                         h->dtype == BP_F32 ? (const void *)h->sp_valf.data() : (const void *)h->sp_vali.data(),
                                         h->fbar);
        else
            st = bp_set_potential(c, h->dtype == BP_F32 ? (const void *)h->tablef.data() : (const void *)h->tablei.data(),
                                  h->T, h->fbar);
        if (st) return bpg_fail(h, st, std::string("bp_iterate_multiscale: level potential: ") + bp_last_error(c));
        bp_set_layout(c, h->layout.L, h->layout.C);
        bp_set_persistent(c, h->persistent);
        const bp_ctx *f = l == 1 ? h : h->levels[l - 2];
        const long long n = (long long)c->W * c->H * c->Mp;
        if (h->dtype == BP_F32) {
            if (!c->ms_logu)
                if (bp_status st2 = bpg_ensure_buffer(c, &c->ms_logu, (size_t)n * 4, "level log unary")) return st2;
            coarsen_f32_kernel<<<bpg::grid_for((long long)c->W * c->H * 32, 256), 256, 0, h->stream>>>(
                (const float *)f->unary, l == 1 ? nullptr : (const float *)f->ms_logu, (float *)c->unary,
                (float *)c->ms_logu, f->W, f->H, c->W, c->H, h->M, h->Mp);
        }
        else
            coarsen_i32_kernel<<<bpg::grid_for(n, 256), 256, 0, h->stream>>>(
                (const int32_t *)f->unary, (int32_t *)c->unary, f->W, f->H, c->W, c->H, h->M, h->Mp);
        if (bp_status st2 = ms_ck(h, cudaGetLastError(), "coarsen launch")) return st2;
        h->launches += 1;
        c->have_unary = true;
        c->log_unary_valid = false;
        c->recorded = false;
    }
    // coarsest first, then copy down and iterate at each finer level
    for (int k = 0; k < n_levels; ++k) {
        const int l = n_levels - 1 - k;
        bp_ctx *cur = l == 0 ? h : h->levels[l - 1];
        if (k == 0) {
            bp_reset_messages(cur);
        } else {
            bp_ctx *coarse = h->levels[l];   // level l + 1
            // the coarse result must be in linear form (it is: BP_SUM / BP_MAX runs)
            const long long n = 4LL * cur->W * cur->H * cur->Mp;
            if (h->dtype == BP_F32)
                upsample_kernel<float><<<bpg::grid_for(n, 256), 256, 0, h->stream>>>(
                    (const float *)coarse->msg[coarse->cur], (float *)cur->msg[cur->cur], coarse->W, coarse->H, cur->W,
                    cur->H, h->M, h->Mp, 1.0f / (float)h->M);
            else
                upsample_kernel<int32_t><<<bpg::grid_for(n, 256), 256, 0, h->stream>>>(
                    (const int32_t *)coarse->msg[coarse->cur], (int32_t *)cur->msg[cur->cur], coarse->W, coarse->H,
                    cur->W, cur->H, h->M, h->Mp, 0);
            if (bp_status st = ms_ck(h, cudaGetLastError(), "upsample launch")) return st;
            h->launches += 1;
            cur->msg_uniform = false;
            cur->msg_log = false;
            cur->recorded = false;
        }
        const long long before = cur->launches;
        bp_status st = bp_iterate(cur, host_iters[k], mode, schedule);
        if (cur != h) h->launches += cur->launches - before;
        if (st) return cur == h ? st : bpg_fail(h, st, std::string("bp_iterate_multiscale: level ") + std::to_string(l) +
                                                           ": " + bp_last_error(cur));
    }
    return BP_OK;
}
