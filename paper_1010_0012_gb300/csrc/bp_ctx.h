// The handle behind bp_handle, and the functions the C-ABI translation units
// share.  Internal; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/bp.h"
#include "bp_internal.h"

struct GraphKey {
    int n, mode, sched, cur, L, C, blocks, persist;
    bool operator<(const GraphKey &o) const {
        return std::tie(n, mode, sched, cur, L, C, blocks, persist) <
               std::tie(o.n, o.mode, o.sched, o.cur, o.L, o.C, o.blocks, o.persist);
    }
};

struct GraphEntry {
    cudaGraphExec_t exec;
    int launches;   // kernels per replay
    int end_cur;    // buffer holding the messages after the replay
};

struct bp_ctx {
    int W = 0, H = 0, M = 0, Mp = 0;
    bp_dtype dtype = BP_F32;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bpg::GridDims dims{};

    void *unary = nullptr;          // [H][W][Mp] g (F32) or E_u (I32)
    float *log_unary = nullptr;     // [H][W][Mp] log g, built on demand
    bool log_unary_valid = false;
    void *msg[2] = {nullptr, nullptr};  // two [4][H][W][Mp] states
    int cur = 0;                    // state holding the current messages
    bool msg_uniform = true;        // reset pending (filled on first use)
    bool msg_log = false;           // current state holds log-messages

    bool have_unary = false, have_potential = false;
    int T = 0, Teff = 0;            // requested and effective (<= M - 1) band half-width
    double fbar = 0;
    float fbarf = 0;
    int32_t ebar = 0;
    std::vector<float> tablef, wf;  // f(d) and f(d) - fbar
    std::vector<int32_t> tablei, wi;
    float *d_wf = nullptr;          // device band tables for the generic kernels
    int32_t *d_wi = nullptr;
    void *d_dense = nullptr;        // device M x M table for the CUDA-core dense baseline

    // general sparse compatibility (bp_set_potential_sparse)
    bool sparse = false;
    std::vector<int32_t> sp_rowptr, sp_cols;
    std::vector<float> sp_valf;      // f(x_i, x_j)
    std::vector<int32_t> sp_vali;    // E(x_i, x_j)
    void *d_sp_len = nullptr, *d_sp_ell = nullptr;   // device pattern (see bp_sparse.h)
    // register-pattern schedule (sparse_reg_plan.cu), when the pattern fits one
    bool sp_reg = false;
    bool sp_p16 = false;    // min-sum register kernel on 16-bit label pairs (Ebar <= kP16MaxEbar)
    int sp_KM = 0, sp_LM = 0, sp_steps = 0, sp_wavefronts = 0;
    void *d_sp_rent = nullptr, *d_sp_rlab = nullptr;
    int sp_kernel = 0;               // BP_SPARSE_AUTO / _LISTS / _REGISTERS
    uint8_t *d_stereo = nullptr;     // staging of host images for bp_set_unary_stereo (2 W H bytes)

    bpg::Layout layout{32, 1};
    bpg::Layout log_layout{32, 1};  // layout of the log-domain forward and adjoint kernels
    bpg::Layout adj_layout{32, 1};  // layout of the adjoint kernel (reads states and scales, any layout)
    bpg::Layout rec_layout{32, 1};  // log layout of the recorded run (its recompute must match it bit for bit)
    bool fast = false;              // register/shuffle kernels serve (M, T)
    int blocks_override = 0;
    bool use_graphs = true;
    std::map<GraphKey, GraphEntry> graphs;

    int *d_status = nullptr;        // device error word (bounded waits)
    void *tune_buf = nullptr;
    long long launches = 0;
    std::string err;

    // recorded log-domain forward (bp_backward)
    int ckpt_every = 5;
    bool recorded = false;
    int rec_iters = 0;
    std::vector<void *> ckpts;      // states at t = 0, every, 2 every, ...
    void *seg_buf = nullptr;        // recomputed states of one segment
    int seg_cap = 0;
    bool last_seg_kept = false;     // seg_buf holds the recorded run's last segment
    void *stats_buf = nullptr;      // [iterations][4][H][W] float2 (C, S/Z) of the recorded run
    size_t stats_cap = 0;
    void *adj[2] = {nullptr, nullptr};   // adjoint message states
    void *dtab_partial = nullptr;   // per-(iteration, block) partial sums of d table, d fbar
    size_t dtab_cap = 0;
    void *dlogg_pad = nullptr;      // [H][W][Mp] accumulated dL/d log g
    void *d_red = nullptr;          // FP64 reduced parameter gradients
    int rec_every = 5;

    // one persistent launch per bp_iterate call (small grids): a one-MRF
    // descriptor and work items for the persistent kernel of the batch path
    int persistent = -1;            // -1 automatic, 0 never, 1 always (when served)
    void *p_mrf = nullptr;          // device BatchMrf
    void *p_items[2] = {nullptr, nullptr};   // synchronous / red-black slot items
    int p_nitems[2] = {0, 0};
    void *p_bar = nullptr;          // grid-barrier words
    bool p_ready = false;           // descriptor matches the current potential

    // coarse levels of bp_iterate_multiscale (child handles, level 1..L-1)
    std::vector<bp_ctx *> levels;
    void *ms_logu = nullptr;        // a level's log unary, scaled to maximum 0 (float)

    // tensor-core dense baseline
    void *tc_a = nullptr;           // packed h rows, bf16 [4*H*W][Mp]
    void *tc_b = nullptr;           // F^T, bf16 [Mp][Mp]
    void *tc_z = nullptr;
    void *tc_maps = nullptr;        // host-side tensor maps (dense_tc.cu)
    bool tc_ready = false;
};

bp_status bpg_fail(bp_ctx *h, bp_status st, const std::string &msg);
bp_status bpg_cuda_fail(bp_ctx *h, cudaError_t e, const char *where);
bp_status bpg_ensure_buffer(bp_ctx *h, void **p, size_t bytes, const char *what);
bp_status bpg_check_device(bp_ctx *h);
size_t bpg_plane_bytes(const bp_ctx *h);
size_t bpg_state_bytes(const bp_ctx *h);
cudaError_t bpg_issue_iteration(bp_ctx *h, int mode, int sched, int &cur, int &count);

bp_status bpg_record_forward(bp_ctx *h, int n_iters);   // bp_backward.cu
float bpg_pair_value_f(const bp_ctx *h, int xi, int xj);   // bp_api.cu
bool bpg_zero_min(const std::vector<int32_t> &w);
bool bpg_packed16(const std::vector<int32_t> &w, int32_t ebar);
int32_t bpg_pair_value_i(const bp_ctx *h, int xi, int xj);
void bpg_free_extras(bp_ctx *h);                         // bp_backward.cu
bp_status bpg_dense_tc_iterate(bp_ctx *h, int n_iters);  // dense_tc.cu
bp_status bpg_dense_tc_iterate_kind(bp_ctx *h, int n_iters, bool fused);
void bpg_free_tc(bp_ctx *h);                             // dense_tc.cu
void bpg_free_levels(bp_ctx *h);                         // bp_multiscale.cu

namespace bpg {
cudaError_t launch_domain_convert(float *planes, long long rows, int M, int Mp, int to_log, cudaStream_t s);
cudaError_t launch_domain_convert_copy(const float *g, float *logg, long long nodes, int M, int Mp, cudaStream_t s);
cudaError_t launch_domain_convert_dense(float *p, long long n, int to_log, cudaStream_t s);
}  // namespace bpg
