// C-ABI layer: handle ownership, argument validation, the iteration driver
// (schedules, CUDA-graph replay) and the tuning entry points.  Declarations
// and the contract of every call are in include/bp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "trace.h"
#include "../../include/bp.h"
#include "bp_batch_internal.h"
#include "bp_internal.h"
#include "bp_ctx.h"
#include "bp_sparse.h"

namespace bpg {
cudaError_t launch_batch_sum(const BatchArgs &a, int family, int blocks, cudaStream_t s);
cudaError_t launch_batch_min(const BatchArgs &a, int family, int blocks, cudaStream_t s);
int batch_max_blocks_sum(int family, bool redblack = false, bool full = false);
int batch_max_blocks_min(int family, bool redblack = false, bool full = false);
}  // namespace bpg

using namespace bpg;

namespace {

thread_local std::string g_global_err;

bp_status fail(bp_ctx *h, bp_status st, const std::string &msg) {
    if (h) h->err = msg; else g_global_err = msg;
    if (st != BP_OK) log_error(st, msg);
    return st;
}

bp_status cuda_fail(bp_ctx *h, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(h, BP_ERR_OOM, m);
    return fail(h, BP_ERR_CUDA, m);
}

#define BP_CK(h, call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

size_t elem_bytes() { return 4; }

}  // namespace

// ------------------------------------------------------------------ helpers --

bp_status bpg_check_device(bp_ctx *h) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
    if (dev != h->device) return fail(h, BP_ERR_STATE, "the current CUDA device differs from the handle's device");
    return BP_OK;
}

static void clear_graphs(bp_ctx *h) {
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
    h->graphs.clear();
}

static bp_status ensure_buffer(bp_ctx *h, void **p, size_t bytes, const char *what) {
    if (*p) return BP_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_fail(h, e, what);
    }
    return BP_OK;
}

size_t bpg_plane_bytes(const bp_ctx *h) { return (size_t)h->dims.plane * elem_bytes(); }
size_t bpg_state_bytes(const bp_ctx *h) { return 4 * bpg_plane_bytes(h); }

// Make the current message buffer hold the representation `want_log`.
static bp_status materialize(bp_ctx *h, bool want_log) {
    const long long rows = 4LL * h->W * h->H;
    if (h->msg_uniform) {
        if (h->dtype == BP_I32) {
            BP_CK(h, launch_fill_messages_i32((int32_t *)h->msg[h->cur], rows, h->M, h->Mp, 0, h->stream));
        } else {
            const float v = want_log ? -log2f((float)h->M) : 1.0f / (float)h->M;   // log domain: base 2
            BP_CK(h, launch_fill_messages_f32((float *)h->msg[h->cur], rows, h->M, h->Mp, v, h->stream));
        }
        h->launches += 1;
        h->msg_uniform = false;
        h->msg_log = want_log && h->dtype == BP_F32;
        return BP_OK;
    }
    if (h->dtype == BP_F32 && h->msg_log != want_log) {
        BP_CK(h, launch_domain_convert((float *)h->msg[h->cur], rows, h->M, h->Mp, want_log ? 1 : 0, h->stream));
        h->launches += 1;
        h->msg_log = want_log;
    }
    return BP_OK;
}

static bp_status ensure_log_unary(bp_ctx *h) {
    if (h->log_unary_valid) return BP_OK;
    bp_status st = ensure_buffer(h, (void **)&h->log_unary, (size_t)h->W * h->H * h->Mp * 4, "log unary");
    if (st) return st;
    BP_CK(h, launch_domain_convert_copy((const float *)h->unary, h->log_unary, (long long)h->W * h->H, h->M, h->Mp,
                                        h->stream));
    h->launches += 1;
    h->log_unary_valid = true;
    return BP_OK;
}

// Issue the kernels of one O(mM) iteration (one or two launches).
static cudaError_t issue_iteration(bp_ctx *h, int mode, int sched, int &cur, int &count) {
    const bool is_log = (mode & BP_LOG) != 0;
    const int nsteps = sched == BP_REDBLACK ? 2 : 1;
    for (int step = 0; step < nsteps; ++step) {
        const int parity = sched == BP_REDBLACK ? step : -1;
        void *in = h->msg[cur];
        void *out = sched == BP_REDBLACK ? h->msg[cur] : h->msg[cur ^ 1];
        cudaError_t e;
        if (h->sparse) {
            if (is_log) return cudaErrorNotSupported;
            if (h->sp_reg && h->sp_kernel != BP_SPARSE_LISTS) {
                SparseRegArgs a{h->unary, in, out, h->dims, parity, (const int2 *)h->d_sp_rent,
                                (const int32_t *)h->d_sp_rlab, h->fbarf, h->ebar, h->d_status, {}};
                e = h->dtype != BP_I32 ? launch_sparse_reg_sum(a, h->sp_KM, h->sp_LM, h->stream)
                    : h->sp_p16        ? launch_sparse_reg_min16(a, h->sp_KM, h->sp_LM, h->stream)
                                       : launch_sparse_reg_min(a, h->sp_KM, h->sp_LM, h->stream);
                if (e != cudaSuccess) return e;
                ++count;
                continue;
            }
            if (h->dtype == BP_I32) {
                SparseArgsI a{(const int32_t *)h->unary, (const int32_t *)in, (int32_t *)out, h->dims, parity,
                              (const int32_t *)h->d_sp_len, (const int2 *)h->d_sp_ell, h->ebar};
                e = launch_sparse_min(a, h->stream);
            } else {
                SparseArgsF a{(const float *)h->unary, (const float *)in, (float *)out, h->dims, parity,
                              (const int32_t *)h->d_sp_len, (const int2 *)h->d_sp_ell, h->fbarf};
                e = launch_sparse_sum(a, h->stream);
            }
            if (e != cudaSuccess) return e;
            ++count;
            continue;
        }
        if (h->dtype == BP_I32) {
            if (h->fast) {
                BandArgsI a{};
                a.e = (const int32_t *)h->unary; a.in = (const int32_t *)in; a.out = (int32_t *)out;
                a.d = h->dims; a.parity = parity; a.T = h->Teff;
                for (int i = 0; i < 2 * h->Teff + 1; ++i) a.w[i] = h->wi[i];
                a.ebar = h->ebar;
                a.zero_min = bpg_zero_min(h->wi) ? 1 : 0;
                a.packed16 = bpg_packed16(h->wi, h->ebar) ? 1 : 0;
                e = launch_band_min(a, h->layout, h->blocks_override, h->stream);
            } else {
                BandArgsGenericI a{(const int32_t *)h->unary, (const int32_t *)in, (int32_t *)out, h->dims,
                                   parity, h->Teff, h->d_wi, h->ebar};
                e = launch_band_min_generic(a, h->stream);
            }
        } else if (h->fast) {
            BandArgsLogF a{};   // stats stay NULL: only the recorded run keeps the scales
            a.g = is_log ? h->log_unary : (const float *)h->unary;
            a.in = (const float *)in; a.out = (float *)out;
            a.d = h->dims; a.parity = parity; a.T = h->Teff;
            for (int i = 0; i < 2 * h->Teff + 1; ++i) a.w[i] = h->wf[i];
            a.fbar = h->fbarf;
            e = is_log ? launch_band_log(a, h->log_layout, h->blocks_override, h->stream)
                       : launch_band_sum(a, h->layout, h->blocks_override, h->stream);
        } else {
            if (is_log) return cudaErrorNotSupported;
            BandArgsGenericF a{(const float *)h->unary, (const float *)in, (float *)out, h->dims, parity,
                               h->Teff, h->d_wf, h->fbarf};
            e = launch_band_sum_generic(a, h->stream);
        }
        if (e != cudaSuccess) return e;
        ++count;
    }
    if (sched != BP_REDBLACK) cur ^= 1;
    return cudaSuccess;
}

// ---- one persistent launch for a whole bp_iterate call -----------------------
// Served for the linear sum-product and min-sum updates with 16 <= Mp <= 256
// and T <= 8 (the label classes of the persistent kernel), on request.  The
// automatic choice is the per-launch form: on GB300, graph-replayed kernel
// boundaries (2.7 us per iteration at 32x32, 6.1 us per red-black half-step
// at 384x288) measured faster than this kernel's grid barrier and per-step
// descriptor reads (5.0 us and 10.2 us).
static bool persistent_served(const bp_ctx *h, int mode) {
    return h->fast && !h->sparse && !(mode & BP_LOG) && h->Mp >= 16 && h->Mp <= 256 && h->Teff <= kTMaxFast;
}

static bool use_persistent(const bp_ctx *h, int mode) {
    return h->persistent == 1 && persistent_served(h, mode);
}

static bp_status persistent_setup(bp_ctx *h) {
    if (h->p_ready) return BP_OK;
    BatchMrf m{};
    m.unary = h->unary;
    m.msg[0] = h->msg[0];
    m.msg[1] = h->msg[1];
    m.plane = h->dims.plane;
    m.W = h->W; m.H = h->H; m.M = h->M; m.Mp = h->Mp; m.T = h->Teff;
    if (h->dtype == BP_F32) {
        for (int i = 0; i < 2 * h->Teff + 1; ++i) m.wf[i] = h->wf[i];
        m.fbar = h->fbarf;
    } else {
        for (int i = 0; i < 2 * h->Teff + 1; ++i) m.wi[i] = h->wi[i];
        m.ebar = h->ebar;
        m.zero_min = bpg_zero_min(h->wi) ? 1 : 0;
        m.packed16 = bpg_packed16(h->wi, h->ebar) ? 1 : 0;
    }
    if (bp_status st = ensure_buffer(h, &h->p_mrf, sizeof(BatchMrf), "persistent descriptor")) return st;
    if (bp_status st = ensure_buffer(h, &h->p_bar, kBatchCtlWords * sizeof(unsigned), "barrier words")) return st;
    const int maxb = h->dtype == BP_I32 ? std::max(batch_max_blocks_min(1, false), batch_max_blocks_min(1, true))
                                        : std::max(batch_max_blocks_sum(1, false), batch_max_blocks_sum(1, true));
    const int gpb = kBlock / batch_lanes_per_node(1, h->Mp);
    for (int sched = 0; sched < 2; ++sched) {
        const int nslots = sched == BP_REDBLACK ? ((h->W + 1) / 2) * h->H : h->W * h->H;
        // about four items per resident block, whole node groups per item
        int tile = (nslots + 4 * maxb - 1) / (4 * maxb);
        tile = std::max(gpb, (tile + gpb - 1) / gpb * gpb);
        std::vector<BatchItem> items;
        for (int s0 = 0; s0 < nslots; s0 += tile) items.push_back(BatchItem{0, s0, std::min(tile, nslots - s0)});
        if (h->p_items[sched]) { cudaFree(h->p_items[sched]); h->p_items[sched] = nullptr; }
        if (bp_status st = ensure_buffer(h, &h->p_items[sched], items.size() * sizeof(BatchItem), "persistent items"))
            return st;
        BP_CK(h, cudaMemcpyAsync(h->p_items[sched], items.data(), items.size() * sizeof(BatchItem),
                                 cudaMemcpyHostToDevice, h->stream));
        h->p_nitems[sched] = (int)items.size();
        BP_CK(h, cudaStreamSynchronize(h->stream));   // the host vector dies here
    }
    BP_CK(h, cudaMemcpyAsync(h->p_mrf, &m, sizeof(BatchMrf), cudaMemcpyHostToDevice, h->stream));
    BP_CK(h, cudaMemsetAsync(h->p_bar, 0, kBatchCtlWords * sizeof(unsigned), h->stream));
    BP_CK(h, cudaStreamSynchronize(h->stream));
    h->p_ready = true;
    return BP_OK;
}

static cudaError_t issue_persistent(bp_ctx *h, int n, int sched, int cur) {
    BatchArgs a{};
    a.mrfs = (const BatchMrf *)h->p_mrf;
    a.items = (const BatchItem *)h->p_items[sched == BP_REDBLACK ? 1 : 0];
    a.n_items = h->p_nitems[sched == BP_REDBLACK ? 1 : 0];
    a.n_iters = n;
    a.start_buf = cur;
    a.redblack = sched == BP_REDBLACK ? 1 : 0;
    a.bar_count = (unsigned *)h->p_bar;
    a.bar_gen = (unsigned *)h->p_bar + kBatchGenWord;
    a.tickets = reinterpret_cast<unsigned long long *>((unsigned *)h->p_bar + kBatchTicketWord);
    a.extra_arrivals = 0;
    a.limit_ns = 2000000000ull;
    a.status = h->d_status;
    cudaError_t e = cudaMemsetAsync(h->p_bar, 0, kBatchZeroBytes, h->stream);   // arrivals, ticket counter
    if (e != cudaSuccess) return e;
    const bool rb = sched == BP_REDBLACK;
    const int maxb = h->dtype == BP_I32 ? batch_max_blocks_min(1, rb) : batch_max_blocks_sum(1, rb);
    const int blocks = std::max(1, std::min(maxb, a.n_items));
    return h->dtype == BP_I32 ? launch_batch_min(a, 1, blocks, h->stream) : launch_batch_sum(a, 1, blocks, h->stream);
}

// Run n iterations, through a cached CUDA graph when possible.
static bp_status run_iterations(bp_ctx *h, int n, int mode, int sched) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    BP_CK(h, cudaStreamIsCapturing(h->stream, &cap));
    const bool persist = use_persistent(h, mode);
    if (persist) {
        if (bp_status st = persistent_setup(h)) return st;
    }
    const bool use_graph = h->use_graphs && cap == cudaStreamCaptureStatusNone && (n > 1 || persist);
    if (!use_graph) {
        if (persist) {
            cudaError_t e = issue_persistent(h, n, sched, h->cur);
            if (e != cudaSuccess) return cuda_fail(h, e, "persistent O(mM) launch");
            h->launches += 1;
            if (sched != BP_REDBLACK) h->cur = (h->cur + n) & 1;
            return BP_OK;
        }
        for (int it = 0; it < n; ++it) {
            int count = 0;
            cudaError_t e = issue_iteration(h, mode, sched, h->cur, count);
            if (e != cudaSuccess) return cuda_fail(h, e, "O(mM) update launch");
            h->launches += count;
        }
        return BP_OK;
    }
    const Layout &lay = (mode & BP_LOG) ? h->log_layout : h->layout;
    const GraphKey key{n, mode, sched, h->cur, lay.L, lay.C, h->blocks_override, persist ? 1 : 0};
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        cudaGraph_t g = nullptr;
        BP_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int cur = h->cur, count = 0;
        cudaError_t e = cudaSuccess;
        if (persist) {
            e = issue_persistent(h, n, sched, cur);
            count = 1;
            if (sched != BP_REDBLACK) cur = (cur + n) & 1;
        } else {
            for (int k = 0; k < n && e == cudaSuccess; ++k) e = issue_iteration(h, mode, sched, cur, count);
        }
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e, "O(mM) update capture"); }
        if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        it = h->graphs.emplace(key, GraphEntry{ex, count, cur}).first;
    }
    BP_CK(h, cudaGraphLaunch(it->second.exec, h->stream));
    h->launches += it->second.launches;
    h->cur = it->second.end_cur;
    return BP_OK;
}

// ------------------------------------------------------------------- ABI ----

extern "C" {

int bp_version(void) { return (0 << 16) | 3; }

const char *bp_last_error(bp_handle h) { return h ? h->err.c_str() : g_global_err.c_str(); }

long long bp_launch_count(bp_handle h) { return h ? h->launches : -1; }

bp_status bp_create(int W, int H, int M, bp_dtype dtype, void *cuda_stream, bp_handle *out) {
    BPG_TRACE("bp_create");
    g_global_err.clear();
    if (!out) return fail(nullptr, BP_ERR_ARG, "bp_create: out is NULL");
    *out = nullptr;
    if (W < 1 || H < 1) return fail(nullptr, BP_ERR_ARG, "bp_create: W and H must be >= 1");
    if (M < 2 || M > 1024) return fail(nullptr, BP_ERR_ARG, "bp_create: M must be in [2, 1024]");
    if (dtype != BP_F32 && dtype != BP_I32) return fail(nullptr, BP_ERR_ARG, "bp_create: unknown dtype");
    const int Mp = padded_labels(M);
    if ((long long)W * H > (1LL << 30) || (long long)W * H * Mp >= (1LL << 31))
        return fail(nullptr, BP_ERR_ARG, "bp_create: grid too large (W*H*Mp must be < 2^31)");
    bp_ctx *h = new bp_ctx();
    h->W = W; h->H = H; h->M = M; h->Mp = Mp; h->dtype = dtype;
    h->dims = GridDims{W, H, M, Mp, (long long)W * H * Mp};
    Layout lays[8];
    const int nlay = std::min(8, layouts_for(Mp, lays, 8));
    h->layout = nlay > 0 ? lays[0] : Layout{32, 1};
    // two chunks per lane halve the threads per node: on grids that then fill
    // the GPU fewer than four times over (384x288, M = 16: one red-black
    // half-step is 55k nodes) one chunk per lane keeps the SMs occupied
    if (h->layout.C == 2 && (long long)W * H * (Mp / 8) < 4LL * device_sm_count() * 2048)
        for (int i = 0; i < nlay; ++i)
            if (lays[i].C == 1) { h->layout = lays[i]; break; }
    // the log-domain forward (recorded and recomputed alike) takes the
    // default layout whatever the grid size (measured at 256x256, M = 64:
    // 25 us per iteration against 29-31 us with one chunk per lane); the
    // adjoint, which holds more state per label, one chunk per lane (it reads
    // the states and the forward's scales, whatever layout made them)
    h->log_layout = nlay > 0 ? lays[0] : Layout{32, 1};   // two chunks per lane where Mp allows
    h->adj_layout = h->log_layout;
    for (int i = 0; i < nlay; ++i)
        if (lays[i].C == 1) h->adj_layout = lays[i];
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { bp_status st = cuda_fail(nullptr, e, "cudaGetDevice"); delete h; return st; }
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamDefault);
        if (e != cudaSuccess) { bp_status st = cuda_fail(nullptr, e, "cudaStreamCreate"); delete h; return st; }
        h->own_stream = true;
    }
    const size_t ub = (size_t)W * H * Mp * 4;
    bp_status st = BP_OK;
    if (!st) st = ensure_buffer(h, &h->unary, ub, "unary buffer");
    if (!st) st = ensure_buffer(h, &h->msg[0], bpg_state_bytes(h), "message buffer 0");
    if (!st) st = ensure_buffer(h, &h->msg[1], bpg_state_bytes(h), "message buffer 1");
    if (!st) st = ensure_buffer(h, (void **)&h->d_status, sizeof(int), "status word");
    if (!st) {
        e = cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMemsetAsync");
    }
    if (st) {
        g_global_err = h->err;
        bp_destroy(h);
        return st;
    }
    *out = h;
    return BP_OK;
}

void bp_destroy(bp_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    clear_graphs(h);
    bpg_free_extras(h);
    void *bufs[] = {h->unary, h->log_unary, h->msg[0], h->msg[1], h->d_wf, h->d_wi, h->d_dense, h->d_status,
                    h->tune_buf, h->d_sp_len, h->d_sp_ell, h->d_sp_rent, h->d_sp_rlab, h->d_stereo};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

bp_status bp_set_unary(bp_handle h, const void *dev_unary) {
    BPG_TRACE("bp_set_unary");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_unary: NULL handle");
    h->err.clear();
    if (!dev_unary) return fail(h, BP_ERR_ARG, "bp_set_unary: NULL unary");
    if (bp_status st = bpg_check_device(h)) return st;
    const long long nodes = (long long)h->W * h->H;
    if (h->dtype == BP_F32)
        BP_CK(h, launch_pad_copy_f32((const float *)dev_unary, (float *)h->unary, nodes, h->M, h->Mp, 0, h->stream));
    else
        BP_CK(h, launch_pad_copy_i32((const int32_t *)dev_unary, (int32_t *)h->unary, nodes, h->M, h->Mp, h->stream));
    h->launches += 1;
    h->have_unary = true;
    h->log_unary_valid = false;
    h->recorded = false;
    return BP_OK;
}

bp_status bp_set_unary_stereo(bp_handle h, const uint8_t *left, const uint8_t *right,
                              const void *host_table, int Tu) {
    BPG_TRACE("bp_set_unary_stereo");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_unary_stereo: NULL handle");
    h->err.clear();
    if (!left || !right || !host_table) return fail(h, BP_ERR_ARG, "bp_set_unary_stereo: NULL argument");
    if (Tu < 0 || Tu > kMaxStereoCost) return fail(h, BP_ERR_ARG, "bp_set_unary_stereo: Tu must be in [0, 255]");
    if (h->dtype == BP_F32) {
        const float *t = (const float *)host_table;
        for (int k = 0; k <= Tu; ++k)
            if (!std::isfinite(t[k]) || t[k] < 0.f)
                return fail(h, BP_ERR_ARG, "bp_set_unary_stereo: table values must be finite and >= 0");
    } else {
        const int32_t *t = (const int32_t *)host_table;
        for (int k = 0; k <= Tu; ++k)
            if (t[k] < 0 || t[k] >= (1 << 26))
                return fail(h, BP_ERR_ARG, "bp_set_unary_stereo: energies must be in [0, 2^26)");
    }
    if (bp_status st = bpg_check_device(h)) return st;
    // images in host memory (pinned or pageable) are copied into the handle's
    // staging buffer on its stream first; device or managed memory is read
    // in place
    const uint8_t *img[2] = {left, right};
    const size_t img_bytes = (size_t)h->W * h->H;
    for (int k = 0; k < 2; ++k) {
        cudaPointerAttributes at{};
        BP_CK(h, cudaPointerGetAttributes(&at, img[k]));
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) continue;
        if (bp_status st = ensure_buffer(h, (void **)&h->d_stereo, 2 * img_bytes, "stereo image staging")) return st;
        BP_CK(h, cudaMemcpyAsync(h->d_stereo + k * img_bytes, img[k], img_bytes, cudaMemcpyHostToDevice, h->stream));
        img[k] = h->d_stereo + k * img_bytes;
    }
    if (h->dtype == BP_F32)
        BP_CK(h, launch_unary_stereo_f32(img[0], img[1], (float *)h->unary, h->W, h->H, h->M, h->Mp, Tu,
                                         (const float *)host_table, h->stream));
    else
        BP_CK(h, launch_unary_stereo_i32(img[0], img[1], (int32_t *)h->unary, h->W, h->H, h->M, h->Mp, Tu,
                                         (const int32_t *)host_table, h->stream));
    h->launches += 1;
    h->have_unary = true;
    h->log_unary_valid = false;
    h->recorded = false;
    return BP_OK;
}

bp_status bp_set_unary_log(bp_handle h, const float *dev_logg) {
    BPG_TRACE("bp_set_unary_log");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_unary_log: NULL handle");
    h->err.clear();
    if (!dev_logg) return fail(h, BP_ERR_ARG, "bp_set_unary_log: NULL unary");
    if (h->dtype != BP_F32) return fail(h, BP_ERR_ARG, "bp_set_unary_log: needs a BP_F32 handle");
    if (bp_status st = bpg_check_device(h)) return st;
    const long long nodes = (long long)h->W * h->H;
    if (bp_status st = ensure_buffer(h, (void **)&h->log_unary, (size_t)nodes * h->Mp * 4, "log unary")) return st;
    // base-2 log g for the log-domain kernels and g for the linear ones
    BP_CK(h, launch_log_unary(dev_logg, h->log_unary, (float *)h->unary, nodes, h->M, h->Mp, h->stream));
    h->launches += 1;
    h->have_unary = true;
    h->log_unary_valid = true;
    h->recorded = false;
    return BP_OK;
}

bp_status bp_set_potential(bp_handle h, const void *host_table, int T, double fbar) {
    BPG_TRACE("bp_set_potential");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_potential: NULL handle");
    h->err.clear();
    if (!host_table) return fail(h, BP_ERR_ARG, "bp_set_potential: NULL table");
    if (T < 0 || T > (1 << 20)) return fail(h, BP_ERR_ARG, "bp_set_potential: T out of range");
    if (!std::isfinite(fbar) || fbar < 0) return fail(h, BP_ERR_ARG, "bp_set_potential: fbar must be finite and >= 0");
    const int m = 2 * T + 1;
    const int Teff = std::min(T, h->M - 1);
    if (h->dtype == BP_F32) {
        const float *tab = (const float *)host_table;
        for (int i = 0; i < m; ++i)
            if (!std::isfinite(tab[i]) || tab[i] < 0)
                return fail(h, BP_ERR_ARG, "bp_set_potential: table entries must be finite and >= 0");
        h->tablef.assign(tab, tab + m);
        h->fbarf = (float)fbar;
        h->wf.resize(2 * Teff + 1);
        for (int d = -Teff; d <= Teff; ++d) h->wf[d + Teff] = (float)((double)tab[d + T] - (double)h->fbarf);
    } else {
        const int32_t *tab = (const int32_t *)host_table;
        if (fbar != std::floor(fbar) || fbar >= (double)(1 << 26))
            return fail(h, BP_ERR_ARG, "bp_set_potential: Ebar must be an integer in [0, 2^26)");
        const int32_t ebar = (int32_t)fbar;
        for (int i = 0; i < m; ++i) {
            if (tab[i] < 0 || tab[i] >= (1 << 26))
                return fail(h, BP_ERR_ARG, "bp_set_potential: energies must lie in [0, 2^26)");
            if (tab[i] > ebar)
                return fail(h, BP_ERR_POTENTIAL,
                            "bp_set_potential: E(d) > Ebar; Eq. 11 is exact only when f >= fbar (Sec. 5)");
        }
        h->tablei.assign(tab, tab + m);
        h->ebar = ebar;
        h->wi.resize(2 * Teff + 1);
        for (int d = -Teff; d <= Teff; ++d) h->wi[d + Teff] = tab[d + T];
    }
    h->sparse = false;
    h->T = T;
    h->Teff = Teff;
    h->fbar = fbar;
    h->fast = Teff <= kTMaxFast && band_fast_available(h->Mp, h->layout, Teff);
    if (!h->fast) {
        const size_t wb = (size_t)(2 * Teff + 1) * 4;
        if (h->d_wf) { cudaFree(h->d_wf); h->d_wf = nullptr; }
        if (h->d_wi) { cudaFree(h->d_wi); h->d_wi = nullptr; }
        if (h->dtype == BP_F32) {
            if (bp_status st = ensure_buffer(h, (void **)&h->d_wf, wb, "band table")) return st;
            BP_CK(h, cudaMemcpyAsync(h->d_wf, h->wf.data(), wb, cudaMemcpyHostToDevice, h->stream));
        } else {
            if (bp_status st = ensure_buffer(h, (void **)&h->d_wi, wb, "band table")) return st;
            BP_CK(h, cudaMemcpyAsync(h->d_wi, h->wi.data(), wb, cudaMemcpyHostToDevice, h->stream));
        }
        // the copy reads pageable host memory owned by the handle's vectors,
        // which stay alive; make it complete before they can change
        BP_CK(h, cudaStreamSynchronize(h->stream));
    }
    if (h->d_dense) { cudaFree(h->d_dense); h->d_dense = nullptr; }
    h->tc_ready = false;
    h->p_ready = false;
    h->have_potential = true;
    h->recorded = false;
    clear_graphs(h);
    return BP_OK;
}

// Order of each receiver label's pattern entries for the sparse kernels: the
// eight lanes of a quarter-warp (receiver labels 8q .. 8q + 7) gather, at
// step i, their i-th entries with 16-byte loads, which conflict when two
// lanes hit the same 16-byte bank group (slot mod 8) at different slots.  At
// every step a maximum matching of lanes to bank groups (augmenting paths)
// picks conflict-free entries for as many lanes as possible; the others take
// their next entry.  Returns, for each CSR position, the CSR index to use.
static std::vector<int> sparse_bank_order(int M, const int32_t *rowptr, const int32_t *cols) {
    std::vector<int> order(rowptr[M]);
    for (int b = 0; b < M; b += 8) {
        const int nl = std::min(8, M - b);
        std::vector<std::vector<int>> rem(nl);
        for (int l = 0; l < nl; ++l)
            for (int p = rowptr[b + l]; p < rowptr[b + l + 1]; ++p) rem[l].push_back(p);
        std::vector<int> filled(nl, 0);
        auto group = [&](int p) { return sp_label_slot(cols[p]) & 7; };
        for (;;) {
            bool any = false;
            for (int l = 0; l < nl; ++l) any = any || !rem[l].empty();
            if (!any) break;
            int owner[8];
            std::fill(owner, owner + 8, -1);
            std::vector<int> pick(nl, -1);   // index into rem[l]
            std::function<bool(int, unsigned &)> augment = [&](int l, unsigned &seen) -> bool {
                for (int j = 0; j < (int)rem[l].size(); ++j) {
                    const int g = group(rem[l][j]);
                    if (seen & (1u << g)) continue;
                    seen |= 1u << g;
                    if (owner[g] < 0 || augment(owner[g], seen)) {
                        owner[g] = l;
                        pick[l] = j;
                        return true;
                    }
                }
                return false;
            };
            std::vector<int> lanes;
            for (int l = 0; l < nl; ++l)
                if (!rem[l].empty()) lanes.push_back(l);
            std::stable_sort(lanes.begin(), lanes.end(), [&](int x, int y) { return rem[x].size() > rem[y].size(); });
            for (int l : lanes) {
                unsigned seen = 0;
                augment(l, seen);
            }
            for (int l : lanes) {
                // a lane whose group was taken over during augmentation keeps
                // its entry in that group only if it still owns it
                int j = pick[l];
                if (j < 0 || owner[group(rem[l][j])] != l) j = 0;
                order[rowptr[b + l] + filled[l]++] = rem[l][j];
                rem[l].erase(rem[l].begin() + j);
            }
        }
    }
    return order;
}

bp_status bp_set_potential_sparse(bp_handle h, const int32_t *host_rowptr, const int32_t *host_cols,
                                  const void *host_vals, double fbar) {
    BPG_TRACE("bp_set_potential_sparse");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_potential_sparse: NULL handle");
    h->err.clear();
    if (!host_rowptr || !host_vals || (!host_cols && host_rowptr[h->M] != 0))
        return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: NULL argument");
    if (!std::isfinite(fbar) || fbar < 0) return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: fbar must be >= 0");
    if (host_rowptr[0] != 0) return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: rowptr[0] must be 0");
    for (int x = 0; x < h->M; ++x)
        if (host_rowptr[x + 1] < host_rowptr[x]) return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: rowptr decreases");
    const int nnz = host_rowptr[h->M];
    if (h->Mp > 512) return fail(h, BP_ERR_UNSUPPORTED, "bp_set_potential_sparse: serves M <= 512");
    std::vector<char> seen(h->M, 0);
    for (int xj = 0; xj < h->M; ++xj) {
        for (int p = host_rowptr[xj]; p < host_rowptr[xj + 1]; ++p) {
            const int xi = host_cols[p];
            if (xi < 0 || xi >= h->M) return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: column out of range");
            if (seen[xi]) return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: repeated column in a row");
            seen[xi] = 1;
        }
        for (int p = host_rowptr[xj]; p < host_rowptr[xj + 1]; ++p) seen[host_cols[p]] = 0;
    }
    std::vector<int32_t> wbits(nnz);   // per entry: f - fbar (float bits) or E
    if (h->dtype == BP_F32) {
        const float *v = (const float *)host_vals;
        for (int p = 0; p < nnz; ++p)
            if (!std::isfinite(v[p]) || v[p] < 0)
                return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: values must be finite and >= 0");
        h->sp_valf.assign(v, v + nnz);
        h->fbarf = (float)fbar;
        for (int p = 0; p < nnz; ++p) {
            const float w = (float)((double)v[p] - (double)h->fbarf);
            std::memcpy(&wbits[p], &w, 4);
        }
    } else {
        if (fbar != std::floor(fbar) || fbar >= (double)(1 << 26))
            return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: Ebar must be an integer in [0, 2^26)");
        const int32_t *v = (const int32_t *)host_vals;
        for (int p = 0; p < nnz; ++p) {
            if (v[p] < 0 || v[p] >= (1 << 26)) return fail(h, BP_ERR_ARG, "bp_set_potential_sparse: energies out of range");
            if (v[p] > (int32_t)fbar)
                return fail(h, BP_ERR_POTENTIAL,
                            "bp_set_potential_sparse: E > Ebar; Eq. 11 is exact only when f >= fbar (Sec. 5)");
        }
        h->sp_vali.assign(v, v + nnz);
        h->ebar = (int32_t)fbar;
        std::memcpy(wbits.data(), v, (size_t)nnz * 4);
    }
    h->sp_rowptr.assign(host_rowptr, host_rowptr + h->M + 1);
    h->sp_cols.assign(host_cols, host_cols + nnz);
    // interleave by receiver label (entry i of x_j at i * M + x_j), sender
    // labels replaced by their shared-memory slots, entries ordered per
    // quarter-warp against bank conflicts
    int rmax = 1;
    std::vector<int32_t> len(h->M);
    for (int xj = 0; xj < h->M; ++xj) {
        len[xj] = host_rowptr[xj + 1] - host_rowptr[xj];
        rmax = std::max(rmax, len[xj]);
    }
    const std::vector<int> order = sparse_bank_order(h->M, host_rowptr, host_cols);
    std::vector<int32_t> ell((size_t)rmax * h->M * 2, 0);
    for (int xj = 0; xj < h->M; ++xj)
        for (int i = 0; i < len[xj]; ++i) {
            const int p = order[host_rowptr[xj] + i];
            ell[((size_t)i * h->M + xj) * 2] = sp_label_slot(host_cols[p]);
            ell[((size_t)i * h->M + xj) * 2 + 1] = wbits[p];
        }
    // the register-pattern schedule, when the pattern fits one (else the list
    // kernels serve); min-sum with Ebar <= kP16MaxEbar runs on 16-bit label pairs
    const bool p16 = h->dtype == BP_I32 && (int32_t)fbar <= kP16MaxEbar;
    SparseRegPlan plan;
    const bool reg_ok = sparse_reg_plan(h->M, h->Mp, host_rowptr, host_cols, wbits.data(), p16 ? 8 : 16, &plan);
    BP_CK(h, cudaStreamSynchronize(h->stream));   // earlier work may still read the old pattern
    void *bufs[] = {h->d_sp_len, h->d_sp_ell, h->d_sp_rent, h->d_sp_rlab};
    for (void *p : bufs)
        if (p) cudaFree(p);
    h->d_sp_len = h->d_sp_ell = h->d_sp_rent = h->d_sp_rlab = nullptr;
    h->sp_reg = false;
    h->sp_p16 = false;
    if (bp_status st = ensure_buffer(h, &h->d_sp_len, (size_t)h->M * 4, "sparse row lengths")) return st;
    if (bp_status st = ensure_buffer(h, &h->d_sp_ell, ell.size() * 4, "sparse pattern")) return st;
    BP_CK(h, cudaMemcpyAsync(h->d_sp_len, len.data(), (size_t)h->M * 4, cudaMemcpyHostToDevice, h->stream));
    BP_CK(h, cudaMemcpyAsync(h->d_sp_ell, ell.data(), ell.size() * 4, cudaMemcpyHostToDevice, h->stream));
    if (reg_ok) {
        const SparseRegMode rmode = h->dtype != BP_I32 ? SparseRegMode::Sum
                                    : p16                ? SparseRegMode::Min16
                                                         : SparseRegMode::Min;
        const std::vector<int32_t> dent = sparse_reg_device_entries(plan, rmode, h->ebar);
        if (bp_status st = ensure_buffer(h, &h->d_sp_rent, dent.size() * 4, "register pattern")) return st;
        if (bp_status st = ensure_buffer(h, &h->d_sp_rlab, plan.lab.size() * 4, "register pattern labels"))
            return st;
        BP_CK(h, cudaMemcpyAsync(h->d_sp_rent, dent.data(), dent.size() * 4, cudaMemcpyHostToDevice, h->stream));
        BP_CK(h, cudaMemcpyAsync(h->d_sp_rlab, plan.lab.data(), plan.lab.size() * 4, cudaMemcpyHostToDevice,
                                 h->stream));
        h->sp_reg = true;
        h->sp_p16 = p16;
        h->sp_KM = plan.KM;
        h->sp_LM = plan.LM;
        h->sp_steps = plan.steps;
        h->sp_wavefronts = plan.wavefronts;
    }
    BP_CK(h, cudaStreamSynchronize(h->stream));
    if (h->d_dense) { cudaFree(h->d_dense); h->d_dense = nullptr; }
    h->sparse = true;
    h->fast = false;
    h->fbar = fbar;
    h->T = 0;
    h->Teff = 0;
    h->tc_ready = false;
    h->p_ready = false;
    h->have_potential = true;
    h->recorded = false;
    clear_graphs(h);
    return BP_OK;
}

bp_status bp_reset_messages(bp_handle h) {
    BPG_TRACE("bp_reset_messages");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_reset_messages: NULL handle");
    h->err.clear();
    h->msg_uniform = true;
    h->recorded = false;
    return BP_OK;
}

bp_status bp_set_layout(bp_handle h, int L, int C) {
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_layout: NULL handle");
    h->err.clear();
    Layout lays[8];
    const int n = std::min(8, layouts_for(h->Mp, lays, 8));
    for (int i = 0; i < n; ++i)
        if (lays[i].L == L && lays[i].C == C) {
            h->layout = lays[i];
            h->log_layout = lays[i];
            if (h->have_potential) h->fast = h->Teff <= kTMaxFast && band_fast_available(h->Mp, h->layout, h->Teff);
            return BP_OK;
        }
    return fail(h, BP_ERR_ARG, "bp_set_layout: layout not compiled for this label count");
}

bp_status bp_get_layout(bp_handle h, int *L, int *C) {
    if (!h || !L || !C) return fail(h, BP_ERR_ARG, "bp_get_layout: NULL argument");
    *L = h->layout.L;
    *C = h->layout.C;
    return BP_OK;
}

bp_status bp_iterate(bp_handle h, int n_iters, int mode, bp_schedule schedule) {
    BPG_TRACE("bp_iterate");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_iterate: NULL handle");
    h->err.clear();
    if (n_iters < 0) return fail(h, BP_ERR_ARG, "bp_iterate: n_iters < 0");
    if (schedule != BP_SYNC && schedule != BP_REDBLACK) return fail(h, BP_ERR_ARG, "bp_iterate: unknown schedule");
    const int base = mode & 1;
    const bool is_log = (mode & BP_LOG) != 0, rec = (mode & BP_RECORD) != 0;
    if (mode & ~(BP_MAX | BP_LOG | BP_RECORD)) return fail(h, BP_ERR_ARG, "bp_iterate: unknown mode bits");
    if (base == BP_MAX && h->dtype != BP_I32) return fail(h, BP_ERR_ARG, "bp_iterate: BP_MAX needs a BP_I32 handle");
    if (base == BP_SUM && h->dtype != BP_F32) return fail(h, BP_ERR_ARG, "bp_iterate: BP_SUM needs a BP_F32 handle");
    if ((is_log || rec) && base != BP_SUM) return fail(h, BP_ERR_ARG, "bp_iterate: BP_LOG/BP_RECORD are sum-product flags");
    if (rec && !is_log) return fail(h, BP_ERR_ARG, "bp_iterate: BP_RECORD needs BP_LOG");
    if (rec && schedule != BP_SYNC) return fail(h, BP_ERR_ARG, "bp_iterate: BP_RECORD needs BP_SYNC");
    if (!h->have_unary || !h->have_potential)
        return fail(h, BP_ERR_STATE, "bp_iterate: set the unary and the potential first");
    if (is_log && (!h->fast || h->sparse))
        return fail(h, BP_ERR_UNSUPPORTED, "bp_iterate: log mode needs a band potential with T <= 8 and M <= 512");
    if (bp_status st = bpg_check_device(h)) return st;
    if (is_log) {
        if (bp_status st = ensure_log_unary(h)) return st;
    }
    if (bp_status st = materialize(h, is_log)) return st;
    if (rec) return bpg_record_forward(h, n_iters);
    h->recorded = false;
    if (n_iters == 0) return BP_OK;
    return run_iterations(h, n_iters, mode & (BP_MAX | BP_LOG), schedule);
}

bp_status bp_iterate_dense(bp_handle h, int n_iters, bp_dense_kind kind) {
    BPG_TRACE("bp_iterate_dense");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_iterate_dense: NULL handle");
    h->err.clear();
    if (n_iters < 0) return fail(h, BP_ERR_ARG, "bp_iterate_dense: n_iters < 0");
    if (!h->have_unary || !h->have_potential)
        return fail(h, BP_ERR_STATE, "bp_iterate_dense: set the unary and the potential first");
    if (bp_status st = bpg_check_device(h)) return st;
    if (bp_status st = materialize(h, false)) return st;
    h->recorded = false;
    if (kind == BP_DENSE_BF16_TC || kind == BP_DENSE_BF16_TC_FUSED) {
        if (h->dtype != BP_F32) return fail(h, BP_ERR_ARG, "bp_iterate_dense: the tensor-core baseline is sum-product");
        return bpg_dense_tc_iterate_kind(h, n_iters, kind == BP_DENSE_BF16_TC_FUSED);
    }
    if (kind != BP_DENSE_CUDA_CORE) return fail(h, BP_ERR_ARG, "bp_iterate_dense: unknown kind");
    // the full M x M table, F[x_i][x_j] (f, or E for min-sum)
    if (!h->d_dense) {
        const size_t bytes = (size_t)h->M * h->M * 4;
        std::vector<float> F;
        std::vector<int32_t> V;
        if (h->dtype == BP_F32) F.resize((size_t)h->M * h->M); else V.resize((size_t)h->M * h->M);
        for (int xi = 0; xi < h->M; ++xi)
            for (int xj = 0; xj < h->M; ++xj) {
                if (h->dtype == BP_F32) F[(size_t)xi * h->M + xj] = bpg_pair_value_f(h, xi, xj);
                else V[(size_t)xi * h->M + xj] = bpg_pair_value_i(h, xi, xj);
            }
        if (bp_status st = ensure_buffer(h, &h->d_dense, bytes, "dense table")) return st;
        BP_CK(h, cudaMemcpyAsync(h->d_dense, h->dtype == BP_F32 ? (const void *)F.data() : (const void *)V.data(),
                                 bytes, cudaMemcpyHostToDevice, h->stream));
        BP_CK(h, cudaStreamSynchronize(h->stream));
    }
    for (int it = 0; it < n_iters; ++it) {
        if (h->dtype == BP_F32) {
            DenseArgsF a{(const float *)h->unary, (const float *)h->msg[h->cur], (float *)h->msg[h->cur ^ 1], h->dims,
                         (const float *)h->d_dense};
            BP_CK(h, launch_dense_sum(a, h->stream));
        } else {
            DenseArgsI a{(const int32_t *)h->unary, (const int32_t *)h->msg[h->cur], (int32_t *)h->msg[h->cur ^ 1],
                         h->dims, (const int32_t *)h->d_dense};
            BP_CK(h, launch_dense_min(a, h->stream));
        }
        h->launches += 1;
        h->cur ^= 1;
    }
    return BP_OK;
}

bp_status bp_beliefs(bp_handle h, void *dev_out, int32_t *dev_map) {
    BPG_TRACE("bp_beliefs");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_beliefs: NULL handle");
    h->err.clear();
    if (!dev_out) return fail(h, BP_ERR_ARG, "bp_beliefs: NULL output");
    if (!h->have_unary) return fail(h, BP_ERR_STATE, "bp_beliefs: set the unary first");
    if (bp_status st = bpg_check_device(h)) return st;
    if (h->msg_uniform)
        if (bp_status st = materialize(h, false)) return st;
    if (h->dtype == BP_F32) {
        const bool lg = h->msg_log;
        if (lg)
            if (bp_status st = ensure_log_unary(h)) return st;
        BP_CK(h, launch_beliefs_f32(lg ? h->log_unary : (const float *)h->unary, (const float *)h->msg[h->cur], h->dims,
                                    lg ? 1 : 0, (float *)dev_out, dev_map, h->stream));
    } else {
        BP_CK(h, launch_beliefs_i32((const int32_t *)h->unary, (const int32_t *)h->msg[h->cur], h->dims,
                                    (int32_t *)dev_out, dev_map, h->stream));
    }
    h->launches += 1;
    return BP_OK;
}

bp_status bp_get_messages(bp_handle h, void *dev_planes) {
    BPG_TRACE("bp_get_messages");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_get_messages: NULL handle");
    h->err.clear();
    if (!dev_planes) return fail(h, BP_ERR_ARG, "bp_get_messages: NULL output");
    if (bp_status st = bpg_check_device(h)) return st;
    if (h->msg_uniform)
        if (bp_status st = materialize(h, false)) return st;
    BP_CK(h, launch_unpad_messages(h->msg[h->cur], dev_planes, h->W, h->H, h->M, h->Mp,
                                   h->dtype == BP_F32 && h->msg_log ? 1 : 0, h->stream));
    h->launches += 1;
    return BP_OK;
}

bp_status bp_set_messages(bp_handle h, const void *dev_planes) {
    BPG_TRACE("bp_set_messages");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_messages: NULL handle");
    h->err.clear();
    if (!dev_planes) return fail(h, BP_ERR_ARG, "bp_set_messages: NULL input");
    if (bp_status st = bpg_check_device(h)) return st;
    const long long rows = 4LL * h->W * h->H;
    if (h->dtype == BP_F32)
        BP_CK(h, launch_pad_copy_f32((const float *)dev_planes, (float *)h->msg[h->cur], rows, h->M, h->Mp, 0, h->stream));
    else
        BP_CK(h, launch_pad_copy_i32((const int32_t *)dev_planes, (int32_t *)h->msg[h->cur], rows, h->M, h->Mp,
                                     h->stream));
    h->launches += 1;
    h->msg_uniform = false;
    h->msg_log = false;
    h->recorded = false;
    return BP_OK;
}

bp_status bp_sync(bp_handle h) {
    BPG_TRACE("bp_sync");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_sync: NULL handle");
    BP_CK(h, cudaStreamSynchronize(h->stream));
    int flag = 0;
    BP_CK(h, cudaMemcpy(&flag, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        BP_CK(h, cudaMemset(h->d_status, 0, sizeof(int)));
        return fail(h, BP_ERR_TIMEOUT, "a bounded device-side wait gave up (status " + std::to_string(flag) + ")");
    }
    return BP_OK;
}

bp_status bp_autotune(bp_handle h, int mode, int n_iters, float *host_best_ms) {
    BPG_TRACE("bp_autotune");
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_autotune: NULL handle");
    h->err.clear();
    if (n_iters < 1) return fail(h, BP_ERR_ARG, "bp_autotune: n_iters < 1");
    if (!h->have_unary || !h->have_potential) return fail(h, BP_ERR_STATE, "bp_autotune: set unary and potential first");
    if (h->sparse) return fail(h, BP_ERR_UNSUPPORTED, "bp_autotune: tunes the band kernels only");
    const bool is_log = (mode & BP_LOG) != 0;
    if (bp_status st = bpg_check_device(h)) return st;
    if (is_log)
        if (bp_status st = ensure_log_unary(h)) return st;
    if (bp_status st = materialize(h, is_log)) return st;
    if (bp_status st = ensure_buffer(h, &h->tune_buf, bpg_state_bytes(h), "autotune buffer")) return st;
    Layout lays[8];
    const int n = std::min(8, layouts_for(h->Mp, lays, 8));
    Layout &target = is_log ? h->log_layout : h->layout;
    const Layout saved = target;
    const int saved_cur = h->cur;
    BP_CK(h, cudaMemcpyAsync(h->tune_buf, h->msg[h->cur], bpg_state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    cudaEvent_t e0, e1;
    BP_CK(h, cudaEventCreate(&e0));
    BP_CK(h, cudaEventCreate(&e1));
    float best = 3e38f;
    Layout best_lay = saved;
    const int md = mode & (BP_MAX | BP_LOG);
    for (int i = 0; i < n; ++i) {
        if (h->Teff > kTMaxFast || !band_fast_available(h->Mp, lays[i], h->Teff)) continue;
        target = lays[i];
        h->fast = true;
        bp_status st = run_iterations(h, n_iters, md, BP_SYNC);        // warm
        if (!st) st = (cudaEventRecord(e0, h->stream) == cudaSuccess) ? BP_OK : BP_ERR_CUDA;
        if (!st) st = run_iterations(h, n_iters, md, BP_SYNC);
        if (!st) st = (cudaEventRecord(e1, h->stream) == cudaSuccess) ? BP_OK : BP_ERR_CUDA;
        if (!st) st = (cudaEventSynchronize(e1) == cudaSuccess) ? BP_OK : BP_ERR_CUDA;
        float ms = 0.f;
        if (!st) cudaEventElapsedTime(&ms, e0, e1);
        if (st) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            target = saved;
            h->fast = h->Teff <= kTMaxFast && band_fast_available(h->Mp, h->layout, h->Teff);
            return st == BP_ERR_CUDA ? fail(h, st, "bp_autotune: timing failed") : st;
        }
        if (ms < best) { best = ms; best_lay = lays[i]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    target = best_lay;
    h->fast = h->Teff <= kTMaxFast && band_fast_available(h->Mp, h->layout, h->Teff);
    h->cur = saved_cur;
    BP_CK(h, cudaMemcpyAsync(h->msg[h->cur], h->tune_buf, bpg_state_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    if (host_best_ms) *host_best_ms = best / (float)n_iters;
    return BP_OK;
}

bp_status bp_set_grid(bp_handle h, int blocks) {
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_grid: NULL handle");
    h->err.clear();
    if (blocks < 0 || blocks > (1 << 20)) return fail(h, BP_ERR_ARG, "bp_set_grid: blocks out of range");
    h->blocks_override = blocks;
    return BP_OK;
}

bp_status bp_sparse_schedule(int M, const int32_t *host_rowptr, const int32_t *host_cols, int gather_bytes,
                             int *KM, int *LM, int *steps, int *wavefronts, int32_t *host_lab, int32_t *host_ent) {
    BPG_TRACE("bp_sparse_schedule");
    g_global_err.clear();
    if (M < 2 || M > 1024) return fail(nullptr, BP_ERR_ARG, "bp_sparse_schedule: M out of range");
    if (!host_rowptr || !KM || !LM || !steps || !wavefronts || (!host_cols && host_rowptr[M] != 0))
        return fail(nullptr, BP_ERR_ARG, "bp_sparse_schedule: NULL argument");
    if (gather_bytes != 16 && gather_bytes != 8)
        return fail(nullptr, BP_ERR_ARG, "bp_sparse_schedule: gather_bytes must be 16 or 8");
    if (host_rowptr[0] != 0) return fail(nullptr, BP_ERR_ARG, "bp_sparse_schedule: rowptr[0] must be 0");
    for (int x = 0; x < M; ++x)
        if (host_rowptr[x + 1] < host_rowptr[x]) return fail(nullptr, BP_ERR_ARG, "bp_sparse_schedule: rowptr decreases");
    for (int p = 0; p < host_rowptr[M]; ++p)
        if (host_cols[p] < 0 || host_cols[p] >= M)
            return fail(nullptr, BP_ERR_ARG, "bp_sparse_schedule: column out of range");
    std::vector<int32_t> index(host_rowptr[M]);
    for (int p = 0; p < host_rowptr[M]; ++p) index[p] = p;
    SparseRegPlan plan;
    *KM = *LM = *steps = *wavefronts = 0;
    if (!sparse_reg_plan(M, padded_labels(M), host_rowptr, host_cols, index.data(), gather_bytes, &plan))
        return BP_OK;
    *KM = plan.KM;
    *LM = plan.LM;
    *steps = plan.steps;
    *wavefronts = plan.wavefronts;
    if (host_lab) std::memcpy(host_lab, plan.lab.data(), plan.lab.size() * 4);
    if (host_ent) std::memcpy(host_ent, plan.ent.data(), plan.ent.size() * 4);
    return BP_OK;
}

bp_status bp_set_sparse_kernel(bp_handle h, int kind) {
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_sparse_kernel: NULL handle");
    h->err.clear();
    if (kind != BP_SPARSE_AUTO && kind != BP_SPARSE_LISTS && kind != BP_SPARSE_REGISTERS)
        return fail(h, BP_ERR_ARG, "bp_set_sparse_kernel: unknown kind");
    if (kind == BP_SPARSE_REGISTERS && h->sparse && !h->sp_reg)
        return fail(h, BP_ERR_UNSUPPORTED, "bp_set_sparse_kernel: this pattern has no register schedule");
    h->sp_kernel = kind;
    clear_graphs(h);
    return BP_OK;
}

bp_status bp_get_sparse_kernel(bp_handle h, int *kind, int *steps, int *wavefronts) {
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_get_sparse_kernel: NULL handle");
    h->err.clear();
    if (!kind || !steps || !wavefronts) return fail(h, BP_ERR_ARG, "bp_get_sparse_kernel: NULL argument");
    if (!h->sparse) return fail(h, BP_ERR_STATE, "bp_get_sparse_kernel: no sparse potential set");
    const bool reg = h->sp_reg && h->sp_kernel != BP_SPARSE_LISTS;
    *kind = reg ? BP_SPARSE_REGISTERS : BP_SPARSE_LISTS;
    *steps = reg ? h->sp_steps : 0;
    *wavefronts = reg ? h->sp_wavefronts : 0;
    return BP_OK;
}

bp_status bp_set_persistent(bp_handle h, int mode) {
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_persistent: NULL handle");
    h->err.clear();
    if (mode < -1 || mode > 1) return fail(h, BP_ERR_ARG, "bp_set_persistent: mode must be -1, 0 or 1");
    h->persistent = mode;
    return BP_OK;
}

bp_status bp_set_checkpoint_interval(bp_handle h, int every) {
    if (!h) return fail(nullptr, BP_ERR_ARG, "bp_set_checkpoint_interval: NULL handle");
    if (every < 1) return fail(h, BP_ERR_ARG, "bp_set_checkpoint_interval: interval must be >= 1");
    h->ckpt_every = every;
    h->recorded = false;
    return BP_OK;
}

}  // extern "C"

// True when the min-sum band of this table runs exactly on 16-bit label pairs
// (MinBand::band_packed): Ebar - min_d E(d) <= 16000.
bool bpg_packed16(const std::vector<int32_t> &w, int32_t ebar) {
    if (w.empty()) return false;
    int64_t emin = ebar;
    for (int32_t v : w) emin = std::min<int64_t>(emin, v);
    return (int64_t)ebar - emin <= 16000;
}

// True when the centre entry E(0) of a band table (2T+1 entries) is its minimum.
bool bpg_zero_min(const std::vector<int32_t> &w) {
    if (w.empty()) return false;
    const int c = (int)w.size() / 2;
    for (int32_t v : w)
        if (v < w[c]) return false;
    return true;
}

// Value of the pairwise potential at (x_i, x_j) as the handle holds it: the
// band table or the sparse list, fbar (Ebar) elsewhere.
float bpg_pair_value_f(const bp_ctx *h, int xi, int xj) {
    if (h->sparse) {
        for (int p = h->sp_rowptr[xj]; p < h->sp_rowptr[xj + 1]; ++p)
            if (h->sp_cols[p] == xi) return h->sp_valf[p];
        return h->fbarf;
    }
    const int d = xi - xj;
    return (d >= -h->T && d <= h->T) ? h->tablef[d + h->T] : h->fbarf;
}

int32_t bpg_pair_value_i(const bp_ctx *h, int xi, int xj) {
    if (h->sparse) {
        for (int p = h->sp_rowptr[xj]; p < h->sp_rowptr[xj + 1]; ++p)
            if (h->sp_cols[p] == xi) return h->sp_vali[p];
        return h->ebar;
    }
    const int d = xi - xj;
    return (d >= -h->T && d <= h->T) ? h->tablei[d + h->T] : h->ebar;
}

// Shared with bp_backward.cu / dense_tc.cu.
bp_status bpg_fail(bp_ctx *h, bp_status st, const std::string &msg) { return fail(h, st, msg); }
bp_status bpg_cuda_fail(bp_ctx *h, cudaError_t e, const char *where) { return cuda_fail(h, e, where); }
bp_status bpg_ensure_buffer(bp_ctx *h, void **p, size_t bytes, const char *what) {
    return ensure_buffer(h, p, bytes, what);
}
cudaError_t bpg_issue_iteration(bp_ctx *h, int mode, int sched, int &cur, int &count) {
    return issue_iteration(h, mode, sched, cur, count);
}
