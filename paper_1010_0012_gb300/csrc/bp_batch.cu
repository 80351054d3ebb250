// Batched O(mM) belief propagation: many independent MRFs of uneven size,
// label count and band width advanced by one persistent cooperative launch
// per bp_batch_iterate call (captured once in a CUDA graph and replayed).
// Declarations and the contract of every call are in include/bp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "trace.h"
#include "../../include/bp.h"
#include "bp_batch_internal.h"
#include "bp_ctx.h"

using namespace bpg;

namespace bpg {
cudaError_t launch_batch_sum(const BatchArgs &a, int family, int blocks, cudaStream_t s);
cudaError_t launch_batch_min(const BatchArgs &a, int family, int blocks, cudaStream_t s);
int batch_max_blocks_sum(int family, bool redblack = false, bool full = false);
int batch_max_blocks_min(int family, bool redblack = false, bool full = false);

int batch_lanes_per_node(int family, int Mp) {
    if (family == 1) return Mp >= 256 ? 32 : Mp / 4;
    return Mp >= 256 ? 32 : Mp / 8;
}
}  // namespace bpg

namespace {

struct MrfHost {
    int W, H, M, Mp, T, Teff;
    std::vector<float> tablef;
    std::vector<int32_t> tablei;
    double fbar;
    void *unary = nullptr;
    void *msg[2] = {nullptr, nullptr};
};

struct BatchGraphKey {
    int n, mode, cur, family, gen, blocks;
    bool operator<(const BatchGraphKey &o) const {
        return std::tie(n, mode, cur, family, gen, blocks) < std::tie(o.n, o.mode, o.cur, o.family, o.gen, o.blocks);
    }
};

thread_local std::string g_batch_err;

}  // namespace

struct bp_batch_ctx {
    int n = 0;
    bp_dtype dtype = BP_F32;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<MrfHost> mrfs;
    BatchMrf *d_mrfs = nullptr;
    BatchItem *d_items = nullptr;
    int n_items = 0, items_cap = 0;
    unsigned *d_bar = nullptr;   // barrier and work-counter words (kBatchCtlWords)
    int *d_status = nullptr;
    int family = 1;              // lane layout of the launch: 1 or 2 for every MRF, 0 when classes differ
    // work decomposition per (Mp, effective T) class: (family, item size in label words)
    std::map<std::pair<int, int>, std::pair<int, int>> class_cfg;
    std::vector<BatchMrf> dm;    // host copy of the device descriptors
    bool all_full = false;       // every MRF has M == Mp
    bool items_dirty = true;
    int cfg_gen = 0;             // bumped at every rebuild of the items (graphs are keyed by it)
    int cur = 0;
    bool uniform_pending = true;
    bool use_graphs = true;
    std::map<BatchGraphKey, cudaGraphExec_t> graphs;
    int extra_arrivals = 0;
    unsigned long long limit_ns = 2000000000ull;
    long long launches = 0;
    std::string err;
};

static bp_status bfail(bp_batch b, bp_status st, const std::string &m) {
    if (b) b->err = m; else g_batch_err = m;
    if (st != BP_OK) log_error(st, m);
    return st;
}

#define BB_CK(b, call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? BP_ERR_OOM : BP_ERR_CUDA,              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    } while (0)

static void clear_batch_graphs(bp_batch b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

static std::pair<int, int> class_of(const MrfHost &m) { return {m.Mp, m.Teff}; }

// Install each class's lane layout in the device descriptors; the launch
// family is that layout when every class shares it, else 0 (per MRF).
static bp_status apply_class_cfg(bp_batch b) {
    int fam = -1;
    for (int k = 0; k < b->n; ++k) {
        const int f = b->class_cfg[class_of(b->mrfs[k])].first;
        b->dm[k].family = f;
        fam = fam < 0 || fam == f ? f : 0;
    }
    b->family = fam < 0 ? 1 : fam;
    BB_CK(b, cudaMemcpyAsync(b->d_mrfs, b->dm.data(), b->n * sizeof(BatchMrf), cudaMemcpyHostToDevice, b->stream));
    BB_CK(b, cudaStreamSynchronize(b->stream));
    b->items_dirty = true;
    return BP_OK;
}

// Cut every MRF into items of about its class's item size in label words,
// whole groups of nodes, listed class by class: widest band first, then most
// labels (one compiled variant of the kernel per class).  only: restrict to
// that class (the autotuner times classes alone).  Cached graphs hold the
// item list's address and count, so they are dropped.
static bp_status build_items(bp_batch b, const std::pair<int, int> *only = nullptr) {
    clear_batch_graphs(b);
    std::vector<int> order(b->n);
    for (int k = 0; k < b->n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const MrfHost &p = b->mrfs[x], &q = b->mrfs[y];
        return std::make_pair(p.Teff, p.Mp) > std::make_pair(q.Teff, q.Mp);
    });
    std::vector<BatchItem> items;
    for (int k : order) {
        const MrfHost &m = b->mrfs[k];
        if (only && class_of(m) != *only) continue;
        const std::pair<int, int> cfg = b->class_cfg[class_of(m)];
        const int gpb = kBlock / batch_lanes_per_node(cfg.first, m.Mp);
        int tile = std::max(gpb, (cfg.second / m.Mp) / gpb * gpb);
        const int N = m.W * m.H;
        for (int n0 = 0; n0 < N; n0 += tile) items.push_back(BatchItem{k, n0, std::min(tile, N - n0)});
    }
    if ((int)items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        BB_CK(b, cudaMalloc(&b->d_items, items.size() * sizeof(BatchItem)));
        b->items_cap = (int)items.size();
    }
    if (!items.empty())
        BB_CK(b, cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                                 b->stream));
    BB_CK(b, cudaStreamSynchronize(b->stream));
    b->n_items = (int)items.size();
    b->items_dirty = only != nullptr;   // a one-class list is not the batch's
    ++b->cfg_gen;
    return BP_OK;
}

static int batch_blocks(bp_batch b) {
    const int maxb = b->dtype == BP_I32 ? batch_max_blocks_min(b->family, false, b->all_full)
                                        : batch_max_blocks_sum(b->family, false, b->all_full);
    return std::max(1, std::min(maxb, b->n_items));
}

static cudaError_t issue_batch(bp_batch b, int n_iters, int cur) {
    BatchArgs a{};
    a.mrfs = b->d_mrfs;
    a.items = b->d_items;
    a.n_items = b->n_items;
    a.n_iters = n_iters;
    a.start_buf = cur;
    a.bar_count = b->d_bar;
    a.bar_gen = b->d_bar + kBatchGenWord;
    a.tickets = reinterpret_cast<unsigned long long *>(b->d_bar + kBatchTicketWord);
    a.full = b->all_full ? 1 : 0;
    a.extra_arrivals = b->extra_arrivals;
    a.limit_ns = b->limit_ns;
    a.status = b->d_status;
    // arrivals and the ticket counter start at 0
    cudaError_t e = cudaMemsetAsync(b->d_bar, 0, kBatchZeroBytes, b->stream);
    if (e != cudaSuccess) return e;
    const int blocks = batch_blocks(b);
    return b->dtype == BP_I32 ? launch_batch_min(a, b->family, blocks, b->stream)
                              : launch_batch_sum(a, b->family, blocks, b->stream);
}

static bp_status materialize_batch(bp_batch b) {
    if (!b->uniform_pending) return BP_OK;
    for (auto &m : b->mrfs) {
        const long long rows = 4LL * m.W * m.H;
        if (b->dtype == BP_I32)
            BB_CK(b, launch_fill_messages_i32((int32_t *)m.msg[b->cur], rows, m.M, m.Mp, 0, b->stream));
        else
            BB_CK(b, launch_fill_messages_f32((float *)m.msg[b->cur], rows, m.M, m.Mp, 1.0f / (float)m.M, b->stream));
        b->launches += 1;
    }
    b->uniform_pending = false;
    return BP_OK;
}

extern "C" {

const char *bp_batch_last_error(bp_batch b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

long long bp_batch_launch_count(bp_batch b) { return b ? b->launches : -1; }

void bp_batch_destroy(bp_batch b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    clear_batch_graphs(b);
    for (auto &m : b->mrfs) {
        if (m.unary) cudaFree(m.unary);
        if (m.msg[0]) cudaFree(m.msg[0]);
        if (m.msg[1]) cudaFree(m.msg[1]);
    }
    void *bufs[] = {b->d_mrfs, b->d_items, b->d_bar, b->d_status};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

bp_status bp_batch_create(int n, const bp_mrf_desc *descs, bp_dtype dtype, void *cuda_stream, bp_batch *out) {
    BPG_TRACE("bp_batch_create");
    g_batch_err.clear();
    if (!out) return bfail(nullptr, BP_ERR_ARG, "bp_batch_create: out is NULL");
    *out = nullptr;
    if (n < 1 || !descs) return bfail(nullptr, BP_ERR_ARG, "bp_batch_create: need n >= 1 descriptors");
    if (dtype != BP_F32 && dtype != BP_I32) return bfail(nullptr, BP_ERR_ARG, "bp_batch_create: unknown dtype");
    for (int k = 0; k < n; ++k) {
        const bp_mrf_desc &d = descs[k];
        std::string where = "bp_batch_create: MRF " + std::to_string(k) + ": ";
        if (d.W < 1 || d.H < 1 || (long long)d.W * d.H > (1LL << 28))
            return bfail(nullptr, BP_ERR_ARG, where + "bad W or H");
        if (d.M < 2 || d.M > 256) return bfail(nullptr, BP_ERR_ARG, where + "M must be in [2, 256]");
        if (d.T < 0 || !d.dev_unary || !d.host_table) return bfail(nullptr, BP_ERR_ARG, where + "bad T or NULL pointer");
        if (std::min(d.T, d.M - 1) > kTMaxFast)
            return bfail(nullptr, BP_ERR_UNSUPPORTED, where + "batched runs serve band half-widths T <= 8");
        if (!std::isfinite(d.fbar) || d.fbar < 0) return bfail(nullptr, BP_ERR_ARG, where + "fbar must be >= 0");
        if (dtype == BP_I32) {
            const int32_t *t = (const int32_t *)d.host_table;
            if (d.fbar != std::floor(d.fbar) || d.fbar >= (double)(1 << 26))
                return bfail(nullptr, BP_ERR_ARG, where + "Ebar must be an integer in [0, 2^26)");
            for (int i = 0; i < 2 * d.T + 1; ++i) {
                if (t[i] < 0 || t[i] >= (1 << 26)) return bfail(nullptr, BP_ERR_ARG, where + "energies out of range");
                if (t[i] > (int32_t)d.fbar)
                    return bfail(nullptr, BP_ERR_POTENTIAL, where + "E(d) > Ebar; Eq. 11 needs f >= fbar (Sec. 5)");
            }
        } else {
            const float *t = (const float *)d.host_table;
            for (int i = 0; i < 2 * d.T + 1; ++i)
                if (!std::isfinite(t[i]) || t[i] < 0) return bfail(nullptr, BP_ERR_ARG, where + "bad table entry");
        }
    }
    bp_batch b = new bp_batch_ctx();
    b->n = n;
    b->dtype = dtype;
    cudaGetDevice(&b->device);
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault) != cudaSuccess) {
            delete b;
            return bfail(nullptr, BP_ERR_CUDA, "bp_batch_create: stream creation failed");
        }
        b->own_stream = true;
    }
    std::vector<BatchMrf> dm(n);
    bp_status st = BP_OK;
    for (int k = 0; k < n && st == BP_OK; ++k) {
        const bp_mrf_desc &d = descs[k];
        MrfHost m;
        m.W = d.W; m.H = d.H; m.M = d.M; m.Mp = padded_labels(d.M);
        if (m.Mp < 16) m.Mp = 16;
        m.T = d.T; m.Teff = std::min(d.T, d.M - 1); m.fbar = d.fbar;
        const size_t nodes = (size_t)d.W * d.H;
        const size_t ub = nodes * m.Mp * 4, sb = 4 * ub;
        b->mrfs.push_back(m);
        MrfHost &mm = b->mrfs.back();
        if (cudaMalloc(&mm.unary, ub) != cudaSuccess || cudaMalloc(&mm.msg[0], sb) != cudaSuccess ||
            cudaMalloc(&mm.msg[1], sb) != cudaSuccess) {
            cudaGetLastError();
            st = bfail(nullptr, BP_ERR_OOM, "bp_batch_create: device allocation failed");
            break;
        }
        cudaError_t e = dtype == BP_F32
                            ? launch_pad_copy_f32((const float *)d.dev_unary, (float *)mm.unary, nodes, d.M, mm.Mp, 0, b->stream)
                            : launch_pad_copy_i32((const int32_t *)d.dev_unary, (int32_t *)mm.unary, nodes, d.M, mm.Mp,
                                                  b->stream);
        if (e != cudaSuccess) { st = bfail(nullptr, BP_ERR_CUDA, "bp_batch_create: unary copy failed"); break; }
        b->launches += 1;
        BatchMrf &x = dm[k];
        x = BatchMrf{};
        x.unary = mm.unary;
        x.msg[0] = mm.msg[0];
        x.msg[1] = mm.msg[1];
        x.plane = (long long)nodes * mm.Mp;
        x.W = d.W; x.H = d.H; x.M = d.M; x.Mp = mm.Mp; x.T = mm.Teff;
        if (dtype == BP_F32) {
            const float *t = (const float *)d.host_table;
            mm.tablef.assign(t, t + 2 * d.T + 1);
            x.fbar = (float)d.fbar;
            for (int dd = -mm.Teff; dd <= mm.Teff; ++dd) x.wf[dd + mm.Teff] = (float)((double)t[dd + d.T] - (double)x.fbar);
        } else {
            const int32_t *t = (const int32_t *)d.host_table;
            mm.tablei.assign(t, t + 2 * d.T + 1);
            x.ebar = (int32_t)d.fbar;
            std::vector<int32_t> wv;
            for (int dd = -mm.Teff; dd <= mm.Teff; ++dd) {
                x.wi[dd + mm.Teff] = t[dd + d.T];
                wv.push_back(t[dd + d.T]);
            }
            x.zero_min = bpg_zero_min(wv) ? 1 : 0;
            x.packed16 = bpg_packed16(wv, x.ebar) ? 1 : 0;
        }
    }
    if (st == BP_OK) {
        if (cudaMalloc(&b->d_mrfs, n * sizeof(BatchMrf)) != cudaSuccess ||
            cudaMalloc(&b->d_bar, kBatchCtlWords * sizeof(unsigned)) != cudaSuccess ||
            cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            st = bfail(nullptr, BP_ERR_OOM, "bp_batch_create: device allocation failed");
        }
    }
    if (st == BP_OK) {
        if (cudaMemcpyAsync(b->d_mrfs, dm.data(), n * sizeof(BatchMrf), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
            cudaMemsetAsync(b->d_bar, 0, kBatchCtlWords * sizeof(unsigned), b->stream) != cudaSuccess ||
            cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            st = bfail(nullptr, BP_ERR_CUDA, "bp_batch_create: descriptor upload failed");
    }
    if (st == BP_OK) {
        b->all_full = true;
        for (const MrfHost &m : b->mrfs) {
            b->all_full = b->all_full && m.M == m.Mp;
            b->class_cfg[class_of(m)] = {1, 16384};   // until tuned: one chunk per lane, 16 K-word items
        }
        b->dm = dm;
        st = apply_class_cfg(b);
        if (!st) st = build_items(b);
        if (st) g_batch_err = b->err;
    }
    if (st != BP_OK) {
        bp_batch_destroy(b);
        return st;
    }
    *out = b;
    return BP_OK;
}

bp_status bp_batch_reset_messages(bp_batch b) {
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_reset_messages: NULL batch");
    b->err.clear();
    b->uniform_pending = true;
    return BP_OK;
}

static bool tiling_ok(int family, int tile_words) {
    return (family == 1 || family == 2) && tile_words >= 256 && tile_words <= (1 << 24);
}

bp_status bp_batch_set_tiling(bp_batch b, int family, int tile_words) {
    BPG_TRACE("bp_batch_set_tiling");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_set_tiling: NULL batch");
    b->err.clear();
    if (!tiling_ok(family, tile_words))
        return bfail(b, BP_ERR_ARG, "bp_batch_set_tiling: family must be 1 or 2 and the tile in [256, 2^24] words");
    for (auto &kv : b->class_cfg) kv.second = {family, tile_words};
    if (bp_status st = apply_class_cfg(b)) return st;
    return build_items(b);
}

// the setting of the class holding the most label words
bp_status bp_batch_get_tiling(bp_batch b, int *family, int *tile_words) {
    if (!b || !family || !tile_words) return bfail(b, BP_ERR_ARG, "bp_batch_get_tiling: NULL argument");
    std::map<std::pair<int, int>, long long> words;
    for (const MrfHost &m : b->mrfs) words[class_of(m)] += (long long)m.W * m.H * m.Mp;
    auto best = words.begin();
    for (auto it = words.begin(); it != words.end(); ++it)
        if (it->second > best->second) best = it;
    *family = b->class_cfg[best->first].first;
    *tile_words = b->class_cfg[best->first].second;
    return BP_OK;
}

int bp_batch_class_count(bp_batch b) { return b ? (int)b->class_cfg.size() : -1; }

bp_status bp_batch_get_class_tiling(bp_batch b, int k, int *Mp, int *T, int *family, int *tile_words) {
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_get_class_tiling: NULL batch");
    b->err.clear();
    if (!Mp || !T || !family || !tile_words) return bfail(b, BP_ERR_ARG, "bp_batch_get_class_tiling: NULL argument");
    if (k < 0 || k >= (int)b->class_cfg.size()) return bfail(b, BP_ERR_ARG, "bp_batch_get_class_tiling: no class k");
    auto it = b->class_cfg.begin();
    std::advance(it, k);
    *Mp = it->first.first;
    *T = it->first.second;
    *family = it->second.first;
    *tile_words = it->second.second;
    return BP_OK;
}

bp_status bp_batch_set_class_tiling(bp_batch b, int Mp, int T, int family, int tile_words) {
    BPG_TRACE("bp_batch_set_class_tiling");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_set_class_tiling: NULL batch");
    b->err.clear();
    auto it = b->class_cfg.find({Mp, T});
    if (it == b->class_cfg.end()) return bfail(b, BP_ERR_ARG, "bp_batch_set_class_tiling: no MRF has that (Mp, T)");
    if (!tiling_ok(family, tile_words))
        return bfail(b, BP_ERR_ARG, "bp_batch_set_class_tiling: family must be 1 or 2 and the tile in [256, 2^24] words");
    it->second = {family, tile_words};
    if (bp_status st = apply_class_cfg(b)) return st;
    return build_items(b);
}

bp_status bp_batch_set_wait_limit(bp_batch b, double seconds, int extra_arrivals) {
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_set_wait_limit: NULL batch");
    b->err.clear();
    if (!(seconds > 0) || seconds > 60 || extra_arrivals < 0 || extra_arrivals > 1)
        return bfail(b, BP_ERR_ARG, "bp_batch_set_wait_limit: need 0 < seconds <= 60 and extra in {0, 1}");
    b->limit_ns = (unsigned long long)(seconds * 1e9);
    b->extra_arrivals = extra_arrivals;
    clear_batch_graphs(b);
    return BP_OK;
}

bp_status bp_batch_iterate(bp_batch b, int n_iters, int mode) {
    BPG_TRACE("bp_batch_iterate");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_iterate: NULL batch");
    b->err.clear();
    if (n_iters < 0) return bfail(b, BP_ERR_ARG, "bp_batch_iterate: n_iters < 0");
    if ((mode == BP_MAX) != (b->dtype == BP_I32) || (mode != BP_SUM && mode != BP_MAX))
        return bfail(b, BP_ERR_ARG, "bp_batch_iterate: BP_SUM needs BP_F32, BP_MAX needs BP_I32");
    if (bp_status st = materialize_batch(b)) return st;
    if (n_iters == 0) return BP_OK;
    if (b->items_dirty)
        if (bp_status st = build_items(b)) return st;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    BB_CK(b, cudaStreamIsCapturing(b->stream, &cap));
    const int end_cur = (b->cur + n_iters) & 1;
    if (b->use_graphs && cap == cudaStreamCaptureStatusNone) {
        const BatchGraphKey key{n_iters, mode, b->cur, b->family, b->cfg_gen, batch_blocks(b)};
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaError_t e = issue_batch(b, n_iters, b->cur);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                ok = e == cudaSuccess && e2 == cudaSuccess && g &&
                     cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
            }
            if (!ok) {
                cudaGetLastError();
                b->use_graphs = false;   // cooperative capture unavailable: launch directly
            } else {
                it = b->graphs.emplace(key, ex).first;
            }
        }
        if (b->use_graphs) {
            BB_CK(b, cudaGraphLaunch(it->second, b->stream));
            b->launches += 1;
            b->cur = end_cur;
            return BP_OK;
        }
    }
    BB_CK(b, issue_batch(b, n_iters, b->cur));
    b->launches += 1;
    b->cur = end_cur;
    return BP_OK;
}

bp_status bp_batch_sync(bp_batch b) {
    BPG_TRACE("bp_batch_sync");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_sync: NULL batch");
    BB_CK(b, cudaStreamSynchronize(b->stream));
    int flag = 0;
    BB_CK(b, cudaMemcpy(&flag, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        BB_CK(b, cudaMemset(b->d_status, 0, sizeof(int)));
        return bfail(b, BP_ERR_TIMEOUT, "the grid barrier of the batch kernel gave up waiting (status " +
                                            std::to_string(flag) + ")");
    }
    return BP_OK;
}

bp_status bp_batch_beliefs(bp_batch b, int k, void *dev_out, int32_t *dev_map) {
    BPG_TRACE("bp_batch_beliefs");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_beliefs: NULL batch");
    b->err.clear();
    if (k < 0 || k >= b->n || !dev_out) return bfail(b, BP_ERR_ARG, "bp_batch_beliefs: bad index or NULL output");
    if (bp_status st = materialize_batch(b)) return st;
    const MrfHost &m = b->mrfs[k];
    const GridDims d{m.W, m.H, m.M, m.Mp, (long long)m.W * m.H * m.Mp};
    if (b->dtype == BP_F32)
        BB_CK(b, launch_beliefs_f32((const float *)m.unary, (const float *)m.msg[b->cur], d, 0, (float *)dev_out, dev_map,
                                    b->stream));
    else
        BB_CK(b, launch_beliefs_i32((const int32_t *)m.unary, (const int32_t *)m.msg[b->cur], d, (int32_t *)dev_out,
                                    dev_map, b->stream));
    b->launches += 1;
    return BP_OK;
}

bp_status bp_batch_get_messages(bp_batch b, int k, void *dev_planes) {
    BPG_TRACE("bp_batch_get_messages");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_get_messages: NULL batch");
    b->err.clear();
    if (k < 0 || k >= b->n || !dev_planes) return bfail(b, BP_ERR_ARG, "bp_batch_get_messages: bad index or NULL output");
    if (bp_status st = materialize_batch(b)) return st;
    const MrfHost &m = b->mrfs[k];
    BB_CK(b, launch_unpad_messages(m.msg[b->cur], dev_planes, m.W, m.H, m.M, m.Mp, 0, b->stream));
    b->launches += 1;
    return BP_OK;
}

// Project-written autotuner, per (Mp, T) class: every (family, tile)
// candidate runs the class's items alone for n_iters iterations (after one
// warm-up run) on the kernel compiled for that family; the fastest is kept for
// the class.  Then whole-batch candidates are timed: the per-class choices,
// those item sizes with one lane layout for every class, and the uniform
// settings; the fastest is kept and its time per iteration returned.  The choices are recorded in a cache file
// keyed by the batch's classes and size (path: $BP_AUTOTUNE_CACHE, if set).
// Leaves the messages reset to the uniform state.
bp_status bp_batch_autotune(bp_batch b, int mode, int n_iters, float *host_best_ms) {
    BPG_TRACE("bp_batch_autotune");
    if (!b) return bfail(nullptr, BP_ERR_ARG, "bp_batch_autotune: NULL batch");
    b->err.clear();
    if (n_iters < 1) return bfail(b, BP_ERR_ARG, "bp_batch_autotune: n_iters < 1");
    if ((mode == BP_MAX) != (b->dtype == BP_I32) || (mode != BP_SUM && mode != BP_MAX))
        return bfail(b, BP_ERR_ARG, "bp_batch_autotune: BP_SUM needs BP_F32, BP_MAX needs BP_I32");
    std::ostringstream sig;
    long long words = 0;
    std::map<std::pair<int, int>, long long> classes;
    for (auto &m : b->mrfs) {
        classes[class_of(m)] += (long long)m.W * m.H;
        words += (long long)m.W * m.H * m.Mp;
    }
    sig << (b->dtype == BP_I32 ? "i32" : "f32") << ":m" << mode << ":w" << (int)std::log2((double)words + 1);
    for (auto &kv : classes) sig << ":" << kv.first.first << "x" << kv.first.second;
    const char *cache = std::getenv("BP_AUTOTUNE_CACHE");
    if (cache) {
        // line: signature, class count, then (Mp, T, family, tile) per class, then ms per iteration
        std::ifstream in(cache);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ls(line);
            std::string key;
            int nc = 0;
            if (!(ls >> key >> nc) || key != sig.str() || nc != (int)b->class_cfg.size()) continue;
            std::map<std::pair<int, int>, std::pair<int, int>> cfg;
            bool good = true;
            for (int i = 0; i < nc && good; ++i) {
                int mp, t, f, tile;
                good = (bool)(ls >> mp >> t >> f >> tile) && b->class_cfg.count({mp, t}) && tiling_ok(f, tile);
                if (good) cfg[{mp, t}] = {f, tile};
            }
            float ms = 0.f;
            if (!good || !(ls >> ms) || (int)cfg.size() != nc) continue;
            b->class_cfg = cfg;
            if (bp_status st = apply_class_cfg(b)) return st;
            if (bp_status st = build_items(b)) return st;
            if (host_best_ms) *host_best_ms = ms;
            return bp_batch_reset_messages(b);
        }
    }
    const int fams[] = {1, 2};
    const int tiles[] = {16384, 65536, 262144};
    cudaEvent_t e0, e1;
    BB_CK(b, cudaEventCreate(&e0));
    BB_CK(b, cudaEventCreate(&e1));
    bp_status st = materialize_batch(b);
    auto timed = [&](auto &&run, float *ms) -> bp_status {
        bp_status r = run();   // warm-up
        if (!r && cudaEventRecord(e0, b->stream) != cudaSuccess) r = BP_ERR_CUDA;
        if (!r) r = run();
        if (!r && cudaEventRecord(e1, b->stream) != cudaSuccess) r = BP_ERR_CUDA;
        if (!r) r = bp_batch_sync(b);
        if (!r && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) r = BP_ERR_CUDA;
        return r;
    };
    for (auto &kv : classes) {
        if (st) break;
        const std::pair<int, int> c = kv.first;
        float best = 3e38f;
        std::pair<int, int> best_cfg = b->class_cfg[c];
        for (int f : fams)
            for (int t : tiles) {
                if (st) break;
                b->class_cfg[c] = {f, t};
                st = build_items(b, &c);
                const int saved_family = b->family;
                b->family = f;   // the class alone runs the kernel compiled for its family
                float ms = 0.f;
                if (!st)
                    st = timed([&]() -> bp_status {
                        return issue_batch(b, n_iters, b->cur) == cudaSuccess ? BP_OK : BP_ERR_CUDA;
                    }, &ms);
                b->family = saved_family;
                if (!st && ms < best) {
                    best = ms;
                    best_cfg = {f, t};
                }
            }
        b->class_cfg[c] = best_cfg;
    }
    // whole-batch candidates: the per-class choices; the same item sizes with
    // one lane layout for every class (one compiled family per launch is
    // cheaper than a launch that switches layouts); one setting for all
    std::vector<std::map<std::pair<int, int>, std::pair<int, int>>> cands;
    cands.push_back(b->class_cfg);
    for (int f : fams) {
        auto c = b->class_cfg;
        for (auto &kv : c) kv.second.first = f;
        cands.push_back(c);
    }
    for (int f : fams)
        for (int t : tiles) {
            auto c = b->class_cfg;
            for (auto &kv : c) kv.second = {f, t};
            cands.push_back(c);
        }
    float total = 3e38f;
    std::map<std::pair<int, int>, std::pair<int, int>> best_cfg = b->class_cfg;
    for (const auto &c : cands) {
        if (st) break;
        b->class_cfg = c;
        float ms = 0.f;
        st = apply_class_cfg(b);
        if (!st) st = build_items(b);
        if (!st) st = timed([&]() { return bp_batch_iterate(b, n_iters, mode); }, &ms);
        if (!st && ms < total) {
            total = ms;
            best_cfg = c;
        }
    }
    b->class_cfg = best_cfg;
    if (!st) st = apply_class_cfg(b);
    if (!st) st = build_items(b);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st == BP_ERR_CUDA ? bfail(b, st, "bp_batch_autotune: timing failed") : st;
    if (cache) {
        std::ofstream o(cache, std::ios::app);
        o << sig.str() << " " << b->class_cfg.size();
        for (auto &kv : b->class_cfg)
            o << " " << kv.first.first << " " << kv.first.second << " " << kv.second.first << " " << kv.second.second;
        o << " " << total / n_iters << "\n";
    }
    if (host_best_ms) *host_best_ms = total / n_iters;
    return bp_batch_reset_messages(b);
}

}  // extern "C"
