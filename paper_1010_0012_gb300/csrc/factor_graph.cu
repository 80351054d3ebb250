// Factor-graph BP with three-variable factors whose compatible triplets are
// sparse (Sec. 7): with f = fbar outside a set of C triplets, the message from
// a factor to its slot-s variable is
//   m(x_s) = sum_{compatible (x_0, x_1, x_2) with that x_s} [f - fbar] n_u(x_u) n_w(x_w)
//            + fbar (sum_x n_u(x)) (sum_x n_w(x))
// (u, w the other two slots): O(C + M) instead of the O(M^3) of the standard
// update, and for min-sum (energies, E <= Ebar)
//   m(x_s) = min( min_{compatible} [E + n_u(x_u) + n_w(x_w)], Ebar + min n_u + min n_w ).
// Declarations and the contract of every call are in include/bp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "trace.h"
#include "../../include/bp.h"
#include "bp_internal.h"

namespace {

constexpr int kFgBlock = 256;
constexpr int kFgWarps = kFgBlock / 32;
constexpr int kMaxDegree = 16;
constexpr int32_t kBig = 1 << 30;

struct FgDims {
    int n_vars, n_factors, M, Mp;
};

// ---- variable -> factor: n = unary x the other incoming factor messages ------
// One warp per variable, lane l on labels l, l + 32, ...  Each incoming
// message is read once per pass; the product over all incoming messages but
// the k-th comes from prefix and suffix products (min-sum: the total minus the
// k-th term, exact in integers).  Pass 0 forms the normaliser (sum) or the
// minimum of every outgoing message, pass 1 writes the normalised messages.
template <bool MIN, typename E, int D>
__device__ __forceinline__ void v2f_label(const E *unary, const E *m_fv, const int (&inc)[D], int deg, long long v,
                                          int x, const FgDims &d, E (&out)[D]) {
    E m[D];
#pragma unroll
    for (int j = 0; j < D; ++j) m[j] = j < deg ? m_fv[(long long)inc[j] * d.Mp + x] : (MIN ? E(0) : E(1));
    const E u = unary[v * d.Mp + x];
    if (MIN) {
        E tot = u;
#pragma unroll
        for (int j = 0; j < D; ++j) tot += m[j];
#pragma unroll
        for (int k = 0; k < D; ++k) out[k] = tot - m[k];
    } else {
        // out[k] = u * prod_{j < k} m_j * prod_{j > k} m_j
        E pre = u;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            out[k] = pre;
            pre *= m[k];
        }
        E suf = E(1);
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            out[k] *= suf;
            suf *= m[k];
        }
    }
    if (x >= d.M)
#pragma unroll
        for (int k = 0; k < D; ++k) out[k] = MIN ? E(kBig) : E(0);
}

// D: a bound on the degree of every variable (4, 8 or 16).  Four blocks per
// SM: the kernel waits on its message loads, and at D = 8 the 64-register
// bound costs no spill (three blocks at the compiler's own choice were
// 3 % slower over a factor-graph iteration)
template <bool MIN, typename E, int D>
__global__ void __launch_bounds__(256, 4) v2f_kernel(const E *unary, const int32_t *var_ptr, const int32_t *var_inc, const E *m_fv, E *n_vf,
                           FgDims d) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    // A variable costs three dependent round trips: its row bounds, its
    // incidence list, its messages.  The walk loads the row bounds two steps
    // ahead and the incidence list one step ahead, so only the messages wait.
    long long v = warp;
    int deg = 0, p1 = 0, deg1 = 0;
    int inc[D];
    {
        int p0 = 0;
        if (v < d.n_vars) { p0 = var_ptr[v]; deg = var_ptr[v + 1] - p0; }
        if (v + nw < d.n_vars) { p1 = var_ptr[v + nw]; deg1 = var_ptr[v + nw + 1] - p1; }
#pragma unroll
        for (int j = 0; j < D; ++j) inc[j] = j < deg ? var_inc[p0 + j] : 0;
    }
    for (; v < d.n_vars; v += nw) {
        int p2 = 0, deg2 = 0;
        if (v + 2 * nw < d.n_vars) { p2 = var_ptr[v + 2 * nw]; deg2 = var_ptr[v + 2 * nw + 1] - p2; }
        int incn[D];
#pragma unroll
        for (int j = 0; j < D; ++j) incn[j] = j < deg1 ? var_inc[p1 + j] : 0;
        E acc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = MIN ? E(kBig) : E(0);
        E out[D];
        for (int x = lane; x < d.Mp; x += 32) {
            v2f_label<MIN, E, D>(unary, m_fv, inc, deg, v, x, d, out);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (MIN) acc[k] = out[k] < acc[k] ? out[k] : acc[k]; else acc[k] += out[k];
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (k >= deg) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const E y = __shfl_xor_sync(0xffffffffu, acc[k], o);
                if (MIN) acc[k] = y < acc[k] ? y : acc[k]; else acc[k] += y;
            }
        }
        for (int x = lane; x < d.Mp; x += 32) {
            v2f_label<MIN, E, D>(unary, m_fv, inc, deg, v, x, d, out);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (k >= deg) break;
                E o;
                if (MIN) o = x < d.M ? out[k] - acc[k] : E(0);
                else o = out[k] / acc[k];
                n_vf[(long long)inc[k] * d.Mp + x] = o;
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) inc[j] = incn[j];
        deg = deg1;
        p1 = p2;
        deg1 = deg2;
    }
}

// ---- factor -> variable: the O(C + M) update -----------------------------------
// The triplet list is held per slot s and output label x_s as a list of
// (x_u | x_w << 16, weight bits), sorted by the offsets (x_u - x_s, x_w - x_s)
// mod M so that lanes working on neighbouring labels gather n_u and n_w from
// different banks of the warp's shared-memory copy of the incoming messages.
// The lists are dealt to lanes in pairs (longest with shortest of the slot,
// on lanes 2j and 2j + 1 of chunk k): the even lane takes the first half of
// the pair's entries, all of the long list's; the odd lane the long list's
// rest (its foreign entries, summed apart) and then its own short list.  One
// shuffle returns the foreign partial to its owner.  A slot then costs about
// its mean list length instead of its longest.  Entries are interleaved by
// lane (step i of chunk k at i * 32 KM + 32 k + lane: consecutive lanes read
// consecutive words, through L1, where the table stays).  One warp per
// factor; no atomics.
// chunks of 32 labels per lane of the compiled f2v kernels (1, 2, 4 or 8)
inline int f2v_chunks(int Mp) {
    const int km = (Mp + 31) / 32;
    return km <= 1 ? 1 : km <= 2 ? 2 : km <= 4 ? 4 : 8;
}

struct FgTable {
    const int2 *ell;        // per slot: [rows_s][32 KM] entries
    const int32_t *meta;    // [3][KM][32][3]: entry count, foreign count, own label (-1: none)
                            // (the kernel reads the last two: past its count a lane reads padding)
    long long base[3];      // start of slot s in ell
    int rows[3];            // steps of slot s
};

template <bool MIN, typename E, int KM>
__global__ void __launch_bounds__(kFgBlock) f2v_kernel(const E *n_vf, E *m_fv, const FgTable tab, FgDims d,
                                                       E fbar_or_ebar) {
    extern __shared__ uint8_t sm[];
    const int M = d.M, Mp = d.Mp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    E *n = (E *)sm + warp * 3 * Mp;                       // [3][Mp] per warp
    const long long gw = (long long)blockIdx.x * kFgWarps + warp, nw = (long long)gridDim.x * kFgWarps;
    for (long long a = gw; a < d.n_factors; a += nw) {
        E red[3];
        for (int s = 0; s < 3; ++s) red[s] = MIN ? E(kBig) : E(0);
        for (int x = lane; x < Mp; x += 32)
            for (int s = 0; s < 3; ++s) {
                E v = n_vf[(a * 3 + s) * Mp + x];
                if (MIN && x >= M) v = E(kBig);
                n[s * Mp + x] = v;
                if (x < M) {
                    if (MIN) red[s] = v < red[s] ? v : red[s]; else red[s] += v;
                }
            }
        for (int s = 0; s < 3; ++s)
            for (int o = 16; o > 0; o >>= 1) {
                const E y = __shfl_xor_sync(0xffffffffu, red[s], o);
                if (MIN) red[s] = y < red[s] ? y : red[s]; else red[s] += y;
            }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int u = s == 0 ? 1 : 0, w = s == 2 ? 1 : 2;   // the other two slots, in order
            const E *nu = n + u * Mp, *nwv = n + w * Mp;
            const E flat = MIN ? fbar_or_ebar + red[u] + red[w] : fbar_or_ebar * red[u] * red[w];
            const int2 *ell = tab.ell + tab.base[s] + lane;
            int nx[KM], lab[KM];
            E acc[KM], accx[KM];
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int32_t *mt = tab.meta + (((long long)s * KM + k) * 32 + lane) * 3;
                nx[k] = __ldg(mt + 1);
                lab[k] = __ldg(mt + 2);
                acc[k] = MIN ? flat : E(0);
                accx[k] = MIN ? E(kBig) : E(0);
            }
            // every lane runs the slot's steps: past its own list it reads
            // padding entries that change nothing, so the loads carry no
            // per-lane bound and the unrolled steps keep several in flight
            const int rows = tab.rows[s];
#pragma unroll 4
            for (int i = 0; i < rows; ++i) {
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    const int2 e = __ldg(ell + (long long)i * (32 * KM) + 32 * k);
                    const E gu = nu[e.x & 0xffff], gwv = nwv[e.x >> 16];
                    if (i < nx[k]) {
                        if (MIN) accx[k] = __viaddmin_s32(e.y, gu + gwv, accx[k]);
                        else accx[k] = fmaf(__int_as_float(e.y), gu * gwv, accx[k]);
                    } else {
                        if (MIN) acc[k] = __viaddmin_s32(e.y, gu + gwv, acc[k]);
                        else acc[k] = fmaf(__int_as_float(e.y), gu * gwv, acc[k]);
                    }
                }
            }
            E norm = MIN ? E(kBig) : E(0);
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                // the partner lane's foreign entries belong to this lane's label
                const E o = __shfl_xor_sync(0xffffffffu, accx[k], 1);
                if (MIN) acc[k] = o < acc[k] ? o : acc[k]; else acc[k] += o;
                if (lab[k] >= 0 && lab[k] < M) {
                    if (!MIN) acc[k] += flat;
                    if (MIN) norm = acc[k] < norm ? acc[k] : norm; else norm += acc[k];
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const E y = __shfl_xor_sync(0xffffffffu, norm, o);
                if (MIN) norm = y < norm ? y : norm; else norm += y;
            }
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                const int x = lab[k];
                if (x >= 0) {
                    E v;
                    if (MIN) v = x < M ? acc[k] - norm : E(0);
                    else v = x < M ? acc[k] / norm : E(0);
                    m_fv[(a * 3 + s) * Mp + x] = v;
                }
            }
        }
        __syncwarp();   // the warp's copy of the messages is rewritten for its next factor
    }
}

// ---- the standard O(M^3) update on CUDA cores (comparison) ---------------------
template <bool MIN, typename E>
__global__ void f2v_dense_kernel(const E *n_vf, E *m_fv, const E *F, FgDims d) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int M = d.M, Mp = d.Mp;
    for (long long a = warp; a < d.n_factors; a += nw) {
        const E *n = n_vf + a * 3 * Mp;
        for (int s = 0; s < 3; ++s) {
            const int u = s == 0 ? 1 : 0, w = s == 2 ? 1 : 2;
            E norm = MIN ? E(kBig) : E(0);
            E outv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int x = lane + 32 * k;
                if (k * 32 >= Mp) break;
                E acc = MIN ? E(kBig) : E(0);
                if (x < M) {
                    for (int xu = 0; xu < M; ++xu)
                        for (int xw = 0; xw < M; ++xw) {
                            int idx[3];
                            idx[s] = x; idx[u] = xu; idx[w] = xw;
                            const E f = F[((long long)idx[0] * M + idx[1]) * M + idx[2]];
                            if (MIN) {
                                const E t = f + n[u * Mp + xu] + n[w * Mp + xw];
                                acc = t < acc ? t : acc;
                            } else {
                                acc = fmaf(f, n[u * Mp + xu] * n[w * Mp + xw], acc);
                            }
                        }
                    if (MIN) norm = acc < norm ? acc : norm; else norm += acc;
                }
                outv[k] = acc;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const E y = __shfl_xor_sync(0xffffffffu, norm, o);
                if (MIN) norm = y < norm ? y : norm; else norm += y;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int x = lane + 32 * k;
                if (k * 32 >= Mp) break;
                if (x < Mp) {
                    E v;
                    if (MIN) v = x < M ? outv[k] - norm : E(0);
                    else v = x < M ? outv[k] / norm : E(0);
                    m_fv[(a * 3 + s) * Mp + x] = v;
                }
            }
        }
    }
}

template <bool MIN, typename E>
__global__ void fg_beliefs_kernel(const E *unary, const int32_t *var_ptr, const int32_t *var_inc, const E *m_fv,
                                  FgDims d, E *out, int32_t *map) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v = warp; v < d.n_vars; v += nw) {
        const int p0 = var_ptr[v], deg = var_ptr[v + 1] - p0;
        E z = 0;
        for (int pass = 0; pass < 2; ++pass) {
            E best = MIN ? E(kBig) : E(-1);
            int bi = 0x7fffffff;
            for (int x = lane; x < d.M; x += 32) {
                E b = unary[v * d.Mp + x];
                for (int j = 0; j < deg; ++j) {
                    const E mj = m_fv[(long long)var_inc[p0 + j] * d.Mp + x];
                    if (MIN) b += mj; else b *= mj;
                }
                if (pass == 0) {
                    if (!MIN) z += b;
                } else {
                    if (!MIN) b = b / z;
                    out[v * d.M + x] = b;
                    if (MIN ? (b < best) : (b > best)) { best = b; bi = x; }
                }
            }
            if (pass == 0) {
                for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
            } else {
                for (int o = 16; o > 0; o >>= 1) {
                    const E ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if ((MIN ? (ob < best) : (ob > best)) || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (map && lane == 0) map[v] = bi;
            }
        }
    }
}

template <typename E>
__global__ void fg_fill_kernel(E *p, long long rows, int M, int Mp, E v) {
    const long long n = rows * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = (i % Mp) < M ? v : E(0);
}

template <typename E>
__global__ void fg_pad_kernel(const E *src, E *dst, long long rows, int M, int Mp) {
    const long long n = rows * Mp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / Mp;
        const int x = (int)(i - r * Mp);
        dst[i] = x < M ? src[r * M + x] : E(0);
    }
}

thread_local std::string g_fg_err;

}  // namespace

struct bp_fg_ctx {
    int n_vars = 0, n_factors = 0, M = 0, Mp = 0;
    int max_degree = 0;          // largest number of factors of one variable
    bp_dtype dtype = BP_F32;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *unary = nullptr;
    int32_t *var_ptr = nullptr, *var_inc = nullptr;
    void *m_fv = nullptr, *n_vf = nullptr;
    int32_t *d_len = nullptr;   // [3][KM][32][3] per lane: entry count, foreign count, own label
    int2 *d_ell = nullptr;      // interleaved triplet lists (FgTable)
    long long ell_base[3] = {0, 0, 0};
    int ell_rows[3] = {0, 0, 0};   // loop steps per slot
    void *d_dense = nullptr;
    int C = 0;
    double fbar = 0;
    std::vector<int32_t> trip;   // [C][3]
    std::vector<float> valf;
    std::vector<int32_t> vali;
    bool have_unary = false, have_factor = false, uniform_pending = true;
    long long launches = 0;
    std::string err;
};

static bp_status fgfail(bp_factor_graph g, bp_status st, const std::string &m) {
    if (g) g->err = m; else g_fg_err = m;
    if (st != BP_OK) bpg::log_error(st, m);
    return st;
}

#define FG_CK(g, call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return fgfail((g), e_ == cudaErrorMemoryAllocation ? BP_ERR_OOM : BP_ERR_CUDA,             \
                          std::string(#call) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

static size_t f2v_smem(int Mp, int elem) { return (size_t)kFgWarps * 3 * Mp * elem; }

static int warp_grid(long long items) {
    long long b = (items * 32 + 255) / 256;
    const long long cap = (long long)bpg::device_sm_count() * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

template <bool MIN, typename E, int KM>
static cudaError_t launch_f2v(bp_factor_graph g, const FgTable &tab, const FgDims &d) {
    const size_t smem = f2v_smem(g->Mp, sizeof(E));
    const void *fn = (const void *)f2v_kernel<MIN, E, KM>;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFgBlock, smem);
    long long blocks = (long long)bpg::device_sm_count() * std::max(1, per_sm);
    blocks = std::min<long long>(blocks, (g->n_factors + kFgWarps - 1) / kFgWarps);
    f2v_kernel<MIN, E, KM><<<(int)blocks, kFgBlock, smem, g->stream>>>((const E *)g->n_vf, (E *)g->m_fv, tab, d,
                                                                      (E)g->fbar);
    return cudaGetLastError();
}

template <bool MIN, typename E, int D>
static void launch_v2f(bp_factor_graph g, const FgDims &d) {
    v2f_kernel<MIN, E, D><<<warp_grid(g->n_vars), 256, 0, g->stream>>>(
        (const E *)g->unary, g->var_ptr, g->var_inc, (const E *)g->m_fv, (E *)g->n_vf, d);
}

extern "C" {

const char *bp_fg_last_error(bp_factor_graph g) { return g ? g->err.c_str() : g_fg_err.c_str(); }
long long bp_fg_launch_count(bp_factor_graph g) { return g ? g->launches : -1; }

void bp_fg_destroy(bp_factor_graph g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    void *bufs[] = {g->unary, g->var_ptr, g->var_inc, g->m_fv, g->n_vf, g->d_len, g->d_ell, g->d_dense};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

bp_status bp_fg_create(int n_vars, int M, int n_factors, const int32_t *host_factor_vars, bp_dtype dtype,
                       void *cuda_stream, bp_factor_graph *out) {
    BPG_TRACE("bp_fg_create");
    g_fg_err.clear();
    if (!out) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_create: out is NULL");
    *out = nullptr;
    if (n_vars < 1 || n_factors < 0 || M < 2 || M > 256 || (n_factors > 0 && !host_factor_vars))
        return fgfail(nullptr, BP_ERR_ARG, "bp_fg_create: need n_vars >= 1, 2 <= M <= 256, factor list");
    if (dtype != BP_F32 && dtype != BP_I32) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_create: unknown dtype");
    if ((long long)n_factors * 3 * 256 >= (1LL << 31) || (long long)n_vars * 256 >= (1LL << 31))
        return fgfail(nullptr, BP_ERR_ARG, "bp_fg_create: graph too large");
    std::vector<int> deg(n_vars, 0);
    for (int a = 0; a < n_factors; ++a) {
        const int32_t *v = host_factor_vars + 3 * a;
        for (int s = 0; s < 3; ++s)
            if (v[s] < 0 || v[s] >= n_vars) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_create: variable out of range");
        if (v[0] == v[1] || v[0] == v[2] || v[1] == v[2])
            return fgfail(nullptr, BP_ERR_ARG, "bp_fg_create: a factor must join three distinct variables");
        for (int s = 0; s < 3; ++s)
            if (++deg[v[s]] > kMaxDegree)
                return fgfail(nullptr, BP_ERR_UNSUPPORTED, "bp_fg_create: a variable is in more than 16 factors");
    }
    bp_factor_graph g = new bp_fg_ctx();
    g->n_vars = n_vars; g->n_factors = n_factors; g->M = M; g->Mp = (M + 3) & ~3; g->dtype = dtype;
    for (int v = 0; v < n_vars; ++v) g->max_degree = std::max(g->max_degree, deg[v]);
    if (cuda_stream) g->stream = (cudaStream_t)cuda_stream;
    else if (cudaStreamCreateWithFlags(&g->stream, cudaStreamDefault) != cudaSuccess) {
        delete g;
        return fgfail(nullptr, BP_ERR_CUDA, "bp_fg_create: stream creation failed");
    } else g->own_stream = true;
    std::vector<int32_t> ptr(n_vars + 1, 0), inc(3 * (size_t)n_factors);
    for (int v = 0; v < n_vars; ++v) ptr[v + 1] = ptr[v] + deg[v];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int a = 0; a < n_factors; ++a)
        for (int s = 0; s < 3; ++s) inc[fill[host_factor_vars[3 * a + s]]++] = 3 * a + s;
    const size_t msgb = (size_t)(n_factors > 0 ? n_factors : 1) * 3 * g->Mp * 4;
    bool ok = cudaMalloc(&g->unary, (size_t)n_vars * g->Mp * 4) == cudaSuccess &&
              cudaMalloc(&g->var_ptr, (n_vars + 1) * 4) == cudaSuccess &&
              cudaMalloc(&g->var_inc, (inc.size() > 0 ? inc.size() : 1) * 4) == cudaSuccess &&
              cudaMalloc(&g->m_fv, msgb) == cudaSuccess && cudaMalloc(&g->n_vf, msgb) == cudaSuccess;
    if (ok) ok = cudaMemcpy(g->var_ptr, ptr.data(), (n_vars + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                 (inc.empty() || cudaMemcpy(g->var_inc, inc.data(), inc.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        bp_fg_destroy(g);
        return fgfail(nullptr, BP_ERR_OOM, "bp_fg_create: device allocation failed");
    }
    *out = g;
    return BP_OK;
}

bp_status bp_fg_set_unary(bp_factor_graph g, const void *dev_unary) {
    BPG_TRACE("bp_fg_set_unary");
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_set_unary: NULL graph");
    g->err.clear();
    if (!dev_unary) return fgfail(g, BP_ERR_ARG, "bp_fg_set_unary: NULL unary");
    if (g->dtype == BP_F32)
        fg_pad_kernel<float><<<bpg::grid_for((long long)g->n_vars * g->Mp, 256), 256, 0, g->stream>>>(
            (const float *)dev_unary, (float *)g->unary, g->n_vars, g->M, g->Mp);
    else
        fg_pad_kernel<int32_t><<<bpg::grid_for((long long)g->n_vars * g->Mp, 256), 256, 0, g->stream>>>(
            (const int32_t *)dev_unary, (int32_t *)g->unary, g->n_vars, g->M, g->Mp);
    FG_CK(g, cudaGetLastError());
    g->launches += 1;
    g->have_unary = true;
    return BP_OK;
}

bp_status bp_fg_set_factor(bp_factor_graph g, int C, const int32_t *host_triplets, const void *host_vals,
                           double fbar) {
    BPG_TRACE("bp_fg_set_factor");
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_set_factor: NULL graph");
    g->err.clear();
    if (C < 0 || (C > 0 && (!host_triplets || !host_vals)))
        return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: bad triplet list");
    if (!std::isfinite(fbar) || fbar < 0) return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: fbar must be >= 0");
    std::vector<char> seen((size_t)g->M * g->M * g->M, 0);
    for (int c = 0; c < C; ++c) {
        const int32_t *t = host_triplets + 3 * c;
        for (int s = 0; s < 3; ++s)
            if (t[s] < 0 || t[s] >= g->M) return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: label out of range");
        char &z = seen[((size_t)t[0] * g->M + t[1]) * g->M + t[2]];
        if (z) return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: repeated triplet");
        z = 1;
    }
    std::vector<int32_t> wbits(C);
    if (g->dtype == BP_F32) {
        const float *v = (const float *)host_vals;
        for (int c = 0; c < C; ++c) {
            if (!std::isfinite(v[c]) || v[c] < 0) return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: bad value");
            const float w = (float)((double)v[c] - (double)(float)fbar);
            wbits[c] = *reinterpret_cast<const int32_t *>(&w);
        }
        g->valf.assign(v, v + C);
    } else {
        if (fbar != std::floor(fbar) || fbar >= (double)(1 << 26))
            return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: Ebar must be an integer in [0, 2^26)");
        const int32_t *v = (const int32_t *)host_vals;
        for (int c = 0; c < C; ++c) {
            if (v[c] < 0 || v[c] >= (1 << 26)) return fgfail(g, BP_ERR_ARG, "bp_fg_set_factor: energy out of range");
            if (v[c] > (int32_t)fbar)
                return fgfail(g, BP_ERR_POTENTIAL, "bp_fg_set_factor: E > Ebar; the max-product form needs f >= fbar");
            wbits[c] = v[c];
        }
        g->vali.assign(v, v + C);
    }
    g->trip.assign(host_triplets, host_triplets + 3 * (size_t)C);
    // per slot s and output label x_s: the list of (x_u, x_w, weight), sorted
    // by the offsets (x_u - x_s, x_w - x_s) mod M, interleaved by label
    const int M = g->M;
    std::vector<std::vector<std::pair<std::pair<int, int>, int2>>> lists((size_t)3 * M);
    for (int c = 0; c < C; ++c) {
        const int32_t *t = host_triplets + 3 * c;
        for (int s = 0; s < 3; ++s) {
            const int u = s == 0 ? 1 : 0, w = s == 2 ? 1 : 2;
            const int key_u = ((t[u] - t[s]) % M + M) % M, key_w = ((t[w] - t[s]) % M + M) % M;
            lists[(size_t)s * M + t[s]].push_back({{key_u, key_w}, make_int2(t[u] | (t[w] << 16), wbits[c])});
        }
    }
    // Balance: per slot, the labels (padded to 32 KM lanes) sorted by list
    // length and paired longest with shortest on the lanes 2j, 2j + 1 of one
    // chunk k.  The pair's two lists are cut in half: the even lane takes the
    // first h entries of the long list, the odd lane the rest of it (its
    // "foreign" entries, into a second accumulator) and then the whole short
    // list.  A slot's loop then runs about its mean list length instead of
    // its longest.  Per (slot, chunk, lane): entry count, foreign count, own
    // label (-1: none).
    const int KM = f2v_chunks(g->Mp), L = 32 * KM;   // the compiled kernel's chunks
    std::vector<int32_t> meta((size_t)3 * L * 3, 0);
    std::vector<std::vector<int2>> lane_list((size_t)3 * L);
    long long base[3], total = 0;
    int rows_s[3];
    for (int s = 0; s < 3; ++s) {
        for (int x = 0; x < M; ++x) {
            auto &l = lists[(size_t)s * M + x];
            std::stable_sort(l.begin(), l.end(), [](const auto &p, const auto &q) { return p.first < q.first; });
        }
        std::vector<int> order(L);
        for (int x = 0; x < L; ++x) order[x] = x;
        auto lenof = [&](int x) { return x < M ? (int)lists[(size_t)s * M + x].size() : 0; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lenof(a) > lenof(b); });
        int rows = 0;
        for (int j = 0; j < L / 2; ++j) {
            const int A = order[j], B = order[L - 1 - j];
            const int la = lenof(A), lb = lenof(B), h = (la + lb + 1) / 2;
            const int k = j / 16, le = 2 * (j % 16), lo = le + 1;
            const size_t pe = ((size_t)s * KM + k) * 32 + le, po = ((size_t)s * KM + k) * 32 + lo;
            auto &ve = lane_list[pe], &vo = lane_list[po];
            for (int i = 0; i < la; ++i) (i < h ? ve : vo).push_back(lists[(size_t)s * M + A][i].second);
            const int nx = (int)vo.size();
            for (int i = 0; i < lb; ++i) vo.push_back(lists[(size_t)s * M + B][i].second);
            meta[pe * 3 + 0] = (int)ve.size();
            meta[pe * 3 + 1] = 0;
            meta[pe * 3 + 2] = A < g->Mp ? A : -1;
            meta[po * 3 + 0] = (int)vo.size();
            meta[po * 3 + 1] = nx;
            meta[po * 3 + 2] = B < g->Mp ? B : -1;
            rows = std::max(rows, (int)std::max(ve.size(), vo.size()));
        }
        rows_s[s] = rows;
        base[s] = total;
        total += (long long)rows * L;
    }
    // steps past a lane's list read an entry that changes nothing: labels 0
    // and weight 0 (sum: adds 0) or E = Ebar (min-sum: never below the flat
    // term Ebar + min n_u + min n_w), so the kernel needs no bound per lane
    const int2 pad = make_int2(0, g->dtype == BP_F32 ? 0 : (int32_t)fbar);
    std::vector<int2> ell((size_t)std::max(1LL, total), pad);
    for (int s = 0; s < 3; ++s)
        for (int k = 0; k < KM; ++k)
            for (int l = 0; l < 32; ++l) {
                const auto &v = lane_list[((size_t)s * KM + k) * 32 + l];
                for (size_t i = 0; i < v.size(); ++i) ell[(size_t)(base[s] + (long long)i * L + k * 32 + l)] = v[i];
            }
    std::vector<int32_t> &len = meta;   // uploaded as the per-lane table
    if (g->d_len) cudaFree(g->d_len);
    if (g->d_ell) cudaFree(g->d_ell);
    if (g->d_dense) cudaFree(g->d_dense);
    g->d_len = nullptr; g->d_ell = nullptr; g->d_dense = nullptr;
    FG_CK(g, cudaMalloc(&g->d_len, len.size() * 4));
    FG_CK(g, cudaMalloc(&g->d_ell, ell.size() * sizeof(int2)));
    FG_CK(g, cudaMemcpy(g->d_len, len.data(), len.size() * 4, cudaMemcpyHostToDevice));
    FG_CK(g, cudaMemcpy(g->d_ell, ell.data(), ell.size() * sizeof(int2), cudaMemcpyHostToDevice));
    for (int s = 0; s < 3; ++s) {
        g->ell_base[s] = base[s];
        g->ell_rows[s] = rows_s[s];
    }
    g->C = C;
    g->fbar = fbar;
    g->have_factor = true;
    return BP_OK;
}

bp_status bp_fg_reset_messages(bp_factor_graph g) {
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_reset_messages: NULL graph");
    g->uniform_pending = true;
    return BP_OK;
}

static bp_status fg_prepare(bp_factor_graph g, int mode) {
    if (!g->have_unary || !g->have_factor) return fgfail(g, BP_ERR_STATE, "set the unary and the factor first");
    if ((mode == BP_MAX) != (g->dtype == BP_I32) || (mode != BP_SUM && mode != BP_MAX))
        return fgfail(g, BP_ERR_ARG, "BP_SUM needs BP_F32, BP_MAX needs BP_I32");
    if (g->uniform_pending && g->n_factors > 0) {
        const long long rows = 3LL * g->n_factors;
        if (g->dtype == BP_F32)
            fg_fill_kernel<float><<<bpg::grid_for(rows * g->Mp, 256), 256, 0, g->stream>>>((float *)g->m_fv, rows, g->M,
                                                                                          g->Mp, 1.0f / g->M);
        else
            fg_fill_kernel<int32_t><<<bpg::grid_for(rows * g->Mp, 256), 256, 0, g->stream>>>((int32_t *)g->m_fv, rows,
                                                                                            g->M, g->Mp, 0);
        FG_CK(g, cudaGetLastError());
        g->launches += 1;
    }
    g->uniform_pending = false;
    return BP_OK;
}

static bp_status fg_v2f(bp_factor_graph g) {
    const FgDims d{g->n_vars, g->n_factors, g->M, g->Mp};
    const int D = g->max_degree <= 4 ? 4 : g->max_degree <= 8 ? 8 : 16;
    if (g->dtype == BP_F32) {
        if (D == 4) launch_v2f<false, float, 4>(g, d);
        else if (D == 8) launch_v2f<false, float, 8>(g, d);
        else launch_v2f<false, float, 16>(g, d);
    } else {
        if (D == 4) launch_v2f<true, int32_t, 4>(g, d);
        else if (D == 8) launch_v2f<true, int32_t, 8>(g, d);
        else launch_v2f<true, int32_t, 16>(g, d);
    }
    FG_CK(g, cudaGetLastError());
    g->launches += 1;
    return BP_OK;
}

bp_status bp_fg_iterate(bp_factor_graph g, int n_iters, int mode) {
    BPG_TRACE("bp_fg_iterate");
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_iterate: NULL graph");
    g->err.clear();
    if (n_iters < 0) return fgfail(g, BP_ERR_ARG, "bp_fg_iterate: n_iters < 0");
    if (bp_status st = fg_prepare(g, mode)) return st;
    if (g->n_factors == 0) return BP_OK;
    const FgDims d{g->n_vars, g->n_factors, g->M, g->Mp};
    const FgTable tab{g->d_ell, g->d_len, {g->ell_base[0], g->ell_base[1], g->ell_base[2]},
                      {g->ell_rows[0], g->ell_rows[1], g->ell_rows[2]}};
    for (int it = 0; it < n_iters; ++it) {
        if (bp_status st = fg_v2f(g)) return st;
        const int km = f2v_chunks(g->Mp);   // the table was built for this many chunks
        cudaError_t e = g->dtype == BP_F32
            ? (km <= 1 ? launch_f2v<false, float, 1>(g, tab, d) : km <= 2 ? launch_f2v<false, float, 2>(g, tab, d)
               : km <= 4 ? launch_f2v<false, float, 4>(g, tab, d) : launch_f2v<false, float, 8>(g, tab, d))
            : (km <= 1 ? launch_f2v<true, int32_t, 1>(g, tab, d) : km <= 2 ? launch_f2v<true, int32_t, 2>(g, tab, d)
               : km <= 4 ? launch_f2v<true, int32_t, 4>(g, tab, d) : launch_f2v<true, int32_t, 8>(g, tab, d));
        FG_CK(g, e);
        g->launches += 1;
    }
    return BP_OK;
}

bp_status bp_fg_iterate_dense(bp_factor_graph g, int n_iters, int mode) {
    BPG_TRACE("bp_fg_iterate_dense");
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_iterate_dense: NULL graph");
    g->err.clear();
    if (n_iters < 0) return fgfail(g, BP_ERR_ARG, "bp_fg_iterate_dense: n_iters < 0");
    if (bp_status st = fg_prepare(g, mode)) return st;
    if (g->n_factors == 0) return BP_OK;
    const size_t M = g->M;
    if (!g->d_dense) {
        std::vector<float> Ff;
        std::vector<int32_t> Fi;
        if (g->dtype == BP_F32) Ff.assign(M * M * M, (float)g->fbar); else Fi.assign(M * M * M, (int32_t)g->fbar);
        for (int c = 0; c < g->C; ++c) {
            const size_t idx = ((size_t)g->trip[3 * c] * M + g->trip[3 * c + 1]) * M + g->trip[3 * c + 2];
            if (g->dtype == BP_F32) Ff[idx] = g->valf[c]; else Fi[idx] = g->vali[c];
        }
        FG_CK(g, cudaMalloc(&g->d_dense, M * M * M * 4));
        FG_CK(g, cudaMemcpy(g->d_dense, g->dtype == BP_F32 ? (const void *)Ff.data() : (const void *)Fi.data(),
                            M * M * M * 4, cudaMemcpyHostToDevice));
    }
    const FgDims d{g->n_vars, g->n_factors, g->M, g->Mp};
    for (int it = 0; it < n_iters; ++it) {
        if (bp_status st = fg_v2f(g)) return st;
        if (g->dtype == BP_F32)
            f2v_dense_kernel<false, float><<<warp_grid(g->n_factors), 256, 0, g->stream>>>(
                (const float *)g->n_vf, (float *)g->m_fv, (const float *)g->d_dense, d);
        else
            f2v_dense_kernel<true, int32_t><<<warp_grid(g->n_factors), 256, 0, g->stream>>>(
                (const int32_t *)g->n_vf, (int32_t *)g->m_fv, (const int32_t *)g->d_dense, d);
        FG_CK(g, cudaGetLastError());
        g->launches += 1;
    }
    return BP_OK;
}

bp_status bp_fg_beliefs(bp_factor_graph g, void *dev_out, int32_t *dev_map) {
    BPG_TRACE("bp_fg_beliefs");
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_beliefs: NULL graph");
    g->err.clear();
    if (!dev_out) return fgfail(g, BP_ERR_ARG, "bp_fg_beliefs: NULL output");
    if (bp_status st = fg_prepare(g, g->dtype == BP_F32 ? BP_SUM : BP_MAX)) return st;
    const FgDims d{g->n_vars, g->n_factors, g->M, g->Mp};
    if (g->dtype == BP_F32)
        fg_beliefs_kernel<false, float><<<warp_grid(g->n_vars), 256, 0, g->stream>>>(
            (const float *)g->unary, g->var_ptr, g->var_inc, (const float *)g->m_fv, d, (float *)dev_out, dev_map);
    else
        fg_beliefs_kernel<true, int32_t><<<warp_grid(g->n_vars), 256, 0, g->stream>>>(
            (const int32_t *)g->unary, g->var_ptr, g->var_inc, (const int32_t *)g->m_fv, d, (int32_t *)dev_out, dev_map);
    FG_CK(g, cudaGetLastError());
    g->launches += 1;
    return BP_OK;
}

bp_status bp_fg_get_messages(bp_factor_graph g, void *dev_out) {
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_get_messages: NULL graph");
    g->err.clear();
    if (!dev_out) return fgfail(g, BP_ERR_ARG, "bp_fg_get_messages: NULL output");
    if (g->n_factors == 0) return BP_OK;
    if (g->uniform_pending) return fgfail(g, BP_ERR_STATE, "bp_fg_get_messages: messages not materialised yet");
    FG_CK(g, bpg::launch_unpad_copy(g->m_fv, dev_out, 3LL * g->n_factors, g->M, g->Mp, g->stream));
    g->launches += 1;
    return BP_OK;
}

bp_status bp_fg_sync(bp_factor_graph g) {
    BPG_TRACE("bp_fg_sync");
    if (!g) return fgfail(nullptr, BP_ERR_ARG, "bp_fg_sync: NULL graph");
    FG_CK(g, cudaStreamSynchronize(g->stream));
    return BP_OK;
}

}  // extern "C"
