// Host-side schedule of a sparse-compatibility pattern for the register
// kernels (sparse_reg.cuh).
//
// The terms of the sum (or the minimum) over a receiver label's compatible
// sender labels can be taken in any order, and the receiver labels of a
// 32-label block can be given to the block's 32 lanes in any order (a store is
// still one 128-byte line).  Both freedoms go into shared-memory bank
// conflicts.  A 16-byte gather by the eight lanes of a quarter-warp costs one
// wavefront per distinct slot in the most-used 16-byte bank group.  Label x
// lives in slot (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7), bank group
// (x >> 2) & 7.
//
// 1. Partition: each block's labels are split into four quarter-warps of
//    eight so that every quarter-warp's entries spread evenly over the eight
//    bank groups.  A quarter-warp whose most-used group holds N entries needs
//    at least max(N, longest list) gathers.  The split minimises the sum and
//    the maximum of that bound by deterministic annealing over swaps.
// 2. Schedule: within a quarter-warp the entries form a bipartite multigraph,
//    lanes against bank groups.  A proper edge colouring with D colours, D its
//    largest degree, exists (Koenig's theorem).  It is found by the classical
//    alternating-path recolouring.  Colour c is step c: at every step each lane
//    takes at most one entry and each bank group serves at most one lane, one
//    wavefront.  Lanes whose list is shorter than D have holes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "bp_sparse.h"

namespace bpg {
namespace {

inline int reg_slot(int x) { return (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7); }
inline int reg_group(int x) { return (x >> 2) & 7; }

struct XorShift {
    uint64_t s;
    uint32_t next() {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return (uint32_t)(s >> 16);
    }
    double unit() { return (next() & 0xFFFFFF) / 16777216.0; }
};

// Edge colouring of a bipartite multigraph with lanes 0..7 on one side and
// bank groups 0..7 on the other; edge e joins lane el[e] and group eg[e].
// Returns the number of colours (the largest degree); col[e] is e's colour.
int colour_edges(const std::vector<int> &el, const std::vector<int> &eg, std::vector<int> &col) {
    const int E = (int)el.size();
    int degL[8] = {}, degG[8] = {};
    for (int e = 0; e < E; ++e) {
        ++degL[el[e]];
        ++degG[eg[e]];
    }
    int D = 0;
    for (int i = 0; i < 8; ++i) D = std::max(D, std::max(degL[i], degG[i]));
    col.assign(E, -1);
    if (D == 0) return 0;
    std::vector<int> atL(8 * D, -1), atG(8 * D, -1);   // edge holding colour c at a vertex
    for (int e = 0; e < E; ++e) {
        const int p = el[e], g = eg[e];
        int a = 0, b = 0;
        while (atL[p * D + a] >= 0) ++a;   // free at the lane (degree < D before e)
        while (atG[g * D + b] >= 0) ++b;   // free at the group
        if (atG[g * D + a] >= 0) {
            // the path from g alternating colours a, b never reaches p (a is
            // free at p); swapping a and b along it frees a at g
            std::vector<int> path;
            bool at_group = true;
            int v = g, c = a;
            for (;;) {
                const int f = at_group ? atG[v * D + c] : atL[v * D + c];
                if (f < 0) break;
                path.push_back(f);
                v = at_group ? el[f] : eg[f];
                at_group = !at_group;
                c = (c == a) ? b : a;
            }
            for (int f : path) {
                atL[el[f] * D + col[f]] = -1;
                atG[eg[f] * D + col[f]] = -1;
            }
            for (int f : path) {
                col[f] = (col[f] == a) ? b : a;
                atL[el[f] * D + col[f]] = f;
                atG[eg[f] * D + col[f]] = f;
            }
        }
        col[e] = a;
        atL[p * D + a] = e;
        atG[g * D + a] = e;
    }
    return D;
}

struct QuarterCost {
    int bound;      // max(largest group count, longest list)
    long long sq;   // sum of squared group counts (a tie-break toward even spreads)
};

QuarterCost quarter_cost(const std::vector<int> &pos, int q, int n, const std::vector<int> &len,
                         const std::vector<int> &hist) {
    int h[8] = {}, lmax = 0;
    for (int i = 8 * q; i < std::min(n, 8 * q + 8); ++i) {
        const int x = pos[i];
        lmax = std::max(lmax, len[x]);
        for (int g = 0; g < 8; ++g) h[g] += hist[x * 8 + g];
    }
    QuarterCost c{lmax, 0};
    for (int g = 0; g < 8; ++g) {
        c.bound = std::max(c.bound, h[g]);
        c.sq += (long long)h[g] * h[g];
    }
    return c;
}

// weight of one partition: the sum and the maximum of the quarter-warp bounds
// first (wavefronts and register steps), then the spread
long long partition_weight(const QuarterCost *qc, int nq) {
    long long sum = 0, mx = 0, sq = 0;
    for (int q = 0; q < nq; ++q) {
        sum += qc[q].bound;
        mx = std::max<long long>(mx, qc[q].bound);
        sq += qc[q].sq;
    }
    return ((2 * sum + mx) << 20) + sq;
}

}  // namespace

bool sparse_reg_plan(int M, int Mp, const int32_t *rowptr, const int32_t *cols, const int32_t *wbits,
                     SparseRegPlan *out) {
    if (Mp > 256 || Mp < 4) return false;
    const int KM = Mp <= 32 ? 1 : Mp / 32;
    int LMcap = 0;
    for (const auto &v : kSparseRegVariants)
        if (v[0] == KM) LMcap = std::max(LMcap, v[1]);
    if (LMcap == 0) return false;
    std::vector<int> len(Mp, 0), hist((size_t)Mp * 8, 0);
    for (int x = 0; x < M; ++x) {
        len[x] = rowptr[x + 1] - rowptr[x];
        if (len[x] > LMcap) return false;
        for (int p = rowptr[x]; p < rowptr[x + 1]; ++p) ++hist[(size_t)x * 8 + reg_group(cols[p])];
    }
    // ent[k][c][lane] with c < LMcap first; compacted to the chosen LM below
    std::vector<int32_t> ent((size_t)KM * LMcap * 32 * 2, 0);
    for (size_t i = 0; i < ent.size(); i += 2) ent[i] = (int32_t)0xFFFF;
    std::vector<int32_t> lab((size_t)KM * 32, -1);
    int steps = 0, wavefronts = 0;
    XorShift rng{0x9E3779B97F4A7C15ull};
    for (int k = 0; k < KM; ++k) {
        const int base = 32 * k, n = std::min(32, Mp - base);
        const int nq = (n + 7) / 8;
        std::vector<int> pos(n);
        for (int i = 0; i < n; ++i) pos[i] = base + i;
        // start from the labels dealt longest list first, round robin over the quarters
        std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) { return len[x] > len[y]; });
        std::vector<int> dealt(n);
        {
            int fill[4] = {0, 0, 0, 0}, q = 0;
            for (int i = 0; i < n; ++i) {
                while (fill[q] >= std::min(8, n - 8 * q)) q = (q + 1) % nq;
                dealt[8 * q + fill[q]++] = pos[i];
                q = (q + 1) % nq;
            }
        }
        pos = dealt;
        QuarterCost qc[4];
        for (int q = 0; q < nq; ++q) qc[q] = quarter_cost(pos, q, n, len, hist);
        if (nq > 1) {
            long long cur = partition_weight(qc, nq), best = cur;
            std::vector<int> best_pos = pos;
            double temp = 2.0 * (1 << 20);
            const int iters = 6000;
            for (int it = 0; it < iters; ++it) {
                const int qa = (int)(rng.next() % nq);
                int qb = (int)(rng.next() % (nq - 1));
                if (qb >= qa) ++qb;
                const int na = std::min(8, n - 8 * qa), nb = std::min(8, n - 8 * qb);
                const int ia = 8 * qa + (int)(rng.next() % na), ib = 8 * qb + (int)(rng.next() % nb);
                std::swap(pos[ia], pos[ib]);
                const QuarterCost ca = qc[qa], cb = qc[qb];
                qc[qa] = quarter_cost(pos, qa, n, len, hist);
                qc[qb] = quarter_cost(pos, qb, n, len, hist);
                const long long w = partition_weight(qc, nq);
                if (w <= cur || rng.unit() < std::exp((double)(cur - w) / temp)) {
                    cur = w;
                    if (cur < best) {
                        best = cur;
                        best_pos = pos;
                    }
                } else {
                    std::swap(pos[ia], pos[ib]);
                    qc[qa] = ca;
                    qc[qb] = cb;
                }
                temp = std::max(1.0, temp * 0.9985);
            }
            pos = best_pos;
        }
        for (int i = 0; i < n; ++i) lab[(size_t)k * 32 + i] = pos[i];
        for (int q = 0; q < nq; ++q) {
            std::vector<int> el, eg, idx;
            for (int i = 8 * q; i < std::min(n, 8 * q + 8); ++i) {
                const int x = pos[i];
                if (x >= M) continue;
                for (int p = rowptr[x]; p < rowptr[x + 1]; ++p) {
                    el.push_back(i - 8 * q);
                    eg.push_back(reg_group(cols[p]));
                    idx.push_back(p);
                }
            }
            std::vector<int> col;
            const int D = colour_edges(el, eg, col);
            if (D > LMcap) return false;
            steps = std::max(steps, D);
            wavefronts += D;
            for (size_t e = 0; e < idx.size(); ++e) {
                const int lane = 8 * q + el[e];
                const size_t o = (((size_t)k * LMcap + col[e]) * 32 + lane) * 2;
                ent[o] = reg_slot(cols[idx[e]]) * 16;
                ent[o + 1] = wbits[idx[e]];
            }
        }
    }
    int LM = 0;
    for (const auto &v : kSparseRegVariants)
        if (v[0] == KM && v[1] >= steps && LM == 0) LM = v[1];
    if (LM == 0) return false;
    out->KM = KM;
    out->LM = LM;
    out->steps = steps;
    out->wavefronts = wavefronts;
    out->lab = lab;
    out->ent.assign((size_t)KM * LM * 32 * 2, 0);
    for (int k = 0; k < KM; ++k)
        for (int c = 0; c < LM; ++c)
            for (int l = 0; l < 32; ++l) {
                const size_t d = (((size_t)k * LM + c) * 32 + l) * 2, s = (((size_t)k * LMcap + c) * 32 + l) * 2;
                out->ent[d] = ent[s];
                out->ent[d + 1] = ent[s + 1];
            }
    return true;
}

}  // namespace bpg
