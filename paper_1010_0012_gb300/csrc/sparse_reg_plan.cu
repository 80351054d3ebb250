// Host-side schedule of a sparse-compatibility pattern for the register
// kernels (sparse_reg.cuh).
//
// The terms of the sum (or the minimum) over a receiver label's compatible
// sender labels can be taken in any order, and the receiver labels of a
// 32-label block can be given to the block's 32 lanes in any order (a store is
// still one 128-byte line).  Both freedoms go into shared-memory bank
// conflicts.  A 16-byte gather by the eight lanes of a quarter-warp costs one
// wavefront per distinct slot in its most-used 16-byte bank group (lanes that
// read the same slot share it).  Label x lives in slot
// (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7), bank group (x >> 2) & 7.
//
// 1. Partition: each block's labels are split into four quarter-warps of
//    eight so that every quarter-warp's entries spread evenly over the eight
//    bank groups (deterministic annealing over swaps of two labels).
// 2. Steps: the kernel runs LM steps per block, LM the smallest compiled step
//    count at least the longest list.  Each lane places its entries on
//    distinct steps (holes elsewhere); the placement minimises the sum over
//    steps of the step's wavefronts, again by deterministic annealing over
//    swaps of two steps of one lane.
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

struct QuarterCost {
    int bound;      // max(largest group count, longest list)
    long long sq;   // sum of squared group counts (a tie-break toward even spreads)
};

// Lanes of a quarter-warp that read the same sender label at the same step
// share one slot, so the bound counts distinct sender labels per bank group.
QuarterCost quarter_cost(const std::vector<int> &pos, int q, int n, const std::vector<int> &len,
                         const std::vector<std::vector<int>> &senders) {
    int h[8] = {}, lmax = 0;
    uint64_t seen[8] = {};   // sender labels < 512
    for (int i = 8 * q; i < std::min(n, 8 * q + 8); ++i) {
        const int x = pos[i];
        lmax = std::max(lmax, len[x]);
        for (int xi : senders[x]) {
            uint64_t &w = seen[xi >> 6];
            const uint64_t b = 1ull << (xi & 63);
            if (!(w & b)) {
                w |= b;
                ++h[reg_group(xi)];
            }
        }
    }
    QuarterCost c{lmax, 0};
    for (int g = 0; g < 8; ++g) {
        c.bound = std::max(c.bound, h[g]);
        c.sq += (long long)h[g] * h[g];
    }
    return c;
}

long long partition_weight(const QuarterCost *qc, int nq) {
    long long sum = 0, sq = 0;
    for (int q = 0; q < nq; ++q) {
        sum += qc[q].bound;
        sq += qc[q].sq;
    }
    return (sum << 20) + sq;
}

// Split the n labels pos[] of one block into quarter-warps (positions 8q ..
// 8q + 7) with evenly spread bank groups.
void partition_block(std::vector<int> &pos, const std::vector<int> &len,
                     const std::vector<std::vector<int>> &senders, XorShift &rng) {
    const int n = (int)pos.size(), nq = (n + 7) / 8;
    std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) { return len[x] > len[y]; });
    std::vector<int> dealt(n);
    int fill[4] = {0, 0, 0, 0}, q = 0;
    for (int i = 0; i < n; ++i) {   // longest lists first, round robin over the quarters
        while (fill[q] >= std::min(8, n - 8 * q)) q = (q + 1) % nq;
        dealt[8 * q + fill[q]++] = pos[i];
        q = (q + 1) % nq;
    }
    pos = dealt;
    if (nq < 2) return;
    QuarterCost qc[4];
    for (int j = 0; j < nq; ++j) qc[j] = quarter_cost(pos, j, n, len, senders);
    long long cur = partition_weight(qc, nq), best = cur;
    std::vector<int> best_pos = pos;
    double temp = 2.0 * (1 << 20);
    for (int it = 0; it < 12000; ++it) {
        const int qa = (int)(rng.next() % nq);
        int qb = (int)(rng.next() % (nq - 1));
        if (qb >= qa) ++qb;
        const int ia = 8 * qa + (int)(rng.next() % std::min(8, n - 8 * qa));
        const int ib = 8 * qb + (int)(rng.next() % std::min(8, n - 8 * qb));
        std::swap(pos[ia], pos[ib]);
        const QuarterCost ca = qc[qa], cb = qc[qb];
        qc[qa] = quarter_cost(pos, qa, n, len, senders);
        qc[qb] = quarter_cost(pos, qb, n, len, senders);
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

// Wavefronts of one step of one quarter-warp: distinct slots in its most-used
// bank group (at least one: hole lanes still issue the gather).
int step_cost(const std::vector<int> &sched, int nl, int LM, int c) {
    int slots[8], groups[8], m = 0;
    for (int l = 0; l < nl; ++l) {
        const int x = sched[l * LM + c];
        if (x < 0) continue;
        const int s = reg_slot(x);
        bool dup = false;
        for (int j = 0; j < m; ++j) dup = dup || slots[j] == s;
        if (!dup) {
            slots[m] = s;
            groups[m++] = reg_group(x);
        }
    }
    int cnt[8] = {}, best = 1;
    for (int j = 0; j < m; ++j) best = std::max(best, ++cnt[groups[j]]);
    return best;
}

// Place the entries (sender labels) of each lane of one quarter-warp on
// distinct steps 0..LM-1; sched[l * LM + c] = sender label or -1 (hole).
// Returns the quarter-warp's wavefronts per node.
int place_quarter(std::vector<int> &sched, const std::vector<std::vector<int>> &lists, int LM, XorShift &rng) {
    const int nl = (int)lists.size();
    sched.assign((size_t)nl * LM, -1);
    for (int l = 0; l < nl; ++l)
        for (size_t i = 0; i < lists[l].size(); ++i) sched[l * LM + (int)i] = lists[l][i];
    std::vector<int> cost(LM);
    int cur = 0;
    for (int c = 0; c < LM; ++c) cur += (cost[c] = step_cost(sched, nl, LM, c));
    if (nl == 0 || LM < 2) return cur;
    int best = cur;
    std::vector<int> best_sched = sched;
    double temp = 1.0;
    const int iters = 10000 * nl;
    for (int it = 0; it < iters && best > LM; ++it) {   // LM: one wavefront per step, the floor
        const int l = (int)(rng.next() % nl);
        const int a = (int)(rng.next() % LM);
        int b = (int)(rng.next() % (LM - 1));
        if (b >= a) ++b;
        if (sched[l * LM + a] < 0 && sched[l * LM + b] < 0) continue;
        std::swap(sched[l * LM + a], sched[l * LM + b]);
        const int ca = step_cost(sched, nl, LM, a), cb = step_cost(sched, nl, LM, b);
        const int next = cur - cost[a] - cost[b] + ca + cb;
        if (next <= cur || rng.unit() < std::exp((double)(cur - next) / temp)) {
            cur = next;
            cost[a] = ca;
            cost[b] = cb;
            if (cur < best) {
                best = cur;
                best_sched = sched;
            }
        } else {
            std::swap(sched[l * LM + a], sched[l * LM + b]);
        }
        temp = std::max(0.02, temp * 0.99993);
    }
    sched = best_sched;
    return best;
}

}  // namespace

bool sparse_reg_plan(int M, int Mp, const int32_t *rowptr, const int32_t *cols, const int32_t *wbits,
                     SparseRegPlan *out) {
    if (Mp > 256 || Mp < 4) return false;
    const int KM = Mp <= 32 ? 1 : Mp / 32;
    std::vector<int> len(Mp, 0);
    std::vector<std::vector<int>> senders(Mp);
    int lmax = 0;
    for (int x = 0; x < M; ++x) {
        len[x] = rowptr[x + 1] - rowptr[x];
        lmax = std::max(lmax, len[x]);
        senders[x].assign(cols + rowptr[x], cols + rowptr[x + 1]);
    }
    int LM = 0;
    for (const auto &v : kSparseRegVariants)
        if (v[0] == KM && v[1] >= lmax && LM == 0) LM = v[1];
    if (LM == 0) return false;
    out->KM = KM;
    out->LM = LM;
    out->steps = LM;
    out->lab.assign((size_t)KM * 32, -1);
    out->ent.assign((size_t)KM * LM * 32 * 2, 0);
    for (size_t i = 0; i < out->ent.size(); i += 2) out->ent[i] = 0xFFFF;
    int wavefronts = 0;
    XorShift rng{0x9E3779B97F4A7C15ull};
    for (int k = 0; k < KM; ++k) {
        const int base = 32 * k, n = std::min(32, Mp - base);
        std::vector<int> pos(n);
        for (int i = 0; i < n; ++i) pos[i] = base + i;
        partition_block(pos, len, senders, rng);
        for (int i = 0; i < n; ++i) out->lab[(size_t)k * 32 + i] = pos[i];
        for (int q = 0; q < 4; ++q) {
            std::vector<std::vector<int>> lists, where;   // sender labels / CSR positions per lane
            for (int i = 8 * q; i < std::min(n, 8 * q + 8); ++i) {
                lists.emplace_back();
                where.emplace_back();
                const int x = pos[i];
                if (x >= M) continue;
                for (int p = rowptr[x]; p < rowptr[x + 1]; ++p) {
                    lists.back().push_back(cols[p]);
                    where.back().push_back(p);
                }
            }
            std::vector<int> sched;
            wavefronts += place_quarter(sched, lists, LM, rng);
            for (int l = 0; l < (int)lists.size(); ++l)
                for (int c = 0; c < LM; ++c) {
                    const int xi = sched[l * LM + c];
                    if (xi < 0) continue;
                    // the CSR position of this sender label in the lane's row
                    int p = -1;
                    for (size_t j = 0; j < lists[l].size(); ++j)
                        if (lists[l][j] == xi) p = where[l][j];
                    const size_t o = (((size_t)k * LM + c) * 32 + 8 * q + l) * 2;
                    out->ent[o] = reg_slot(xi) * 16;
                    out->ent[o + 1] = wbits[p];
                }
        }
    }
    out->wavefronts = wavefronts;
    return true;
}

std::vector<int32_t> sparse_reg_device_entries(const SparseRegPlan &plan, bool min_sum) {
    std::vector<int32_t> ent = plan.ent;
    for (int k = 0; k < plan.KM; ++k)
        for (int c = 0; c < plan.LM; ++c)
            for (int q = 0; q < 4; ++q) {
                const size_t b = (((size_t)k * plan.LM + c) * 32 + 8 * q) * 2;
                int32_t share = 0;   // a slot another lane of the quarter reads at this step
                for (int l = 0; l < 8; ++l)
                    if (ent[b + 2 * l] != 0xFFFF) {
                        share = ent[b + 2 * l];
                        break;
                    }
                for (int l = 0; l < 8; ++l)
                    if (ent[b + 2 * l] == 0xFFFF) {
                        ent[b + 2 * l] = share;
                        ent[b + 2 * l + 1] = min_sum ? kSparseHoleE : 0;   // 0: the bits of 0.0f
                    }
            }
    return ent;
}

}  // namespace bpg
