// Host-side schedule of a sparse-compatibility pattern for the register
// kernels (sparse_reg.cuh).
//
// The terms of the sum (or the minimum) over a receiver label's compatible
// sender labels can be taken in any order, and the receiver labels of a
// 32-label block can be given to the block's 32 lanes in any order (a store is
// still one 128-byte line).  Both freedoms go into shared-memory bank
// conflicts.  A gather costs, per set of lanes served together, one wavefront
// per distinct slot in its most-used bank group (lanes that read the same slot
// share it): 16-byte slots are served to the eight lanes of a quarter-warp
// from eight 16-byte bank groups, 8-byte slots (the 16-bit min-sum form) to
// the sixteen lanes of a half-warp from sixteen 8-byte groups.
//
// 1. Partition: each block's labels are split into lane sets so that every
//    set's entries spread evenly over the bank groups (deterministic
//    annealing over swaps of two labels).
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

// How the kernel's h slice is gathered.  16-byte slots (four FP32 / int32 h
// per label): label x in slot (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7),
// bank group (x >> 2) & 7 of the 8 served per wavefront, for the eight lanes
// of a quarter-warp.  8-byte slots (four 16-bit h): slot
// (x & ~63) | ((x & 3) << 4) | ((x >> 2) & 15), bank group (x >> 2) & 15 of
// 16, for the sixteen lanes of a half-warp.  In both, the lanes of a set
// storing labels 4l + j in phase 1 hit distinct groups.
struct Shape {
    int set;          // lanes served together
    int groups;       // bank groups per wavefront
    int slot_bytes;
    int slot(int x) const {
        return slot_bytes == 16 ? (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7)
                                : (x & ~63) | ((x & 3) << 4) | ((x >> 2) & 15);
    }
    int group(int x) const { return (x >> 2) & (groups - 1); }
};

Shape shape_of(int gather_bytes) { return gather_bytes == 8 ? Shape{16, 16, 8} : Shape{8, 8, 16}; }

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

struct SetCost {
    int bound;      // max(largest group count, longest list)
    long long sq;   // sum of squared group counts (a tie-break toward even spreads)
};

// Lanes of a set that read the same sender label at the same step share
// one slot, so the bound counts distinct sender labels per bank group.
SetCost set_cost(const Shape &gs, const std::vector<int> &pos, int q, int n, const std::vector<int> &len,
                         const std::vector<std::vector<int>> &senders) {
    int h[16] = {}, lmax = 0;
    uint64_t seen[8] = {};   // sender labels < 512
    for (int i = gs.set * q; i < std::min(n, gs.set * q + gs.set); ++i) {
        const int x = pos[i];
        lmax = std::max(lmax, len[x]);
        for (int xi : senders[x]) {
            uint64_t &w = seen[xi >> 6];
            const uint64_t b = 1ull << (xi & 63);
            if (!(w & b)) {
                w |= b;
                ++h[gs.group(xi)];
            }
        }
    }
    SetCost c{lmax, 0};
    for (int g = 0; g < gs.groups; ++g) {
        c.bound = std::max(c.bound, h[g]);
        c.sq += (long long)h[g] * h[g];
    }
    return c;
}

long long partition_weight(const SetCost *qc, int nq) {
    long long sum = 0, sq = 0;
    for (int q = 0; q < nq; ++q) {
        sum += qc[q].bound;
        sq += qc[q].sq;
    }
    return (sum << 20) + sq;
}

// Split the n labels pos[] of one block into lane sets (positions S q ..
// S q + S - 1, S = 8 or 16) with evenly spread bank groups.
void partition_block(const Shape &gs, std::vector<int> &pos, const std::vector<int> &len,
                     const std::vector<std::vector<int>> &senders, XorShift &rng) {
    const int S = gs.set, n = (int)pos.size(), nq = (n + S - 1) / S;
    std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) { return len[x] > len[y]; });
    std::vector<int> dealt(n);
    int fill[4] = {0, 0, 0, 0}, q = 0;
    for (int i = 0; i < n; ++i) {   // longest lists first, round robin over the sets
        while (fill[q] >= std::min(S, n - S * q)) q = (q + 1) % nq;
        dealt[S * q + fill[q]++] = pos[i];
        q = (q + 1) % nq;
    }
    pos = dealt;
    if (nq < 2) return;
    SetCost qc[4];
    for (int j = 0; j < nq; ++j) qc[j] = set_cost(gs, pos, j, n, len, senders);
    long long cur = partition_weight(qc, nq), best = cur;
    std::vector<int> best_pos = pos;
    double temp = 2.0 * (1 << 20);
    for (int it = 0; it < 12000; ++it) {
        const int qa = (int)(rng.next() % nq);
        int qb = (int)(rng.next() % (nq - 1));
        if (qb >= qa) ++qb;
        const int ia = S * qa + (int)(rng.next() % std::min(S, n - S * qa));
        const int ib = S * qb + (int)(rng.next() % std::min(S, n - S * qb));
        std::swap(pos[ia], pos[ib]);
        const SetCost ca = qc[qa], cb = qc[qb];
        qc[qa] = set_cost(gs, pos, qa, n, len, senders);
        qc[qb] = set_cost(gs, pos, qb, n, len, senders);
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

// Wavefronts of one step of one lane set: distinct slots in its most-used
// bank group (at least one: hole lanes still issue the gather).
int step_cost(const Shape &gs, const std::vector<int> &sched, int nl, int LM, int c) {
    int slots[16], groups[16], m = 0;
    for (int l = 0; l < nl; ++l) {
        const int x = sched[l * LM + c];
        if (x < 0) continue;
        const int s = gs.slot(x);
        bool dup = false;
        for (int j = 0; j < m; ++j) dup = dup || slots[j] == s;
        if (!dup) {
            slots[m] = s;
            groups[m++] = gs.group(x);
        }
    }
    int cnt[16] = {}, best = 1;
    for (int j = 0; j < m; ++j) best = std::max(best, ++cnt[groups[j]]);
    return best;
}

// Place the entries (sender labels) of each lane of one lane set on
// distinct steps 0..LM-1; sched[l * LM + c] = sender label or -1 (hole).
// Returns the set's wavefronts per node.
int place_set(const Shape &gs, std::vector<int> &sched, const std::vector<std::vector<int>> &lists, int LM,
                  XorShift &rng) {
    const int nl = (int)lists.size();
    sched.assign((size_t)nl * LM, -1);
    for (int l = 0; l < nl; ++l)
        for (size_t i = 0; i < lists[l].size(); ++i) sched[l * LM + (int)i] = lists[l][i];
    std::vector<int> cost(LM);
    int cur = 0;
    for (int c = 0; c < LM; ++c) cur += (cost[c] = step_cost(gs, sched, nl, LM, c));
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
        const int ca = step_cost(gs, sched, nl, LM, a), cb = step_cost(gs, sched, nl, LM, b);
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
                     int gather_bytes, SparseRegPlan *out) {
    if (Mp > 256 || Mp < 4 || (gather_bytes != 16 && gather_bytes != 8)) return false;
    const Shape gs = shape_of(gather_bytes);
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
    out->gather_bytes = gather_bytes;
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
        partition_block(gs, pos, len, senders, rng);
        for (int i = 0; i < n; ++i) out->lab[(size_t)k * 32 + i] = pos[i];
        for (int q = 0; q < 32 / gs.set; ++q) {
            std::vector<std::vector<int>> lists, where;   // sender labels / CSR positions per lane
            for (int i = gs.set * q; i < std::min(n, gs.set * q + gs.set); ++i) {
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
            wavefronts += place_set(gs, sched, lists, LM, rng);
            for (int l = 0; l < (int)lists.size(); ++l)
                for (int c = 0; c < LM; ++c) {
                    const int xi = sched[l * LM + c];
                    if (xi < 0) continue;
                    // the CSR position of this sender label in the lane's row
                    int p = -1;
                    for (size_t j = 0; j < lists[l].size(); ++j)
                        if (lists[l][j] == xi) p = where[l][j];
                    const size_t o = (((size_t)k * LM + c) * 32 + gs.set * q + l) * 2;
                    out->ent[o] = gs.slot(xi) * gs.slot_bytes;
                    out->ent[o + 1] = wbits[p];
                }
        }
    }
    out->wavefronts = wavefronts;
    return true;
}

std::vector<int32_t> sparse_reg_device_entries(const SparseRegPlan &plan, SparseRegMode mode, int32_t ebar) {
    const int S = shape_of(plan.gather_bytes).set;
    std::vector<int32_t> ent = plan.ent;
    const int32_t hole = mode == SparseRegMode::Sum   ? 0   // the bits of 0.0f
                         : mode == SparseRegMode::Min ? kSparseHoleE
                                                      : (ebar + 1) | ((ebar + 1) << 16);
    for (int k = 0; k < plan.KM; ++k)
        for (int c = 0; c < plan.LM; ++c)
            for (int q = 0; q < 32 / S; ++q) {
                const size_t b = (((size_t)k * plan.LM + c) * 32 + S * q) * 2;
                int32_t share = 0;   // a slot another lane of the set reads at this step
                for (int l = 0; l < S; ++l)
                    if (ent[b + 2 * l] != 0xFFFF) {
                        share = ent[b + 2 * l];
                        break;
                    }
                for (int l = 0; l < S; ++l) {
                    if (ent[b + 2 * l] == 0xFFFF) {
                        ent[b + 2 * l] = share;
                        ent[b + 2 * l + 1] = hole;
                    } else if (mode == SparseRegMode::Min16) {
                        ent[b + 2 * l + 1] |= ent[b + 2 * l + 1] << 16;
                    }
                }
            }
    return ent;
}

}  // namespace bpg
