// Launch interface of the sparse-compatibility kernels.  Internal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bp_internal.h"

namespace bpg {

// The pattern, interleaved by receiver label: entry i of x_j (the shared-
// memory slot of its sender label x_i, and the value bits) sits at
// ell[i * M + x_j], i < len[x_j].
//
// Slot of label x in the list kernels' per-warp h arrays: a rotation by
// x / 4 + x / 16 inside each group of four labels.  Lane l of a quarter-warp
// stores label 4l + j to bank group 4 (l & 1) + ((j + l + l / 4) & 3): eight
// different groups for the eight lanes.
inline int sp_label_slot(int x) { return (x & ~3) | ((x + (x >> 2) + (x >> 4)) & 3); }
struct SparseArgsF {
    const float *g;
    const float *in;
    float *out;
    GridDims d;
    int parity;
    const int32_t *len;      // device [M]: compatible sender labels per receiver label
    const int2 *ell;         // device [max len][M]: (slot of x_i, bits of f(x_i, x_j) - fbar)
    float fbar;
};

struct SparseArgsI {
    const int32_t *eu;
    const int32_t *in;
    int32_t *out;
    GridDims d;
    int parity;
    const int32_t *len;
    const int2 *ell;         // (slot of x_i, E(x_i, x_j))
    int32_t ebar;
};

cudaError_t launch_sparse_sum(const SparseArgsF &a, cudaStream_t s);
cudaError_t launch_sparse_min(const SparseArgsI &a, cudaStream_t s);

// ---- register-pattern kernels (sparse_reg.cuh) ----------------------------
// Lane l of 32-label receiver block k owns the receiver label lab[k][l] (-1:
// none) and, for each step c < LM, the entry ent[k][c][l] = (byte offset of
// the sender label's h slot, or 0xFFFF for a hole; bits of f - fbar, or E).
// The device copy of a schedule has no holes: a hole reads slot 0 (label 0,
// always a label) with the value 0.0f (sum: adds nothing) or kSparseHoleE
// (min-sum: E + h never goes below Ebar + min h, the flat term).
constexpr int32_t kSparseHoleE = 1 << 29;
// Largest Ebar of the 16-bit min-sum form: its operands stay in [0, 2 Ebar + 2].
constexpr int32_t kP16MaxEbar = 16382;

// How a launch walks its nodes: slots per row, and the grid stride in whole
// rows and remaining slots (set by the launcher).
struct SparseWalk {
    int row, dq, dr;
};

struct SparseRegArgs {
    const void *u;           // [H][W][Mp] g (float) or E_u (int32)
    const void *in;          // [4][H][W][Mp] incoming messages
    void *out;               // [4][H][W][Mp] updated messages
    GridDims d;
    int parity;
    const int2 *ent;         // device [KM][LM][32]
    const int32_t *lab;      // device [KM][32]
    float fbar;
    int32_t ebar;
    int *status;             // device error word: 301 when a bounded wait gave up
    SparseWalk walk;         // set by the launcher
};

// (KM, LM) pairs compiled: KM = 32-label receiver blocks (Mp <= 32 KM), LM =
// register steps per block; LM ascending for each KM.
constexpr int kSparseRegVariants[][2] = {{1, 16}, {1, 48}, {2, 8}, {2, 12}, {2, 24}, {4, 6},
                                          {4, 9},  {4, 12}, {8, 4}, {8, 6}};

struct SparseRegPlan {
    int KM = 0, LM = 0;
    int gather_bytes = 16;         // 16: FP32 / int32 slots; 8: the 16-bit min-sum form
    int steps = 0;                 // steps every lane runs per block (= LM)
    int wavefronts = 0;            // gather wavefronts per node (sum over blocks, lane sets, steps)
    std::vector<int32_t> ent;      // [KM][LM][32][2]
    std::vector<int32_t> lab;      // [KM][32]
};

// Schedules a pattern (CSR by receiver label; wbits = value bits per entry)
// for the register kernels with gathers of gather_bytes (16: quarter-warps,
// 8: half-warps); holes have offset 0xFFFF.  False when Mp > 256 or when a
// list is longer than the steps of every compiled variant (the list kernels
// serve it).
bool sparse_reg_plan(int M, int Mp, const int32_t *rowptr, const int32_t *cols, const int32_t *wbits,
                     int gather_bytes, SparseRegPlan *out);

enum class SparseRegMode { Sum, Min, Min16 };

// The entries as the kernel takes them: a hole reads a slot that another lane
// of its lane set reads at that step (no extra wavefront), or slot 0, with a
// value that changes nothing (0.0f; kSparseHoleE; Ebar + 1 in both halves of
// the 16-bit form, whose weights are E in both halves).
std::vector<int32_t> sparse_reg_device_entries(const SparseRegPlan &plan, SparseRegMode mode, int32_t ebar);

cudaError_t launch_sparse_reg_sum(const SparseRegArgs &a, int KM, int LM, cudaStream_t s);
cudaError_t launch_sparse_reg_min(const SparseRegArgs &a, int KM, int LM, cudaStream_t s);
cudaError_t launch_sparse_reg_min16(const SparseRegArgs &a, int KM, int LM, cudaStream_t s);

}  // namespace bpg
