// Internal host-side interface between the C-ABI layer (bp_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bpg {

// Largest band half-width served by the register/shuffle kernels; wider bands
// use the shared-memory kernels.
constexpr int kTMaxFast = 8;
constexpr int kBlock = 256;   // threads per block of the O(mM) kernels

// Message planes and unaries are stored with the label count padded to Mp,
// a multiple of 4 (16-byte vectors); padded labels hold 0 and are masked.
struct GridDims {
    int W, H, M, Mp;
    long long plane;   // H * W * Mp elements per plane
};

// Arguments of one launch of an O(mM) update over a set of nodes.
//   parity < 0: every node (synchronous iteration, in != out);
//   parity 0/1: nodes with (r + c) % 2 == parity (red-black half-step, in == out).
struct BandArgsF {
    const float *g;    // [H][W][Mp] unary (linear, or log g in log mode)
    const float *in;   // [4][H][W][Mp] incoming messages
    float *out;        // [4][H][W][Mp] updated messages
    GridDims d;
    int parity;
    int T;
    float w[2 * kTMaxFast + 1];  // f(d) - fbar, d = -T..T
    float fbar;
};

// The log-domain kernel's arguments: those of the linear one and, nullable,
// the per-message output [H][W][4] of the forward's scale C = A + log2 Z
// (A the max shift, Z the normaliser) and S / Z, which the adjoint reads
// instead of recomputing them.  (A type of its own, so that the linear
// kernel's parameters stay as they are.)
struct BandArgsLogF : BandArgsF {
    float2 *stats;
};

struct BandArgsI {
    const int32_t *e;  // [H][W][Mp] unary energies
    const int32_t *in;
    int32_t *out;
    GridDims d;
    int parity;
    int T;
    int32_t w[2 * kTMaxFast + 1];  // E(d), d = -T..T
    int32_t ebar;
    int zero_min;                  // 1 if E(0) is the table's minimum
    int packed16;                  // 1: Ebar - min E(d) <= 16000, the band runs on 16-bit label pairs
};

// Shared-memory O(mM) kernels for any T (table on the device).
struct BandArgsGenericF {
    const float *g;
    const float *in;
    float *out;
    GridDims d;
    int parity;
    int T;
    const float *w;    // device [2T + 1], f(d) - fbar
    float fbar;
};

struct BandArgsGenericI {
    const int32_t *e;
    const int32_t *in;
    int32_t *out;
    GridDims d;
    int parity;
    int T;
    const int32_t *w;  // device [2T + 1], E(d)
    int32_t ebar;
};

// Dense O(M^2) CUDA-core baseline (Eq. 2 / Eq. 9), synchronous.
struct DenseArgsF {
    const float *g;
    const float *in;
    float *out;
    GridDims d;
    const float *F;    // device [M][M], F[x_i * M + x_j]
};

struct DenseArgsI {
    const int32_t *e;
    const int32_t *in;
    int32_t *out;
    GridDims d;
    const int32_t *V;  // device [M][M]
};

// A (lanes per node, 4-label chunks per lane) layout of the fast kernels.
struct Layout {
    int L, C;
};

// Layouts compiled for a padded label count Mp (the first is the default).
int layouts_for(int Mp, Layout *out, int max_out);
int padded_labels(int M);   // Mp for a label count M

// Launchers return cudaSuccess or the launch error.  `blocks` <= 0 picks a
// persistent grid (SM count x resident blocks per SM).
cudaError_t launch_band_sum(const BandArgsF &a, Layout lay, int blocks, cudaStream_t s);
cudaError_t launch_band_min(const BandArgsI &a, Layout lay, int blocks, cudaStream_t s);
cudaError_t launch_band_log(const BandArgsLogF &a, Layout lay, int blocks, cudaStream_t s);
bool band_fast_available(int Mp, Layout lay, int T);

cudaError_t launch_band_sum_generic(const BandArgsGenericF &a, cudaStream_t s);
cudaError_t launch_band_min_generic(const BandArgsGenericI &a, cudaStream_t s);

cudaError_t launch_dense_sum(const DenseArgsF &a, cudaStream_t s);
cudaError_t launch_dense_min(const DenseArgsI &a, cudaStream_t s);

// Stereo unary from the image pair (unary_stereo.cu): out[node][x] =
// table[min(|R - L(c + x)|, Tu)] (Tu where c + x >= W), 0 on padded labels.
constexpr int kMaxStereoCost = 255;
cudaError_t launch_unary_stereo_f32(const uint8_t *left, const uint8_t *right, float *out, int W, int H, int M,
                                    int Mp, int Tu, const float *host_table, cudaStream_t s);
cudaError_t launch_unary_stereo_i32(const uint8_t *left, const uint8_t *right, int32_t *out, int W, int H, int M,
                                    int Mp, int Tu, const int32_t *host_table, cudaStream_t s);

// Utility kernels (aux_kernels.cu).
// transform: 0 copy, 1 log, 2 exp, 3 natural log -> base-2 log
cudaError_t launch_pad_copy_f32(const float *src, float *dst, long long nodes, int M, int Mp,
                                int transform, cudaStream_t s);
// natural log g -> padded base-2 log g and padded g, in one pass
cudaError_t launch_log_unary(const float *src, float *dst_log2, float *dst_lin, long long nodes, int M, int Mp,
                             cudaStream_t s);
cudaError_t launch_pad_copy_i32(const int32_t *src, int32_t *dst, long long nodes, int M, int Mp,
                                cudaStream_t s);
cudaError_t launch_unpad_copy(const void *src, void *dst, long long rows, int M, int Mp,
                              cudaStream_t s);   // 4-byte elements
// message planes out: slots without a neighbour as 0; exp2_log: base-2 log state to linear
cudaError_t launch_unpad_messages(const void *src, void *dst, int W, int H, int M, int Mp, int exp2_log,
                                  cudaStream_t s);
cudaError_t launch_fill_messages_f32(float *planes, long long nodes4, int M, int Mp, float value,
                                     cudaStream_t s);
cudaError_t launch_fill_messages_i32(int32_t *planes, long long nodes4, int M, int Mp,
                                     int32_t value, cudaStream_t s);
cudaError_t launch_beliefs_f32(const float *g, const float *planes, GridDims d, int log_domain,
                               float *out, int32_t *map, cudaStream_t s);
cudaError_t launch_beliefs_i32(const int32_t *e, const int32_t *planes, GridDims d, int32_t *out,
                               int32_t *map, cudaStream_t s);

constexpr int kMaxDevices = 64;   // per-device caches are indexed by ordinal below this
int device_sm_count();           // SMs of the current device (cached per device)
int current_device();            // cudaGetDevice, 0 on error
int grid_for(long long n, int block);   // blocks for a grid-stride elementwise kernel

}  // namespace bpg
