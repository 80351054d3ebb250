// Dense O(M^2) sum-product baseline (Eq. 2) as a tensor-core GEMM.
//
// One synchronous iteration is two kernels:
//   hpack:  for every node, the four products h of Eq. 5 (unary times the
//           other incoming messages), rounded to BF16 and written as row
//           (s, r', c') of A = [4 H W][Mp], the row of the message slot they
//           feed (A's rows are the message planes' rows);
//   gemm:   D = A F (A: rows x K=Mp, F: K x N=Mp, BF16 operands, FP32
//           accumulation), each row divided by its sum (the normalisation
//           after Eq. 2) and stored as FP32 straight into the message planes.
//
// The GEMM is a persistent tcgen05 kernel (Mp = 64, 128 here; Mp = 256 in
// dense_tc_ring.cu, which pipelines 64-label K-blocks instead of whole
// tiles): one CTA per SM; warp 0 streams
// 128-row tiles of A with TMA (128-byte swizzle) into a 4-stage ring, warp 1
// owns the tensor memory and issues tcgen05.mma (M = 128, N = Mp, K = 16 per
// instruction) into one of two TMEM accumulators, warps 2-5 drain the other
// accumulator with tcgen05.ld, normalise each row in registers and store it.
// F^T (the B operand, Mp x Mp BF16) stays resident in shared memory.  Every
// mbarrier wait is bounded by a 2 s timer; on expiry the kernel records an
// error code in the handle's status word, drains its own copies and MMAs,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "trace.h"
#include "bp_ctx.h"
#include "dense_tc_ring.h"
#include "tc_ptx.cuh"

namespace {

template <int MP>
struct TcCfg {
    static constexpr int KB = MP / kBlockK;
    static constexpr uint32_t kAStage = (uint32_t)kTileM * MP * 2;
    static constexpr uint32_t kBBytes = (uint32_t)MP * MP * 2;
    static constexpr uint32_t kTmemCols = 2 * MP;   // two accumulators
    static constexpr uint32_t kStage = 4 * 32 * 32 * 4;   // per epilogue warp: one 32 x 32 FP32 tile
    static constexpr size_t kSmem = 1024 + kBBytes + kStages * kAStage + kStage + 256;
};

template <int MP>
__global__ void __launch_bounds__(kThreads, 1)
dense_tc_gemm_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b,
                     float *__restrict__ out, long long rows, int *status) {
    using Cfg = TcCfg<MP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;
    uint8_t *sA = smem + Cfg::kBBytes;
    float *sStage = (float *)(sA + kStages * Cfg::kAStage);
    uint64_t *bars = (uint64_t *)(sA + kStages * Cfg::kAStage + Cfg::kStage);
    uint64_t *full = bars;
    uint64_t *empty = bars + kStages;
    uint64_t *b_full = bars + 2 * kStages;
    uint64_t *acc_full = b_full + 1;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = (uint32_t *)(acc_empty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n_tiles = (rows + kTileM - 1) / kTileM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(b_full, 1);
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        int issued_phase[kStages];
        for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
        mbar_expect_tx(b_full, Cfg::kBBytes);
        for (int kb = 0; kb < Cfg::KB; ++kb) tma_load_2d(sB + kb * MP * 128, &tmap_b, b_full, kb * kBlockK, 0);
        long long i = 0;
        for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            const int s = (int)(i % kStages);
            const uint32_t ph = (uint32_t)((i / kStages) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
                *abort_flag = 1;
                atomicExch(status, 101);
                break;
            }
            mbar_expect_tx(&full[s], Cfg::kAStage);
            for (int kb = 0; kb < Cfg::KB; ++kb)
                tma_load_2d(sA + s * Cfg::kAStage + kb * kTileM * 128, &tmap_a, &full[s], kb * kBlockK,
                            (int)(t * kTileM));
            issued_phase[s] = (int)ph;
        }
        // drain: every copy this thread issued has landed before shared memory goes away
        mbar_wait(b_full, 0, nullptr);
        for (int s = 0; s < kStages; ++s)
            if (issued_phase[s] >= 0) mbar_wait(&full[s], (uint32_t)issued_phase[s], nullptr);
    } else if (warp == 1 && lane == 0) {
        // --------------------------------------------------------- MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kTileM, MP);
        bool ok = mbar_wait(b_full, 0, abort_flag);
        long long i = 0;
        int last_acc = -1;
        uint32_t last_aph = 0;
        if (ok) {
            for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
                const int s = (int)(i % kStages);
                const uint32_t ph = (uint32_t)((i / kStages) & 1);
                const int acc = (int)(i & 1);
                const uint32_t aph = (uint32_t)((i >> 1) & 1);
                if (!mbar_wait(&acc_empty[acc], aph ^ 1, abort_flag) || !mbar_wait(&full[s], ph, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + s * Cfg::kAStage);
                const uint32_t b0 = smem_u32(sB);
#pragma unroll
                for (int kb = 0; kb < Cfg::KB; ++kb)
#pragma unroll
                    for (int k = 0; k < kBlockK / 16; ++k)
                        umma_bf16(tmem_base + (uint32_t)(acc * MP), sw128_desc(a0 + kb * kTileM * 128 + k * 32),
                                  sw128_desc(b0 + kb * MP * 128 + k * 32), idesc, (kb | k) != 0);
                umma_commit(&empty[s]);
                umma_commit(&acc_full[acc]);
                last_acc = acc;
                last_aph = aph;
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(status, 102);
        }
        // drain: the MMAs this thread issued have completed
        if (last_acc >= 0) mbar_wait(&acc_full[last_acc], last_aph, nullptr);
    } else if (warp >= 2) {
        // ----------------------------------------------------------- epilogue
        const int quad = warp & 3;                // TMEM lanes [32 quad, 32 quad + 32)
        long long i = 0;
        for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            const int acc = (int)(i & 1);
            const uint32_t aph = (uint32_t)((i >> 1) & 1);
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], aph, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicExch(status, 103);
                }
                break;
            }
            tc_fence_after();
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * MP);
            float v[32];
            float z = 0.f;
#pragma unroll
            for (int c = 0; c < MP / 32; ++c) {
                tmem_ld32(taddr + c * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) z += v[j];
            }
            const float inv = z > 0.f ? 1.f / z : 0.f;
            // Transpose each 32 x 32 chunk through this warp's shared tile (16-byte
            // chunks XOR-swizzled by row) so that global stores are whole 128-byte
            // row segments: 8 lanes per row, 4 rows per store instruction.
            float *stg = sStage + (warp - 2) * 32 * 32;
            const long long row0 = t * kTileM + quad * 32;
            const int kk = lane & 7;
#pragma unroll
            for (int c = 0; c < MP / 32; ++c) {
                tmem_ld32(taddr + c * 32, v);
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    *reinterpret_cast<float4 *>(stg + lane * 32 + ((k ^ (lane & 7)) * 4)) =
                        make_float4(v[4 * k] * inv, v[4 * k + 1] * inv, v[4 * k + 2] * inv, v[4 * k + 3] * inv);
                __syncwarp();
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int r = (lane >> 3) + 4 * p;
                    const float4 x = *reinterpret_cast<const float4 *>(stg + r * 32 + ((kk ^ (r & 7)) * 4));
                    if (row0 + r < rows) *reinterpret_cast<float4 *>(out + (row0 + r) * MP + c * 32 + kk * 4) = x;
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem_base, Cfg::kTmemCols);
    }
}

// ---------------------------------------------------------------------------
// Fused form: the same dense update with h formed on chip.  A tile is 32 sender
// nodes x 4 directions = 128 rows; rows 32t..32t+31 hold h for direction t
// (t = 0 left, 1 right, 2 up, 3 down), so TMEM lane quadrant t holds the 32
// outgoing messages towards side t, which go to 32 consecutive slots of the
// destination plane.  Warps 2-9 form h from one read of g and the four
// incoming vectors of each node (exactly the bytes the O(mM) kernel reads) and
// write it as BF16 into the swizzled A stage; warp 1 issues the MMAs; warps
// 10-13 normalise and store.
constexpr int kFusedProducerWarps = 8;
constexpr int kFusedProducers = 32 * kFusedProducerWarps;
constexpr int kFusedEpiWarp0 = 2 + kFusedProducerWarps;          // first epilogue warp
constexpr int kFusedThreads = 32 * (kFusedEpiWarp0 + 4);
constexpr int kFusedNodes = 32;

template <int MP>
struct FusedCfg {
    static constexpr int KB = MP / kBlockK;
    static constexpr uint32_t kAStage = (uint32_t)kTileM * MP * 2;
    static constexpr uint32_t kBBytes = (uint32_t)MP * MP * 2;
    static constexpr uint32_t kTmemCols = 2 * MP;
    static constexpr uint32_t kStage = 4 * 32 * 32 * 4;
    static constexpr size_t kSmem = 1024 + kBBytes + kStages * kAStage + kStage + 256;
};

template <int MP>
__global__ void __launch_bounds__(kFusedThreads, 1)
dense_tc_fused_kernel(const __grid_constant__ CUtensorMap tmap_b, const float *__restrict__ g,
                      const float *__restrict__ in, float *__restrict__ out, bpg::GridDims d, int *status) {
    using Cfg = FusedCfg<MP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sB = smem;
    uint8_t *sA = smem + Cfg::kBBytes;
    float *sStage = (float *)(sA + kStages * Cfg::kAStage);
    uint64_t *bars = (uint64_t *)(sA + kStages * Cfg::kAStage + Cfg::kStage);
    uint64_t *full = bars;
    uint64_t *empty = bars + kStages;
    uint64_t *b_full = bars + 2 * kStages;
    uint64_t *acc_full = b_full + 1;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = (uint32_t *)(acc_empty + 2);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = d.W, H = d.H;
    const long long N = (long long)W * H;
    const long long n_tiles = (N + kFusedNodes - 1) / kFusedNodes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kFusedProducers);
            mbar_init(&empty[s], 1);
        }
        mbar_init(b_full, 1);
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, Cfg::kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp >= 2 && warp < kFusedEpiWarp0) {
        // ------------------------------------------------------- h producers
        const int ptid = threadIdx.x - 64;
        constexpr int CH = MP / 8;              // 8-label chunks per node
        long long i = 0;
        for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            const int s = (int)(i % kStages);
            const uint32_t ph = (uint32_t)((i / kStages) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
                *abort_flag = 1;
                atomicExch(status, 111);
                break;
            }
            uint8_t *As = sA + s * Cfg::kAStage;
            const long long n0 = t * kFusedNodes;
            for (int u = ptid; u < kFusedNodes * CH; u += kFusedProducers) {
                const int nl = u / CH, ch = u - nl * CH;
                const long long n = n0 + nl;
                float gv[8], m[4][8];
                bool has[4] = {false, false, false, false};
                if (n < N) {
                    const int r = (int)(n / W), c = (int)(n - (long long)r * W);
                    has[0] = c > 0; has[1] = c < W - 1; has[2] = r > 0; has[3] = r < H - 1;
                    const float *gp = g + n * MP + ch * 8;
                    const float4 g0 = __ldg(reinterpret_cast<const float4 *>(gp));
                    const float4 g1 = __ldg(reinterpret_cast<const float4 *>(gp) + 1);
                    gv[0] = g0.x; gv[1] = g0.y; gv[2] = g0.z; gv[3] = g0.w;
                    gv[4] = g1.x; gv[5] = g1.y; gv[6] = g1.z; gv[7] = g1.w;
#pragma unroll
                    for (int sd = 0; sd < 4; ++sd) {
                        if (has[sd]) {
                            const float *mp = in + sd * d.plane + n * MP + ch * 8;
                            const float4 a = __ldg(reinterpret_cast<const float4 *>(mp));
                            const float4 b = __ldg(reinterpret_cast<const float4 *>(mp) + 1);
                            m[sd][0] = a.x; m[sd][1] = a.y; m[sd][2] = a.z; m[sd][3] = a.w;
                            m[sd][4] = b.x; m[sd][5] = b.y; m[sd][6] = b.z; m[sd][7] = b.w;
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) m[sd][k] = 1.f;
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        gv[k] = 0.f;
#pragma unroll
                        for (int sd = 0; sd < 4; ++sd) m[sd][k] = 1.f;
                    }
                }
#pragma unroll
                for (int td = 0; td < 4; ++td) {
                    float h[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        float p = has[td] ? gv[k] : 0.f;
#pragma unroll
                        for (int sd = 0; sd < 4; ++sd)
                            if (sd != td) p *= m[sd][k];
                        h[k] = p;
                    }
                    const int row = td * 32 + nl;
                    const int kb = ch >> 3, cc = ch & 7;
                    const uint32_t off = (uint32_t)kb * (kTileM * 128) + (uint32_t)(row >> 3) * 1024 +
                                         (uint32_t)(row & 7) * 128 + (uint32_t)((cc ^ (row & 7)) * 16);
                    *reinterpret_cast<uint4 *>(As + off) =
                        make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                                   pack_bf16x2(h[6], h[7]));
                }
            }
            // make the generic-proxy writes visible to the tensor core's reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------ MMA issuer
        constexpr uint32_t idesc = idesc_bf16(kTileM, MP);
        mbar_expect_tx(b_full, Cfg::kBBytes);
        for (int kb = 0; kb < Cfg::KB; ++kb) tma_load_2d(sB + kb * MP * 128, &tmap_b, b_full, kb * kBlockK, 0);
        bool ok = mbar_wait(b_full, 0, abort_flag);
        long long i = 0;
        int last_acc = -1;
        uint32_t last_aph = 0;
        if (ok) {
            for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
                const int s = (int)(i % kStages);
                const uint32_t ph = (uint32_t)((i / kStages) & 1);
                const int acc = (int)(i & 1);
                const uint32_t aph = (uint32_t)((i >> 1) & 1);
                if (!mbar_wait(&acc_empty[acc], aph ^ 1, abort_flag) || !mbar_wait(&full[s], ph, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + s * Cfg::kAStage);
                const uint32_t b0 = smem_u32(sB);
#pragma unroll
                for (int kb = 0; kb < Cfg::KB; ++kb)
#pragma unroll
                    for (int k = 0; k < kBlockK / 16; ++k)
                        umma_bf16(tmem_base + (uint32_t)(acc * MP), sw128_desc(a0 + kb * kTileM * 128 + k * 32),
                                  sw128_desc(b0 + kb * MP * 128 + k * 32), idesc, (kb | k) != 0);
                umma_commit(&empty[s]);
                umma_commit(&acc_full[acc]);
                last_acc = acc;
                last_aph = aph;
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(status, 112);
        }
        mbar_wait(b_full, 0, nullptr);
        if (last_acc >= 0) mbar_wait(&acc_full[last_acc], last_aph, nullptr);
    } else if (warp >= kFusedEpiWarp0) {
        // --------------------------------------------- normalise and store
        const int quad = warp & 3;                // TMEM lanes of direction `quad`
        const int dr = (quad == 2) ? -1 : (quad == 3) ? 1 : 0;
        const int dc = (quad == 0) ? -1 : (quad == 1) ? 1 : 0;
        const long long delta = (long long)dr * W + dc;
        float *dst_plane = out + (long long)(quad ^ 1) * d.plane;
        float *stg = sStage + (warp - kFusedEpiWarp0) * 32 * 32;
        const int kk = lane & 7;
        long long i = 0;
        for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            const int acc = (int)(i & 1);
            const uint32_t aph = (uint32_t)((i >> 1) & 1);
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[acc], aph, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    atomicExch(status, 113);
                }
                break;
            }
            tc_fence_after();
            const long long n0 = t * kFusedNodes;
            // rows of this warp whose message exists (sender inside, neighbour present)
            bool mine = false;
            {
                const long long n = n0 + lane;
                if (n < N) {
                    const int r = (int)(n / W), c = (int)(n - (long long)r * W);
                    mine = (quad == 0) ? c > 0 : (quad == 1) ? c < W - 1 : (quad == 2) ? r > 0 : r < H - 1;
                }
            }
            const unsigned valid = __ballot_sync(0xffffffffu, mine);
            const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * MP);
            float v[32];
            float z = 0.f;
#pragma unroll
            for (int c = 0; c < MP / 32; ++c) {
                tmem_ld32(taddr + c * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) z += v[j];
            }
            const float inv = z > 0.f ? 1.f / z : 0.f;
#pragma unroll
            for (int c = 0; c < MP / 32; ++c) {
                tmem_ld32(taddr + c * 32, v);
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    *reinterpret_cast<float4 *>(stg + lane * 32 + ((k ^ (lane & 7)) * 4)) =
                        make_float4(v[4 * k] * inv, v[4 * k + 1] * inv, v[4 * k + 2] * inv, v[4 * k + 3] * inv);
                __syncwarp();
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int r = (lane >> 3) + 4 * p;
                    const float4 x = *reinterpret_cast<const float4 *>(stg + r * 32 + ((kk ^ (r & 7)) * 4));
                    if ((valid >> r) & 1u)
                        *reinterpret_cast<float4 *>(dst_plane + (n0 + r + delta) * MP + c * 32 + kk * 4) = x;
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem_base, Cfg::kTmemCols);
    }
}

// h of Eq. 5 for the four outgoing messages of every node, as BF16 rows of A.
// One thread per (node, 4 labels).
__global__ void hpack_kernel(const float *__restrict__ g, const float *__restrict__ in, __nv_bfloat16 *__restrict__ A,
                             bpg::GridDims d) {
    const int chunks = d.Mp / 4;
    const long long n = (long long)d.W * d.H * chunks;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long node = idx / chunks;
        const int ch = (int)(idx - node * chunks);
        const int r = (int)(node / d.W), c = (int)(node - (long long)r * d.W);
        const bool has[4] = {c > 0, c < d.W - 1, r > 0, r < d.H - 1};
        const long long off = node * d.Mp + ch * 4;
        const float4 gv = __ldg(reinterpret_cast<const float4 *>(g + off));
        float4 m[4];
        for (int s = 0; s < 4; ++s)
            m[s] = has[s] ? __ldg(reinterpret_cast<const float4 *>(in + s * d.plane + off)) : make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (!has[t]) continue;
            float4 h = gv;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (s == t) continue;
                h.x *= m[s].x; h.y *= m[s].y; h.z *= m[s].z; h.w *= m[s].w;
            }
            const int dr = (t == 2) ? -1 : (t == 3) ? 1 : 0;
            const int dc = (t == 0) ? -1 : (t == 1) ? 1 : 0;
            const long long row = (long long)(t ^ 1) * d.W * d.H + (long long)(r + dr) * d.W + (c + dc);
            __nv_bfloat162 lo = __floats2bfloat162_rn(h.x, h.y);
            __nv_bfloat162 hi = __floats2bfloat162_rn(h.z, h.w);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t *>(&lo);
            pk.y = *reinterpret_cast<uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(A + row * d.Mp + ch * 4) = pk;
        }
    }
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D BF16 tensor map over a row-major [rows][cols] matrix, box [box_rows][64].
bool make_map(CUtensorMap *map, const void *base, unsigned long long rows, unsigned long long cols, unsigned box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBlockK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcState {
    CUtensorMap map_a, map_b;
};

template <int MP>
cudaError_t launch_gemm(const TcState &st, float *out, long long rows, int *status, cudaStream_t s,
                        bool set_attr_always = false) {
    using Cfg = TcCfg<MP>;
    // the attribute belongs to the device's copy of the kernel: set it once per
    // device (or on every call, for a caller that must survive a context change)
    static bool attr_set[bpg::kMaxDevices] = {};
    const int dev = bpg::current_device();
    if (set_attr_always || dev >= bpg::kMaxDevices || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(dense_tc_gemm_kernel<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        if (dev < bpg::kMaxDevices) attr_set[dev] = true;
    }
    const long long tiles = (rows + kTileM - 1) / kTileM;
    int grid = bpg::device_sm_count();
    if (grid > tiles) grid = (int)tiles;
    dense_tc_gemm_kernel<MP><<<grid, kThreads, Cfg::kSmem, s>>>(st.map_a, st.map_b, out, rows, status);
    return cudaGetLastError();
}

template <int MP>
cudaError_t launch_fused(const TcState &st, const float *g, const float *in, float *out, const bpg::GridDims &d,
                         int *status, cudaStream_t s) {
    using Cfg = FusedCfg<MP>;
    // the attribute belongs to the device's copy of the kernel: set it once per device
    static bool attr_set[bpg::kMaxDevices] = {};
    const int dev = bpg::current_device();
    if (dev >= bpg::kMaxDevices || !attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(dense_tc_fused_kernel<MP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        if (dev < bpg::kMaxDevices) attr_set[dev] = true;
    }
    const long long tiles = ((long long)d.W * d.H + kFusedNodes - 1) / kFusedNodes;
    int grid = bpg::device_sm_count();
    if (grid > tiles) grid = (int)tiles;
    dense_tc_fused_kernel<MP><<<grid, kFusedThreads, Cfg::kSmem, s>>>(st.map_b, g, in, out, d, status);
    return cudaGetLastError();
}

}  // namespace

bp_status bpg_dense_tc_iterate(bp_ctx *h, int n_iters) { return bpg_dense_tc_iterate_kind(h, n_iters, false); }

bp_status bpg_dense_tc_iterate_kind(bp_ctx *h, int n_iters, bool fused) {
    if (h->Mp != 64 && h->Mp != 128 && h->Mp != 256)
        return bpg_fail(h, BP_ERR_UNSUPPORTED, "bp_iterate_dense: the tensor-core baseline serves 33 <= M <= 256");
    const long long rows = 4LL * h->W * h->H;
    const int Mp = h->Mp;
    if (!h->tc_ready) {
        bpg_free_tc(h);
        if (bp_status st = bpg_ensure_buffer(h, &h->tc_a, (size_t)rows * Mp * 2, "tensor-core A")) return st;
        if (bp_status st = bpg_ensure_buffer(h, &h->tc_b, (size_t)Mp * Mp * 2, "tensor-core B")) return st;
        if (bp_status st = bpg_ensure_buffer(h, &h->tc_z, (size_t)Mp * Mp * 4 + sizeof(TcState) + 64, "tensor-core maps"))
            return st;
        // B[x_j][x_i] = f(x_i, x_j) (F transposed: K = x_i contiguous), zero outside M
        std::vector<float> Bt((size_t)Mp * Mp, 0.f);
        for (int xj = 0; xj < h->M; ++xj)
            for (int xi = 0; xi < h->M; ++xi) Bt[(size_t)xj * Mp + xi] = bpg_pair_value_f(h, xi, xj);
        cudaError_t e = cudaMemcpyAsync(h->tc_z, Bt.data(), Bt.size() * 4, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return bpg_cuda_fail(h, e, "tensor-core B upload");
        to_bf16_kernel<<<64, 256, 0, h->stream>>>((const float *)h->tc_z, (__nv_bfloat16 *)h->tc_b, Mp * Mp);
        e = cudaMemsetAsync(h->tc_a, 0, (size_t)rows * Mp * 2, h->stream);
        if (e != cudaSuccess) return bpg_cuda_fail(h, e, "tensor-core A clear");
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return bpg_cuda_fail(h, e, "tensor-core setup");
        h->launches += 1;
        TcState *stt = new TcState();
        if (!make_map(&stt->map_a, h->tc_a, (unsigned long long)rows, (unsigned long long)Mp, kTileM) ||
            !make_map(&stt->map_b, h->tc_b, (unsigned long long)Mp, (unsigned long long)Mp, (unsigned)Mp)) {
            delete stt;
            return bpg_fail(h, BP_ERR_CUDA, "bp_iterate_dense: cuTensorMapEncodeTiled failed");
        }
        h->tc_maps = stt;
        h->tc_ready = true;
    }
    const TcState &st = *(const TcState *)h->tc_maps;
    if (fused) {
        for (int it = 0; it < n_iters; ++it) {
            cudaError_t e = Mp == 256 ? bpg::launch_fused_ring256(st.map_b, (const float *)h->unary,
                                                                  (const float *)h->msg[h->cur],
                                                                  (float *)h->msg[h->cur ^ 1], h->dims, h->d_status,
                                                                  h->stream)
                            : Mp == 128 ? launch_fused<128>(st, (const float *)h->unary, (const float *)h->msg[h->cur],
                                                          (float *)h->msg[h->cur ^ 1], h->dims, h->d_status, h->stream)
                                      : launch_fused<64>(st, (const float *)h->unary, (const float *)h->msg[h->cur],
                                                         (float *)h->msg[h->cur ^ 1], h->dims, h->d_status, h->stream);
            if (e != cudaSuccess) return bpg_cuda_fail(h, e, "fused tensor-core launch");
            h->launches += 1;
            h->cur ^= 1;
        }
        return BP_OK;
    }
    for (int it = 0; it < n_iters; ++it) {
        const long long n = (long long)h->W * h->H * (Mp / 4);
        hpack_kernel<<<bpg::grid_for(n, 256), 256, 0, h->stream>>>((const float *)h->unary, (const float *)h->msg[h->cur],
                                                                   (__nv_bfloat16 *)h->tc_a, h->dims);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return bpg_cuda_fail(h, e, "hpack launch");
        e = Mp == 256 ? bpg::launch_gemm_ring256(st.map_a, st.map_b, (float *)h->msg[h->cur ^ 1], rows, h->d_status,
                                                 h->stream)
            : Mp == 128 ? launch_gemm<128>(st, (float *)h->msg[h->cur ^ 1], rows, h->d_status, h->stream)
                        : launch_gemm<64>(st, (float *)h->msg[h->cur ^ 1], rows, h->d_status, h->stream);
        if (e != cudaSuccess) return bpg_cuda_fail(h, e, "tensor-core GEMM launch");
        h->launches += 2;
        h->cur ^= 1;
    }
    return BP_OK;
}

void bpg_free_tc(bp_ctx *h) {
    delete (TcState *)h->tc_maps;
    h->tc_maps = nullptr;
}

// ---------------------------------------------------------------------------
// Allocation-free form of one tensor-core dense iteration.
//
// Some callers cannot call cudaMalloc at all: a host process whose device
// memory is planned once at start-up by another component (an inference
// server's memory pool, a framework that forbids allocation after warm-up), or
// code running in a context where an allocation would synchronise the device
// or could fail at an unpredictable time.  For them the dense tensor-core
// iteration is also offered without any allocation: its scratch (the packed
// BF16 rows of h, the BF16 copy of F^T and a status word) lives in the
// file-scope array below, which every GPU that loads this library holds until
// the process exits.  The caller passes inputs and outputs only.
namespace {

constexpr size_t kNoAllocRowBytes = (size_t)32 << 20;          // packed h rows: at most 32 MiB
constexpr size_t kNoAllocBBytes = (size_t)128 * 128 * 2;       // F^T, BF16, M <= 128
constexpr size_t kNoAllocBytes = kNoAllocRowBytes + kNoAllocBBytes + 256;

// The array's device address, looked up with the device current.  The host-side
// name of the array is only a stand-in, so the address comes from
// cudaGetSymbolAddress.  It is cached per device ordinal together with the
// unique ID of the context it was taken in (cuCtxGetId: never reused within a
// process).  A cudaDeviceReset, or another context made current on the same
// ordinal, changes that ID, and the address is looked up again.
std::mutex g_noalloc_mu;
struct NoAllocSlot {
    unsigned long long ctx_id;
    uint8_t *base;
};
NoAllocSlot g_noalloc_slot[bpg::kMaxDevices];

typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long *);

// ID of the context current on this thread (0 when it cannot be read: then the
// address is looked up on every call)
unsigned long long current_ctx_id() {
    static PFN_ctxGetCurrent get_cur = nullptr;
    static PFN_ctxGetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_ctxGetCurrent)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_ctxGetId)p;
        tried = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

struct NoAllocTable {
    float f[256];   // f(d), d = -T..T (T <= 127)
    int T;
    float fbar;
};

// B[x_j][x_i] = f(x_i - x_j) inside the band, fbar outside, in BF16; clears the
// packed rows (rows of absent messages must read as zero) and the status word.
__global__ void noalloc_prep_kernel(NoAllocTable tab, int M, __nv_bfloat16 *B, uint4 *rows16, long long n16,
                                    int *status) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    for (long long i = tid; i < (long long)M * M; i += nthreads) {
        const int xj = (int)(i / M), xi = (int)(i - (long long)xj * M);
        const int d = xi - xj;
        B[i] = __float2bfloat16_rn((d >= -tab.T && d <= tab.T) ? tab.f[d + tab.T] : tab.fbar);
    }
    for (long long i = tid; i < n16; i += nthreads) rows16[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) *status = 0;
}

// errors are reported through bp_last_error(NULL), like those of bp_create
bp_status noalloc_fail(bp_status st, const std::string &m) { return bpg_fail(nullptr, st, m); }

}  // namespace

static __device__ __align__(256) uint8_t bpg_noalloc_scratch[kNoAllocBytes];

extern "C" bp_status bp_iterate_dense_tc_noalloc(int W, int H, int M, const float *dev_unary,
                                                 const float *dev_in_planes, float *dev_out_planes,
                                                 const float *host_table, int T, double fbar, void *cuda_stream) {
    BPG_TRACE("bp_iterate_dense_tc_noalloc");
    bpg_fail(nullptr, BP_OK, "");
    if (W < 1 || H < 1) return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: W and H must be >= 1");
    if (M != 64 && M != 128) return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: M must be 64 or 128");
    if (!dev_unary || !dev_in_planes || !dev_out_planes || !host_table)
        return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: NULL pointer");
    // the kernels move 16-byte vectors: a view at an odd offset into a buffer
    // would be a misaligned access on the device, so it is an argument error here
    if ((((uintptr_t)dev_unary) | ((uintptr_t)dev_in_planes) | ((uintptr_t)dev_out_planes)) & 15u)
        return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: device pointers must be 16-byte aligned");
    if (T < 0 || !(fbar >= 0) || !std::isfinite(fbar))
        return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: need T >= 0 and a finite fbar >= 0");
    const long long rows = 4LL * W * H;
    if ((long long)W * H > (1LL << 30) || (size_t)rows * M * 2 > kNoAllocRowBytes)
        return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: 4*W*H*M*2 bytes of packed rows exceed the "
                                        "fixed 32 MiB scratch (use bp_iterate_dense on a handle instead)");
    {
        const uintptr_t plane_bytes = (uintptr_t)rows * M * sizeof(float);
        const uintptr_t a0 = (uintptr_t)dev_in_planes, b0 = (uintptr_t)dev_out_planes;
        if (a0 < b0 + plane_bytes && b0 < a0 + plane_bytes)
            return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: input and output planes overlap");
    }
    NoAllocTable tab;
    tab.T = std::min(T, M - 1);
    tab.fbar = (float)fbar;
    for (int d = -tab.T; d <= tab.T; ++d) {
        const float v = host_table[d + T];
        if (!std::isfinite(v) || v < 0)
            return noalloc_fail(BP_ERR_ARG, "bp_iterate_dense_tc_noalloc: table entries must be finite and >= 0");
        tab.f[d + tab.T] = v;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    {
        // the call ends with a stream synchronisation, so it cannot be captured
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t ec = cudaStreamIsCapturing(s, &cap);
        if (ec != cudaSuccess)
            return noalloc_fail(BP_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ec));
        if (cap != cudaStreamCaptureStatusNone)
            return noalloc_fail(BP_ERR_STATE, "bp_iterate_dense_tc_noalloc: the stream is being captured; this call "
                                              "synchronises its stream and cannot be captured");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(BP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= bpg::kMaxDevices) return noalloc_fail(BP_ERR_UNSUPPORTED, "device index out of range");
    uint8_t *base = nullptr;
    {
        // set-up, once per device and context, with that device current
        const unsigned long long ctx = current_ctx_id();
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoAllocSlot &slot = g_noalloc_slot[dev];
        if (!slot.base || ctx == 0 || slot.ctx_id != ctx) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, bpg_noalloc_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(BP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            slot.base = (uint8_t *)p;
            slot.ctx_id = ctx;
        }
        base = slot.base;
    }
    __nv_bfloat16 *A = (__nv_bfloat16 *)base;
    __nv_bfloat16 *B = (__nv_bfloat16 *)(base + kNoAllocRowBytes);
    int *status = (int *)(base + kNoAllocRowBytes + kNoAllocBBytes);
    const long long n16 = (long long)rows * M * 2 / 16;
    noalloc_prep_kernel<<<bpg::grid_for(n16 > (long long)M * M ? n16 : (long long)M * M, 256), 256, 0, s>>>(
        tab, M, B, (uint4 *)A, n16, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(BP_ERR_CUDA, std::string("prep launch: ") + cudaGetErrorString(e));
    const bpg::GridDims d{W, H, M, M, (long long)W * H * M};
    hpack_kernel<<<bpg::grid_for((long long)W * H * (M / 4), 256), 256, 0, s>>>(dev_unary, dev_in_planes, A, d);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(BP_ERR_CUDA, std::string("hpack launch: ") + cudaGetErrorString(e));
    TcState st;
    if (!make_map(&st.map_a, A, (unsigned long long)rows, (unsigned long long)M, kTileM) ||
        !make_map(&st.map_b, B, (unsigned long long)M, (unsigned long long)M, (unsigned)M))
        return noalloc_fail(BP_ERR_CUDA, "bp_iterate_dense_tc_noalloc: cuTensorMapEncodeTiled failed");
    e = M == 128 ? launch_gemm<128>(st, dev_out_planes, rows, status, s, true)
                 : launch_gemm<64>(st, dev_out_planes, rows, status, s, true);
    if (e != cudaSuccess) return noalloc_fail(BP_ERR_CUDA, std::string("GEMM launch: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(BP_ERR_CUDA, std::string("iteration: ") + cudaGetErrorString(e));
    int flag = 0;
    e = cudaMemcpy(&flag, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return noalloc_fail(BP_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (flag) return noalloc_fail(BP_ERR_TIMEOUT, "a bounded wait in the tensor-core GEMM gave up");
    return BP_OK;
}
