// Dense O(M^2) sum-product baseline (Eq. 2) on the tensor cores for Mp = 256.
//
// The same persistent tcgen05 kernels as dense_tc.cu (packed: TMA-streamed
// BF16 h rows; fused: h formed on chip), with one change of shape.  At 256
// labels, F^T (the resident B operand) is 128 KB and one 128-row A tile is
// 64 KB, so the ring of whole A tiles that serves 64 and 128 labels does not
// fit in 227 KB.  The pipeline unit is instead one 64-label K-block of a tile
// (128 rows x 128 bytes, 16 KB), in a ring of five.  The MMA issuer runs four
// tcgen05.mma (M = 128, N = 256, K = 16) per K-block into one of two
// 256-column TMEM accumulators (all 512 columns), and commits each K-block's
// stage back to its producer.  The epilogue is unchanged: tcgen05.ld of a
// row's 256 sums, the row's total, normalised stores through a swizzled
// per-warp tile.  Every mbarrier wait is bounded (2 s); on expiry the kernel
// records an error code in the status word, drains its copies and MMAs,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dense_tc_ring.h"
#include "tc_ptx.cuh"

namespace {

constexpr int kRingMP = 256;
constexpr int kRingKB = kRingMP / kBlockK;                     // K-blocks per tile
constexpr int kRingStages = 5;
constexpr uint32_t kKStage = (uint32_t)kTileM * 128;           // one K-block of A: 16 KB
constexpr uint32_t kRingB = (uint32_t)kRingMP * kRingMP * 2;   // F^T, BF16: 128 KB
constexpr uint32_t kRingTmemCols = 2 * kRingMP;                // two accumulators
constexpr uint32_t kRingEpi = 4 * 32 * 32 * 4;                 // four 32 x 32 FP32 epilogue tiles
constexpr size_t kRingSmem = 1024 + kRingB + kRingStages * kKStage + kRingEpi + 256;
static_assert(kRingSmem <= 232448, "shared memory of the Mp = 256 ring");

constexpr int kRingProducerWarps = 8;   // fused form: h producers
constexpr int kRingProducers = 32 * kRingProducerWarps;
constexpr int kRingEpiWarp0 = 2 + kRingProducerWarps;
constexpr int kRingFusedThreads = 32 * (kRingEpiWarp0 + 4);
constexpr int kRingNodes = 32;          // fused form: sender nodes per tile (4 directions = 128 rows)

struct RingSmem {
    uint8_t *B, *A;
    float *epi;
    uint64_t *full, *empty, *b_full, *acc_full, *acc_empty;
    uint32_t *tmem_slot;
    volatile int *abort_flag;
};

__device__ __forceinline__ RingSmem ring_smem(uint8_t *raw) {
    RingSmem m;
    uint8_t *base = (uint8_t *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    m.B = base;
    m.A = base + kRingB;
    m.epi = (float *)(m.A + kRingStages * kKStage);
    uint64_t *bars = (uint64_t *)((uint8_t *)m.epi + kRingEpi);
    m.full = bars;
    m.empty = bars + kRingStages;
    m.b_full = bars + 2 * kRingStages;
    m.acc_full = m.b_full + 1;
    m.acc_empty = m.acc_full + 2;
    m.tmem_slot = (uint32_t *)(m.acc_empty + 2);
    m.abort_flag = (volatile int *)(m.tmem_slot + 1);
    return m;
}

__device__ __forceinline__ void ring_init(const RingSmem &m, uint32_t full_count) {
    for (int s = 0; s < kRingStages; ++s) {
        mbar_init(&m.full[s], full_count);
        mbar_init(&m.empty[s], 1);
    }
    mbar_init(m.b_full, 1);
    for (int a = 0; a < 2; ++a) {
        mbar_init(&m.acc_full[a], 1);
        mbar_init(&m.acc_empty[a], 4);
    }
    *m.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// MMA issuer of both forms (one thread): per tile, wait for a free
// accumulator, then per K-block for its stage; four MMAs per K-block.
// Returns false on a time-out; *last_acc / *last_aph: the last committed tile.
__device__ __forceinline__ bool ring_mma(const RingSmem &m, uint32_t tmem_base, long long n_tiles, int &last_acc,
                                         uint32_t &last_aph) {
    constexpr uint32_t idesc = idesc_bf16(kTileM, kRingMP);
    if (!mbar_wait(m.b_full, 0, m.abort_flag)) return false;
    long long i = 0, j = 0;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
        const int acc = (int)(j & 1);
        const uint32_t aph = (uint32_t)((j >> 1) & 1);
        if (!mbar_wait(&m.acc_empty[acc], aph ^ 1, m.abort_flag)) return false;
        for (int kb = 0; kb < kRingKB; ++kb, ++i) {
            const int s = (int)(i % kRingStages);
            const uint32_t ph = (uint32_t)((i / kRingStages) & 1);
            if (!mbar_wait(&m.full[s], ph, m.abort_flag)) return false;
            tc_fence_after();
            const uint32_t a0 = smem_u32(m.A + s * kKStage);
            const uint32_t b0 = smem_u32(m.B + kb * kRingMP * 128);
#pragma unroll
            for (int k = 0; k < kBlockK / 16; ++k)
                umma_bf16(tmem_base + (uint32_t)(acc * kRingMP), sw128_desc(a0 + k * 32), sw128_desc(b0 + k * 32),
                          idesc, (kb | k) != 0);
            umma_commit(&m.empty[s]);
        }
        umma_commit(&m.acc_full[acc]);
        last_acc = acc;
        last_aph = aph;
    }
    return true;
}

// Epilogue warp (one of four; quad = its TMEM lane quadrant) for one tile
// held in accumulator acc: each of its 32 rows divided by the row's total,
// written as whole 128-byte row segments through the warp's swizzled tile.
// dst(r) is the destination of row r (or nullptr to skip it).
template <typename Dst>
__device__ __forceinline__ void ring_store_tile(uint32_t taddr, float *stg, int lane, Dst dst) {
    float v[32];
    float z = 0.f;
#pragma unroll
    for (int c = 0; c < kRingMP / 32; ++c) {
        tmem_ld32(taddr + c * 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) z += v[j];
    }
    const float inv = z > 0.f ? 1.f / z : 0.f;
    const int kk = lane & 7;
#pragma unroll
    for (int c = 0; c < kRingMP / 32; ++c) {
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
            float *o = dst(r);
            if (o) *reinterpret_cast<float4 *>(o + c * 32 + kk * 4) = x;
        }
        __syncwarp();
    }
}

// ---- packed form: warp 0 streams A's K-blocks by TMA, warp 1 issues the
// MMAs, warps 2-5 normalise and store ------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
dense_tc_gemm_ring_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b,
                          float *__restrict__ out, long long rows, int *status) {
    extern __shared__ uint8_t smem_raw[];
    const RingSmem m = ring_smem(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n_tiles = (rows + kTileM - 1) / kTileM;
    if (threadIdx.x == 0) ring_init(m, 1);
    if (warp == 1) tmem_alloc(m.tmem_slot, kRingTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *m.tmem_slot;

    if (warp == 0 && lane == 0) {
        int issued_phase[kRingStages];
        for (int s = 0; s < kRingStages; ++s) issued_phase[s] = -1;
        mbar_expect_tx(m.b_full, kRingB);
        for (int kb = 0; kb < kRingKB; ++kb) tma_load_2d(m.B + kb * kRingMP * 128, &tmap_b, m.b_full, kb * kBlockK, 0);
        long long i = 0;
        bool ok = true;
        for (long long t = blockIdx.x; ok && t < n_tiles; t += gridDim.x)
            for (int kb = 0; kb < kRingKB; ++kb, ++i) {
                const int s = (int)(i % kRingStages);
                const uint32_t ph = (uint32_t)((i / kRingStages) & 1);
                if (!mbar_wait(&m.empty[s], ph ^ 1, m.abort_flag)) {
                    *m.abort_flag = 1;
                    atomicExch(status, 121);
                    ok = false;
                    break;
                }
                mbar_expect_tx(&m.full[s], kKStage);
                tma_load_2d(m.A + s * kKStage, &tmap_a, &m.full[s], kb * kBlockK, (int)(t * kTileM));
                issued_phase[s] = (int)ph;
            }
        // drain: every copy this thread issued has landed before shared memory goes away
        mbar_wait(m.b_full, 0, nullptr);
        for (int s = 0; s < kRingStages; ++s)
            if (issued_phase[s] >= 0) mbar_wait(&m.full[s], (uint32_t)issued_phase[s], nullptr);
    } else if (warp == 1 && lane == 0) {
        int last_acc = -1;
        uint32_t last_aph = 0;
        if (!ring_mma(m, tmem_base, n_tiles, last_acc, last_aph)) {
            *m.abort_flag = 1;
            atomicExch(status, 122);
        }
        if (last_acc >= 0) mbar_wait(&m.acc_full[last_acc], last_aph, nullptr);
    } else if (warp >= 2) {
        const int quad = warp & 3;
        float *stg = m.epi + (warp - 2) * 32 * 32;
        long long j = 0;
        for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
            const int acc = (int)(j & 1);
            const uint32_t aph = (uint32_t)((j >> 1) & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&m.acc_full[acc], aph, m.abort_flag))) {
                if (lane == 0) {
                    *m.abort_flag = 1;
                    atomicExch(status, 123);
                }
                break;
            }
            tc_fence_after();
            const long long row0 = t * kTileM + quad * 32;
            ring_store_tile(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * kRingMP), stg, lane,
                            [&](int r) -> float * { return row0 + r < rows ? out + (row0 + r) * kRingMP : nullptr; });
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&m.acc_empty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem_base, kRingTmemCols);
    }
}

// ---- fused form: 32 sender nodes x 4 directions = 128 rows per tile (rows
// 32 t .. 32 t + 31: direction t); warps 2-9 form h of one K-block (64 labels)
// from g and the incoming vectors, as BF16 into the swizzled stage; warp 1
// loads F^T and issues the MMAs; warps 10-13 normalise and store the 32
// messages towards side `quad` into 32 consecutive slots of its plane -----------
__global__ void __launch_bounds__(kRingFusedThreads, 1)
dense_tc_fused_ring_kernel(const __grid_constant__ CUtensorMap tmap_b, const float *__restrict__ g,
                           const float *__restrict__ in, float *__restrict__ out, bpg::GridDims d, int *status) {
    extern __shared__ uint8_t smem_raw[];
    const RingSmem m = ring_smem(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = d.W, H = d.H;
    const long long N = (long long)W * H;
    const long long n_tiles = (N + kRingNodes - 1) / kRingNodes;
    if (threadIdx.x == 0) ring_init(m, kRingProducers);
    if (warp == 1) tmem_alloc(m.tmem_slot, kRingTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *m.tmem_slot;

    if (warp >= 2 && warp < kRingEpiWarp0) {
        // unit of a producer thread: node nl of the tile, labels kb * 64 + cc * 8 .. + 8
        const int ptid = threadIdx.x - 64;
        const int nl = ptid >> 3, cc = ptid & 7;
        long long i = 0;
        bool ok = true;
        for (long long t = blockIdx.x; ok && t < n_tiles; t += gridDim.x) {
            const long long n = t * kRingNodes + nl;
            bool has[4] = {false, false, false, false};
            if (n < N) {
                const int r = (int)(n / W), c = (int)(n - (long long)r * W);
                has[0] = c > 0;
                has[1] = c < W - 1;
                has[2] = r > 0;
                has[3] = r < H - 1;
            }
            for (int kb = 0; kb < kRingKB; ++kb, ++i) {
                const int s = (int)(i % kRingStages);
                const uint32_t ph = (uint32_t)((i / kRingStages) & 1);
                if (!mbar_wait(&m.empty[s], ph ^ 1, m.abort_flag)) {
                    *m.abort_flag = 1;
                    atomicExch(status, 131);
                    ok = false;
                    break;
                }
                float gv[8], mv[4][8];
                if (n < N) {
                    const long long off = n * kRingMP + kb * kBlockK + cc * 8;
                    const float4 g0 = __ldg(reinterpret_cast<const float4 *>(g + off));
                    const float4 g1 = __ldg(reinterpret_cast<const float4 *>(g + off) + 1);
                    gv[0] = g0.x; gv[1] = g0.y; gv[2] = g0.z; gv[3] = g0.w;
                    gv[4] = g1.x; gv[5] = g1.y; gv[6] = g1.z; gv[7] = g1.w;
#pragma unroll
                    for (int sd = 0; sd < 4; ++sd) {
                        if (has[sd]) {
                            const float *mp = in + sd * d.plane + off;
                            const float4 a = __ldg(reinterpret_cast<const float4 *>(mp));
                            const float4 b = __ldg(reinterpret_cast<const float4 *>(mp) + 1);
                            mv[sd][0] = a.x; mv[sd][1] = a.y; mv[sd][2] = a.z; mv[sd][3] = a.w;
                            mv[sd][4] = b.x; mv[sd][5] = b.y; mv[sd][6] = b.z; mv[sd][7] = b.w;
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) mv[sd][k] = 1.f;
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        gv[k] = 0.f;
#pragma unroll
                        for (int sd = 0; sd < 4; ++sd) mv[sd][k] = 1.f;
                    }
                }
                uint8_t *As = m.A + s * kKStage;
#pragma unroll
                for (int td = 0; td < 4; ++td) {
                    float h[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        float p = has[td] ? gv[k] : 0.f;
#pragma unroll
                        for (int sd = 0; sd < 4; ++sd)
                            if (sd != td) p *= mv[sd][k];
                        h[k] = p;
                    }
                    const int row = td * 32 + nl;
                    const uint32_t o = (uint32_t)(row >> 3) * 1024 + (uint32_t)(row & 7) * 128 +
                                       (uint32_t)((cc ^ (row & 7)) * 16);
                    *reinterpret_cast<uint4 *>(As + o) = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                                                                    pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
                }
                // make the generic-proxy writes visible to the tensor core's reads
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&m.full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        mbar_expect_tx(m.b_full, kRingB);
        for (int kb = 0; kb < kRingKB; ++kb) tma_load_2d(m.B + kb * kRingMP * 128, &tmap_b, m.b_full, kb * kBlockK, 0);
        int last_acc = -1;
        uint32_t last_aph = 0;
        if (!ring_mma(m, tmem_base, n_tiles, last_acc, last_aph)) {
            *m.abort_flag = 1;
            atomicExch(status, 132);
        }
        mbar_wait(m.b_full, 0, nullptr);
        if (last_acc >= 0) mbar_wait(&m.acc_full[last_acc], last_aph, nullptr);
    } else if (warp >= kRingEpiWarp0) {
        const int quad = warp & 3;   // TMEM lanes of direction `quad`
        const int dr = (quad == 2) ? -1 : (quad == 3) ? 1 : 0;
        const int dc = (quad == 0) ? -1 : (quad == 1) ? 1 : 0;
        const long long delta = (long long)dr * W + dc;
        float *dst_plane = out + (long long)(quad ^ 1) * d.plane;
        float *stg = m.epi + (warp - kRingEpiWarp0) * 32 * 32;
        long long j = 0;
        for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
            const int acc = (int)(j & 1);
            const uint32_t aph = (uint32_t)((j >> 1) & 1);
            if (!__all_sync(0xffffffffu, mbar_wait(&m.acc_full[acc], aph, m.abort_flag))) {
                if (lane == 0) {
                    *m.abort_flag = 1;
                    atomicExch(status, 133);
                }
                break;
            }
            tc_fence_after();
            const long long n0 = t * kRingNodes;
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
            ring_store_tile(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * kRingMP), stg, lane,
                            [&](int r) -> float * {
                                return ((valid >> r) & 1u) ? dst_plane + (n0 + r + delta) * kRingMP : nullptr;
                            });
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&m.acc_empty[acc]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tmem_base, kRingTmemCols);
    }
}

template <typename K>
cudaError_t set_ring_smem(K kern) {
    // the attribute belongs to the device's copy of the kernel: set it once per device
    static bool attr_set[bpg::kMaxDevices] = {};
    const int dev = bpg::current_device();
    if (dev < bpg::kMaxDevices && attr_set[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmem);
    if (e == cudaSuccess && dev < bpg::kMaxDevices) attr_set[dev] = true;
    return e;
}

}  // namespace

namespace bpg {

cudaError_t launch_gemm_ring256(const CUtensorMap &map_a, const CUtensorMap &map_b, float *out, long long rows,
                                int *status, cudaStream_t s) {
    cudaError_t e = set_ring_smem(dense_tc_gemm_ring_kernel);
    if (e != cudaSuccess) return e;
    const long long tiles = (rows + kTileM - 1) / kTileM;
    int grid = device_sm_count();
    if (grid > tiles) grid = (int)tiles;
    dense_tc_gemm_ring_kernel<<<grid, kThreads, kRingSmem, s>>>(map_a, map_b, out, rows, status);
    return cudaGetLastError();
}

cudaError_t launch_fused_ring256(const CUtensorMap &map_b, const float *g, const float *in, float *out,
                                 const GridDims &d, int *status, cudaStream_t s) {
    cudaError_t e = set_ring_smem(dense_tc_fused_ring_kernel);
    if (e != cudaSuccess) return e;
    const long long tiles = ((long long)d.W * d.H + kRingNodes - 1) / kRingNodes;
    int grid = device_sm_count();
    if (grid > tiles) grid = (int)tiles;
    dense_tc_fused_ring_kernel<<<grid, kRingFusedThreads, kRingSmem, s>>>(map_b, g, in, out, d, status);
    return cudaGetLastError();
}

}  // namespace bpg
