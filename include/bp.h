/*
 * bp.h -- exact O(mM) belief propagation on 4-connected grids (C ABI).
 *
 * Pairwise MRF (Eq. 1):  P(x) ~ prod_<ij> f(x_i, x_j) prod_i g_i(x_i)
 * on an H x W 4-connected lattice with M labels per node (the stereo model of
 * Sec. 6).  The pairwise potential has the sparse compatibility property
 * (Sec. 1, Sec. 4): f(x_i, x_j) = fbar whenever |x_i - x_j| > T, so a message
 * update (Eq. 2) is computed exactly in O(mM), m = 2T + 1, as
 *     m_ij(x_j) = sum_{|x_i - x_j| <= T} [f(x_i, x_j) - fbar] h(x_i) + fbar sum_x h(x)    (Eq. 7)
 * for sum-product, and for max-product in energies (min-sum) as
 *     m_ij(x_j) = min{ min_{|x_i - x_j| <= T} [E(x_i - x_j) + h(x_i)], Ebar + min_x h(x) } (Eq. 11)
 * with h the unary times the other incoming messages (Eq. 5).
 *
 * Conventions shared by every call:
 *  - Arrays passed as `dev_*` are CUDA device pointers on the current device;
 *    arrays passed as `host_*` are host pointers.  The library never keeps a
 *    caller pointer after a call returns: inputs are copied into buffers the
 *    handle owns, outputs are written into caller buffers.  Device inputs are
 *    read, and outputs written, by work on the handle's stream that may still
 *    be running when the call returns: keep such a buffer unchanged (and
 *    allocated) until that stream has reached the work, e.g. by bp_sync or by
 *    ordering the caller's stream after it.  Host arrays are read before the
 *    call returns, except where a call says otherwise.
 *  - Layouts are C order with the label innermost: a unary or belief array is
 *    [H][W][M]; message planes are [4][H][W][M], where plane s holds the
 *    message INTO node (r, c) from its neighbour on side s
 *    (0: left (r, c-1), 1: right (r, c+1), 2: up (r-1, c), 3: down (r+1, c)).
 *    Slots without a neighbour (grid border) are never read.
 *  - dtype BP_F32 (sum-product on float32 potentials g, f) or BP_I32
 *    (min-sum on int32 energies E_u, E).  Energies must lie in [0, 2^26).
 *  - All device work is ordered on the handle's stream.  Argument and state
 *    errors are returned synchronously and nothing is launched; device
 *    errors and kernel time-outs surface at the next call or at bp_sync.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Tracing: the main calls (create, set, iterate, beliefs, backward, sync,
 *    autotune, of single grids, batches and factor graphs) each open an NVTX
 *    range named after the call.  With the environment variable BP_LOG set to
 *    a value other than 0 when the first of them runs, each also writes one
 *    line to stderr with its host-side time ("[bp] <call> <us> us host"), and
 *    every error any call reports is written as "[bp] error <status>: <message>".
 */
#ifndef BPGRID_BP_H
#define BPGRID_BP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bp_ctx *bp_handle;

typedef enum {
    BP_OK = 0,
    BP_ERR_ARG = 1,         /* bad argument (null pointer, size, range)          */
    BP_ERR_STATE = 2,       /* call out of order (e.g. iterate before set_unary) */
    BP_ERR_CUDA = 3,        /* a CUDA runtime error; see bp_last_error           */
    BP_ERR_OOM = 4,         /* device allocation failed                          */
    BP_ERR_POTENTIAL = 5,   /* max mode with E(d) > Ebar: Eq. 11 needs f >= fbar */
    BP_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up                */
    BP_ERR_UNSUPPORTED = 7  /* valid request outside what the library serves     */
} bp_status;

/* Message-passing mode (Sec. 3 and Sec. 5).  BP_LOG and BP_RECORD are flags
 * or-ed onto BP_SUM: BP_LOG keeps log-messages (numerically robust form of the
 * same update); BP_RECORD additionally stores checkpoints for bp_backward. */
typedef enum { BP_SUM = 0, BP_MAX = 1, BP_LOG = 2, BP_RECORD = 4 } bp_mode;

/* Schedules.  BP_SYNC: every message of iteration t+1 from those of
 * iteration t.  BP_REDBLACK: the checkerboard schedule (Sec. 2, from [2]):
 * an iteration is a half-step over nodes with (r + c) even, sending all their
 * messages, then one over nodes with (r + c) odd, in place. */
typedef enum { BP_SYNC = 0, BP_REDBLACK = 1 } bp_schedule;

typedef enum { BP_F32 = 0, BP_I32 = 1 } bp_dtype;

/* O(M^2) baselines of the standard update (Eq. 2 / Eq. 9), for comparison. */
typedef enum {
    BP_DENSE_CUDA_CORE = 0, /* FP32 sum-product or int32 min-sum, CUDA cores          */
    BP_DENSE_BF16_TC = 1,   /* sum-product as a (nodes*4 x M)(M x M) tcgen05 GEMM,    */
                            /* BF16 operands, FP32 accumulate, normalising epilogue;  */
                            /* h rows packed to HBM by a separate kernel (M 33..256)  */
    BP_DENSE_BF16_TC_FUSED = 2 /* the same GEMM with h formed on chip from one read  */
                            /* of the node's vectors (same HBM bytes as the O(mM)     */
                            /* update; M 33..256)                                     */
} bp_dense_kind;

/* Create a handle for the pairwise MRF of Eq. 1 on an H x W 4-connected grid
 * (the stereo lattice of Sec. 6) with M labels (2 <= M <= 1024,
 * 1 <= W, H, W*H*M < 2^31).  cuda_stream: a cudaStream_t to order all work on,
 * or NULL for a stream the handle creates (blocking with respect to the legacy
 * default stream).  Allocates the message buffers.  On error *out is NULL. */
bp_status bp_create(int W, int H, int M, bp_dtype dtype, void *cuda_stream, bp_handle *out);

/* Unary potential g_i(x) (Eq. 1): dev_unary [H][W][M], float32 g > 0 for
 * BP_F32, int32 energies E_u >= 0 for BP_I32.  Copied into the handle. */
bp_status bp_set_unary(bp_handle h, const void *dev_unary);

/* The unary of the stereo model (Sec. 6) formed on the device from the image
 * pair: left, right [H][W] uint8 (row-major, right = reference),
 * cost(r, c, x) = min(|R(r,c) - L(r,c+x)|, Tu), and Tu where c + x >= W.
 * host_table holds Tu + 1 values indexed by the cost: float32 g (e.g.
 * exp(-beta cost)) for BP_F32, int32 energies E_u for BP_I32; it is read
 * during the call.  The images may be device (or managed) memory, read in
 * place on the handle's stream, or host memory, which the call copies into a
 * handle-owned staging buffer on that stream (asynchronously from pinned
 * memory, before returning from pageable memory); either way they must stay
 * valid until that work has run.  Equivalent to bp_set_unary of
 * table[cost].  BP_ERR_ARG for Tu outside [0, 255], a negative or non-finite
 * g, or an energy outside [0, 2^26). */
bp_status bp_set_unary_stereo(bp_handle h, const uint8_t *left, const uint8_t *right,
                              const void *host_table, int Tu);

/* The same unary (Eq. 1's g) given as log g (BP_F32 only): dev_logg
 * [H][W][M] float32.  Log-domain runs use these values as they are (no round
 * trip through g); it is the parameter bp_backward differentiates against. */
bp_status bp_set_unary_log(bp_handle h, const float *dev_logg);

/* Pairwise potential with the sparse compatibility property (Sec. 4):
 * host_table[d + T] = f(d), d = x_i - x_j (sender minus receiver label),
 * -T <= d <= T; every pair with |d| > T has the value fbar.
 * BP_F32: float32 table, f > 0, fbar >= 0 (fbar = 0 is the pruned form Eq. 8).
 * BP_I32: int32 energies E(d) >= 0 and Ebar = fbar (an integer); since the
 * max-product form Eq. 11 is exact only when f >= fbar (Sec. 5), i.e.
 * E(d) <= Ebar, a table with some E(d) > Ebar returns BP_ERR_POTENTIAL.
 * 0 <= T; T >= M - 1 makes the band cover every label pair. */
bp_status bp_set_potential(bp_handle h, const void *host_table, int T, double fbar);

/* General sparse compatibility (Sec. 4: Nbd(x_j) of any shape; Sec. 7:
 * robust potentials that are not a function of x_i - x_j).  For each receiver
 * label x_j, host_cols[host_rowptr[x_j] .. host_rowptr[x_j+1]) lists the
 * compatible sender labels x_i (distinct, in [0, M)) and host_vals holds
 * f(x_i, x_j) (float32) or E(x_i, x_j) (int32) for them; every other pair has
 * fbar (Ebar).  host_rowptr has M+1 entries, rowptr[0] = 0.  One message then
 * costs O(nnz) with nnz = rowptr[M] (O(mM) for m pairs per label).  Replaces
 * any band potential; BP_ERR_POTENTIAL in max mode if some E > Ebar;
 * BP_ERR_UNSUPPORTED for M > 512.  The pattern is copied to the device (8
 * bytes per receiver label per entry of the longest list), and, where it fits
 * the register kernel (bp_set_sparse_kernel), scheduled on the host for it.  Log mode and
 * bp_backward need a band potential. */
bp_status bp_set_potential_sparse(bp_handle h, const int32_t *host_rowptr, const int32_t *host_cols,
                                  const void *host_vals, double fbar);

/* Uniform initial messages: 1/M (sum), 0 (min-sum), log(1/M) (log mode).
 * The paper leaves the start state open (Sec. 2 runs BP from any messages);
 * uniform is the usual choice and is normalised as after Eq. 2. */
bp_status bp_reset_messages(bp_handle h);

/* Run n_iters iterations of the O(mM) update under `schedule`: Eq. 7 for
 * sum-product, Eq. 11 (energies) for max-product, every message of every
 * node per iteration (Sec. 4's per-message cost O(mM) instead of Eq. 2's
 * O(M^2)).  mode: BP_SUM (needs BP_F32), BP_MAX (needs BP_I32), or BP_SUM|BP_LOG and
 * BP_SUM|BP_LOG|BP_RECORD (log-messages, BP_SYNC only).  Messages are
 * normalised after each update (sum 1, or minimum 0 for min-sum). */
bp_status bp_iterate(bp_handle h, int n_iters, int mode, bp_schedule schedule);

/* Coarse-to-fine BP (the multi-scale scheme of [2], combined with the O(mM)
 * update as Sec. 2 and Sec. 6 suggest).  Level l+1 has one node per 2 x 2 block
 * of level l, unary = product of the block's g scaled to maximum 1 per node
 * (BP is unchanged by that scale; it keeps FP32 in range) or the sum of the
 * block's energies for min-sum,
 * the handle's pairwise potential at every level.  host_iters[k] iterations run
 * at level n_levels-1-k (coarsest first, host_iters[n_levels-1] on this grid);
 * each finer level starts from the coarser level's final messages copied by
 * direction (uniform where the coarse node has no neighbour on that side).
 * mode BP_SUM or BP_MAX; either schedule.  Leaves this grid's messages as after
 * bp_iterate.  The coarse levels are allocated on the first call. */
bp_status bp_iterate_multiscale(bp_handle h, int n_levels, const int *host_iters, int mode, bp_schedule schedule);

/* Run n_iters synchronous iterations of the dense O(M^2) update (Eq. 2 or
 * Eq. 9), the baseline the O(mM) update is measured against. */
bp_status bp_iterate_dense(bp_handle h, int n_iters, bp_dense_kind kind);

/* Beliefs (Eq. 3) into dev_out [H][W][M]: float32 normalised beliefs
 * (BP_F32; in log mode the normalised log-beliefs) or int32 min-sum beliefs
 * E_u + sum of incoming messages (BP_I32).  dev_map (nullable) [H][W] int32
 * receives the MAP label: argmax (sum) / argmin (min-sum), lowest label on ties. */
bp_status bp_beliefs(bp_handle h, void *dev_out, int32_t *dev_map);

/* Copy the current message planes out / in: the messages m_ij(x_j) of Eq. 2
 * ([4][H][W][M], dtype of the handle).  Float32 messages cross this boundary linear (normalised) in every
 * mode: after log-mode iterations bp_get_messages returns exp of the
 * log-domain state, and bp_set_messages installs a linear state.  Slots
 * without a neighbour (never read by any update) come out as 0 and are
 * ignored on the way in.  Used to checkpoint or inject a state. */
bp_status bp_get_messages(bp_handle h, void *dev_planes);
bp_status bp_set_messages(bp_handle h, const void *dev_planes);

/* Reverse mode of the recorded log-domain sum-product run (bp_iterate with
 * BP_SUM|BP_LOG|BP_RECORD) followed by bp_beliefs: the gradient of a loss of
 * the beliefs (Eq. 3) through the unrolled Eq. 7 updates, for learning the
 * potentials (parameter estimation needs sum-product marginals, Sec. 2 and
 * Sec. 7).  The
 * adjoint of Eq. 7 is again a band of width 2T + 1 plus a constant term, so
 * it also costs O(mM) per message.  Given
 * dev_dlogb = dL/d log b [H][W][M], writes dev_dlogg = dL/d log g [H][W][M]
 * and, in float64, host_dtable[d + T] = dL/d f(d) (2T + 1 values) and
 * *host_dfbar = dL/d fbar, with f(d) and fbar independent parameters.
 * Synchronises the handle's stream. */
bp_status bp_backward(bp_handle h, const float *dev_dlogb, float *dev_dlogg, double *host_dtable,
                      double *host_dfbar);

/* bp_backward with the parameter gradients in device memory: dev_dtable
 * [2T + 1] and *dev_dfbar (float64, device) are written by copies on the
 * handle's stream, like dev_dlogg, and nothing synchronises, so a caller can
 * queue more work behind the reverse pass (no counterpart in the paper; the
 * values equal bp_backward's bit for bit). */
bp_status bp_backward_device(bp_handle h, const float *dev_dlogb, float *dev_dlogg, double *dev_dtable,
                             double *dev_dfbar);

/* Checkpoint interval used by BP_RECORD runs (default 5): the recorded run
 * keeps every `every`-th message state, and bp_backward recomputes the states
 * between them (no counterpart in the paper). */
bp_status bp_set_checkpoint_interval(bp_handle h, int every);

/* Wait for the handle's stream; reports device errors and time-outs (no
 * counterpart in the paper, like the rest of the handle management). */
bp_status bp_sync(bp_handle h);

/* Last error message of the handle (never NULL; "" if none; no counterpart
 * in the paper).  Valid until
 * the next call on the handle.  bp_last_error(NULL) reports errors of
 * bp_create and of calls given a NULL handle. */
const char *bp_last_error(bp_handle h);

/* Release everything the handle owns.  NULL is ignored (no counterpart in
 * the paper). */
void bp_destroy(bp_handle h);

/* ---- tuning (no counterpart in the paper: how the O(mM) update of Eq. 7 /
 * Eq. 11 maps onto the GPU; results do not depend on these settings) ---------
 * The O(mM) kernel assigns L lanes to a node, each lane holding V = 4C
 * consecutive labels (L * 4C = padded label count).  The log-domain kernels
 * (BP_LOG iterations, the recorded forward and its adjoint) keep a layout of
 * their own, by default one chunk per lane.  bp_set_layout sets (L, C) for
 * both; bp_get_layout reports the plain-mode layout; bp_autotune times every
 * layout available for the handle's (M, T, mode) and keeps the fastest for
 * the layout that mode uses (the log-domain one when mode has BP_LOG). */
bp_status bp_set_layout(bp_handle h, int lanes_per_node, int vec_chunks);
bp_status bp_get_layout(bp_handle h, int *lanes_per_node, int *vec_chunks);
bp_status bp_autotune(bp_handle h, int mode, int n_iters, float *host_best_ms);
/* Blocks per launch of the O(mM) register kernels (grid-stride over nodes);
 * 0 (default) = SM count x resident blocks per SM.  Tuning, as above: no
 * counterpart in the paper. */
bp_status bp_set_grid(bp_handle h, int blocks);

/* Allocation-free dense tensor-core iteration (no counterpart in the paper;
 * an addition for callers that cannot allocate device memory).  Some callers
 * cannot call cudaMalloc: their device memory is planned once by another
 * component (a serving process's memory pool, a framework that forbids
 * allocation after warm-up), or an allocation at that point could synchronise
 * the device or fail unpredictably.  This call runs one synchronous iteration
 * of the BF16 tensor-core O(M^2) update (as bp_iterate_dense with
 * BP_DENSE_BF16_TC) without any allocation: its scratch lives in a fixed
 * device array of 32 MiB + 32 KiB inside the library, which every GPU that
 * loads the library holds until the process exits.
 *   W, H, M         grid and label count; M must be 64 or 128, and the packed
 *                   rows 4*W*H*M*2 bytes must fit in 32 MiB (W*H <= 32768 at
 *                   M = 128, <= 65536 at M = 64); larger sizes return BP_ERR_ARG.
 *   dev_unary       [H][W][M] float32 g > 0;
 *   dev_in_planes   [4][H][W][M] float32 current messages (layout as above);
 *   dev_out_planes  [4][H][W][M] float32 updated messages, a range that must
 *                   not overlap dev_in_planes; slots without a neighbour
 *                   receive 0;
 *   host_table      2T+1 float32 values f(d), d = -T..T, and fbar outside
 *                   (for T >= M only d = -(M-1)..M-1 is read).
 * The three device pointers must be 16-byte aligned (the kernels move 16-byte
 * vectors); a misaligned or overlapping argument returns BP_ERR_ARG before
 * anything is launched.
 * Set-up: the first call on a device (and again after the device's context
 * changes, e.g. after cudaDeviceReset) looks up the array's device address
 * with that device current.  Under lazy module loading that first call is also
 * the one that loads the library's kernels, at which point the driver places
 * the 32 MiB array on the device: make it once at start-up, as a warm-up.
 * The call enqueues its kernels on cuda_stream (NULL: the legacy default
 * stream), then synchronises that stream and reads a status word back, so it
 * returns after its kernels have completed and cannot be captured into a CUDA
 * graph (a capturing stream returns BP_ERR_STATE).  All calls share the one
 * array, which keeps the last call's contents: calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Errors are reported through bp_last_error(NULL). */
bp_status bp_iterate_dense_tc_noalloc(int W, int H, int M, const float *dev_unary, const float *dev_in_planes,
                                      float *dev_out_planes, const float *host_table, int T, double fbar,
                                      void *cuda_stream);

/* ---- batches of independent MRFs --------------------------------------------
 * Many MRFs of different size, label count and band width (each an H x W
 * grid as above, homogeneous within itself; Eq. 1 with per-MRF potentials,
 * the inhomogeneous case of Sec. 1) advanced together by ONE persistent
 * cooperative kernel launch per bp_batch_iterate call, captured once in a CUDA
 * graph and replayed.  Synchronous schedule only; 2 <= M <= 256, band
 * half-width min(T, M-1) <= 8.  Inside the launch, blocks take the work items
 * (grouped by band width and label count) from a shared counter. */
typedef struct {
    int W, H, M;               /* grid and label count of this MRF                 */
    int T;                     /* band half-width                                  */
    const void *dev_unary;     /* [H][W][M] g (float32) or E_u (int32); copied     */
    const void *host_table;    /* 2T+1 values f(d) (float32) or E(d) (int32)       */
    double fbar;               /* fbar, or the integer Ebar for min-sum            */
} bp_mrf_desc;

typedef struct bp_batch_ctx *bp_batch;

/* Validate the n descriptors (as bp_set_potential would: BP_ERR_POTENTIAL for
 * E(d) > Ebar), allocate every MRF's unary and two message states, copy the
 * unaries, and cut the nodes into work items.  cuda_stream as in bp_create. */
bp_status bp_batch_create(int n, const bp_mrf_desc *descs, bp_dtype dtype, void *cuda_stream, bp_batch *out);
/* Uniform start state of every MRF (as bp_reset_messages). */
bp_status bp_batch_reset_messages(bp_batch b);
/* n_iters synchronous iterations (Eq. 7 or Eq. 11, each MRF with its own
 * potential) of every MRF in one launch.  mode BP_SUM
 * (float32 batch) or BP_MAX (int32 batch).  Between iterations the blocks meet
 * at a grid barrier whose wait is bounded; a wait that runs out ends the
 * kernel and the next bp_batch_sync returns BP_ERR_TIMEOUT. */
bp_status bp_batch_iterate(bp_batch b, int n_iters, int mode);
/* Beliefs / MAP (Eq. 3, as bp_beliefs) and message planes (as
 * bp_get_messages) of MRF k; BP_ERR_ARG for k outside [0, n). */
bp_status bp_batch_beliefs(bp_batch b, int k, void *dev_out, int32_t *dev_map);
bp_status bp_batch_get_messages(bp_batch b, int k, void *dev_planes);
/* Work decomposition (no counterpart in the paper; min-sum results do not
 * depend on it, sum-product results only through the order of the terms of
 * each sum): per (padded label count Mp, effective band half-width T) class
 * of the batch, the lane layout (family 1: 4 labels per lane; 2: 8 labels per
 * lane) and the item size in label words (256 .. 2^24).  One launch can mix
 * classes of different families.
 * bp_batch_set_tiling sets every class; bp_batch_get_tiling reports the
 * setting of the class holding the most label words.  bp_batch_class_count
 * returns the number of classes (-1 for NULL); bp_batch_get_class_tiling
 * reports class k (classes in increasing (Mp, T) order; BP_ERR_ARG outside
 * [0, count)); bp_batch_set_class_tiling sets the class (Mp, T) (BP_ERR_ARG if
 * no MRF of the batch has it).
 * bp_batch_autotune times, class by class, every (family, tile) candidate on
 * that class's items alone for n_iters iterations and keeps each class's
 * fastest; then it times the whole batch under those choices, under the same
 * item sizes with one family for every class, and under each single setting
 * for all classes, and keeps the fastest: *host_best_ms (nullable) is its
 * time per iteration.  The choices are cached in $BP_AUTOTUNE_CACHE when
 * set (a second call on a batch of the same classes and size reads them).
 * Resets the messages. */
bp_status bp_batch_set_tiling(bp_batch b, int family, int tile_words);
bp_status bp_batch_get_tiling(bp_batch b, int *family, int *tile_words);
int bp_batch_class_count(bp_batch b);
bp_status bp_batch_get_class_tiling(bp_batch b, int k, int *Mp, int *T, int *family, int *tile_words);
bp_status bp_batch_set_class_tiling(bp_batch b, int Mp, int T, int family, int tile_words);
bp_status bp_batch_autotune(bp_batch b, int mode, int n_iters, float *host_best_ms);
/* Bound of the grid-barrier wait (default 2 s; failure detection, no
 * counterpart in the paper).  extra_arrivals = 1 makes the
 * barrier wait for one block that does not exist, so that every wait runs
 * out: a fault-free way to exercise the time-out path. */
bp_status bp_batch_set_wait_limit(bp_batch b, double seconds, int extra_arrivals);
/* As bp_sync, bp_last_error (NULL: errors of bp_batch_create and of calls
 * given a NULL batch), bp_launch_count and bp_destroy, for a batch. */
bp_status bp_batch_sync(bp_batch b);
const char *bp_batch_last_error(bp_batch b);
long long bp_batch_launch_count(bp_batch b);
void bp_batch_destroy(bp_batch b);

/* How bp_iterate issues the linear sum-product and min-sum updates (no
 * counterpart in the paper; the updates themselves are Eq. 7 / Eq. 11):
 * 0: one launch per iteration (two per red-black iteration);
 * 1: ONE persistent cooperative launch for the whole call, with a bounded grid
 *    barrier between iterations (half-steps), where served (16 < Mp <= 256
 *    after padding, T <= 8); otherwise as 0;
 * -1 (default): the faster form as measured on GB300, currently 0 at every
 *    size (CUDA-graph replay of per-iteration launches beats the persistent
 *    kernel's grid barrier even on 32 x 32 grids).  Results are identical. */
bp_status bp_set_persistent(bp_handle h, int mode);

/* Which kernel runs a general sparse-compatibility potential (no counterpart
 * in the paper; both compute Sec. 4's O(nnz) form of Eq. 7 / Eq. 11 and give
 * the same messages up to the order of the terms of each sum):
 *   BP_SPARSE_LISTS      per-label entry lists read from the device for
 *                        every node (any pattern, M <= 512);
 *   BP_SPARSE_REGISTERS  the pattern held in registers for the whole launch,
 *                        its entries scheduled on the host so that the
 *                        shared-memory gathers do not conflict (M <= 256 and
 *                        a schedule of at most 48, 24, 12 or 6 steps per
 *                        32-label block for M <= 32, 64, 128, 256).
 *                        Min-sum with Ebar <= 16382 runs it on 16-bit label
 *                        pairs: h - min h clamped to Ebar + 1 (terms above
 *                        never beat the flat term Ebar + min h), two
 *                        directions per add-min; the messages equal the
 *                        32-bit kernel's exactly;
 *   BP_SPARSE_AUTO       (default) the register kernel where the pattern has
 *                        a schedule, else the lists.
 * bp_set_sparse_kernel returns BP_ERR_UNSUPPORTED when the current pattern has
 * no register schedule and BP_SPARSE_REGISTERS is asked for.
 * bp_get_sparse_kernel reports the kernel that runs, and for the register
 * kernel the steps per block and the gather wavefronts per node of the
 * schedule (0 for the lists); BP_ERR_STATE without a sparse potential. */
typedef enum { BP_SPARSE_AUTO = 0, BP_SPARSE_LISTS = 1, BP_SPARSE_REGISTERS = 2 } bp_sparse_kernel;
bp_status bp_set_sparse_kernel(bp_handle h, int kind);
bp_status bp_get_sparse_kernel(bp_handle h, int *kind, int *steps, int *wavefronts);

/* The register kernel's schedule of a pattern, computed on the host only (no
 * device, no handle; no counterpart in the paper).  Pattern as for
 * bp_set_potential_sparse (CSR by receiver label, M labels).  gather_bytes:
 * 16 for the FP32 / int32 kernels (16-byte h slots, label x in slot
 * (x & ~31) | ((x & 3) << 3) | ((x >> 2) & 7), served to quarter-warps from
 * eight 16-byte bank groups), 8 for the 16-bit min-sum form that min-sum
 * potentials with Ebar <= 16382 run (8-byte slots
 * (x & ~63) | ((x & 3) << 4) | ((x >> 2) & 15), half-warps, sixteen 8-byte
 * groups).  *KM = 32-label receiver blocks, *LM = register steps per block,
 * *steps = LM, *wavefronts = gather wavefronts per node; all 0 when the
 * pattern has no register schedule.  host_lab [KM][32] (nullable) receives
 * each lane's receiver label (-1: none); host_ent [KM][LM][32][2] (nullable)
 * each lane's entry per step: the byte offset of the sender label's h slot
 * (0xFFFF for a hole) and the entry's CSR position in host_cols.  Call with
 * NULL buffers first to learn KM and LM.  Errors through bp_last_error(NULL). */
bp_status bp_sparse_schedule(int M, const int32_t *host_rowptr, const int32_t *host_cols, int gather_bytes,
                             int *KM, int *LM, int *steps, int *wavefronts, int32_t *host_lab, int32_t *host_ent);

/* ---- factor graphs with three-variable factors (Sec. 7) --------------------
 * Variables v = 0..n_vars-1 with M labels and unaries g_v (or energies E_v);
 * factors a = 0..n_factors-1, each joining the three distinct variables
 * host_factor_vars[3a .. 3a+2] (slots 0, 1, 2), all sharing one potential
 * f(x_0, x_1, x_2) that equals fbar except on C listed compatible triplets.
 * A flooding iteration updates every variable-to-factor message, then every
 * factor-to-variable message:
 *   m_{a->v}(x_s) = sum over listed triplets with that x_s of [f - fbar] n_u n_w
 *                   + fbar (sum n_u)(sum n_w)                      O(C + M), not O(M^3)
 * (min-sum: min over listed triplets of E + n_u + n_w, against Ebar + min n_u
 * + min n_w; needs E <= Ebar).  Messages are normalised (sum 1 / minimum 0).
 * 2 <= M <= 256; a variable may belong to at most 16 factors. */
typedef struct bp_fg_ctx *bp_factor_graph;

/* A factor graph of n_vars variables and n_factors three-variable factors
 * (Sec. 7); cuda_stream and errors as in bp_create. */
bp_status bp_fg_create(int n_vars, int M, int n_factors, const int32_t *host_factor_vars, bp_dtype dtype,
                       void *cuda_stream, bp_factor_graph *out);
/* Unaries g_v (Eq. 1's single-variable factors), dev_unary [n_vars][M]:
 * float32 g > 0 or int32 energies; copied. */
bp_status bp_fg_set_unary(bp_factor_graph g, const void *dev_unary);
/* The shared factor potential with sparse compatibility (Sec. 7: C listed
 * triplets, fbar elsewhere).  host_triplets [C][3] distinct (x_0, x_1, x_2)
 * in [0, M); host_vals [C] f
 * (float32) or E (int32); fbar (or the integer Ebar) elsewhere.
 * BP_ERR_POTENTIAL in max mode if some E > Ebar.  The table is copied to the
 * device as three per-slot lists (8 bytes per output label per entry of the
 * longest list of that slot). */
bp_status bp_fg_set_factor(bp_factor_graph g, int C, const int32_t *host_triplets, const void *host_vals,
                           double fbar);
/* Uniform start state (as bp_reset_messages). */
bp_status bp_fg_reset_messages(bp_factor_graph g);
/* n_iters flooding iterations, mode BP_SUM (float32) or BP_MAX (int32), with
 * the O(C + M) factor update above (Sec. 7's extension of Eq. 7 / Eq. 11). */
bp_status bp_fg_iterate(bp_factor_graph g, int n_iters, int mode);
/* The same iterations with the standard O(M^3) factor update (the sum over
 * all M^2 pairs of the other two variables, the cost Sec. 7 avoids), for
 * comparison. */
bp_status bp_fg_iterate_dense(bp_factor_graph g, int n_iters, int mode);
/* Beliefs (Eq. 3 on the factor graph) [n_vars][M] (normalised float32, or
 * int32 E_v + sum of messages) and MAP labels (nullable), lowest label on ties. */
bp_status bp_fg_beliefs(bp_factor_graph g, void *dev_out, int32_t *dev_map);
/* Factor-to-variable messages m_{a->v} (Sec. 7) [n_factors][3][M] (slot order). */
bp_status bp_fg_get_messages(bp_factor_graph g, void *dev_out);
/* As bp_sync, bp_last_error (NULL: errors of bp_fg_create and of calls given
 * a NULL graph), bp_launch_count and bp_destroy, for a factor graph. */
bp_status bp_fg_sync(bp_factor_graph g);
const char *bp_fg_last_error(bp_factor_graph g);
long long bp_fg_launch_count(bp_factor_graph g);
void bp_fg_destroy(bp_factor_graph g);

/* Number of kernel launches the library issued on this handle so far (no
 * counterpart in the paper; lets a caller count the GPU work of a call). */
long long bp_launch_count(bp_handle h);

/* Library version, (major << 16) | minor (no counterpart in the paper). */
int bp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BPGRID_BP_H */
