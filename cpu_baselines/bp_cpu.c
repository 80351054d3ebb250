/*
 * CPU throughput baselines for the benchmark -- MEASUREMENT INFRASTRUCTURE.
 *
 * Not the oracle (that is FP64 dense BP, written for obviousness) and not the
 * product (the CUDA library has no CPU path).  Sec. 6 of the paper times the
 * standard O(M^2) sum-product update against the O(mM) update on a CPU; these
 * two functions make the same comparison on the host cores of the GPU machine:
 *
 *   cpu_dense_iteration  Eq. 2:  m(x_j) = sum_{x_i} f(x_i, x_j) h(x_i)
 *   cpu_band_iteration   Eq. 7:  m(x_j) = fbar S + sum_{|d|<=T} (f(d) - fbar) h(x_j + d)
 *
 * with h(x_i) = g(x_i) prod_{k != j} m_ki(x_i), S = sum_x h(x), and each new
 * message divided by its sum.  FP32, one synchronous iteration, OpenMP over
 * grid rows, plain loops the compiler can vectorise.
 *
 * Layout: g [H][W][M]; in, out [4][H][W][M]; plane s holds the message INTO
 * (r, c) from its neighbour on side s (0 left, 1 right, 2 up, 3 down).  The
 * nodes of rows [row_lo, row_hi) send their outgoing messages; a message sent
 * towards side t lands in the neighbour's plane t ^ 1.  Slots of absent
 * neighbours are never read or written.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CPU_MAX_LABELS 1024

int cpu_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static const int kDr[4] = {0, 0, -1, 1};
static const int kDc[4] = {-1, 1, 0, 0};

static int check_args(int W, int H, int M, int row_lo, int row_hi) {
    if (W < 1 || H < 1 || M < 2 || M > CPU_MAX_LABELS) return 1;
    if (row_lo < 0 || row_hi > H || row_lo > row_hi) return 1;
    return 0;
}

/* h for the message leaving (r, c) towards side t */
static void form_h(int W, int H, int M, const float *g, const float *in, int r, int c, int t, float *h) {
    const long N = (long)W * H, node = (long)r * W + c;
    memcpy(h, g + node * M, sizeof(float) * (size_t)M);
    for (int s = 0; s < 4; ++s) {
        if (s == t) continue;
        const int rs = r + kDr[s], cs = c + kDc[s];
        if (rs < 0 || rs >= H || cs < 0 || cs >= W) continue;
        const float *m = in + ((long)s * N + node) * M;
        for (int x = 0; x < M; ++x) h[x] *= m[x];
    }
}

static void normalise(int M, float *o) {
    float z = 0.f;
    for (int x = 0; x < M; ++x) z += o[x];
    const float inv = 1.f / z;
    for (int x = 0; x < M; ++x) o[x] *= inv;
}

/* band[d + T] = f(d) for |d| <= T */
int cpu_band_iteration(int W, int H, int M, const float *g, const float *in, float *out,
                       const float *band, int T, float fbar, int row_lo, int row_hi, int n_threads) {
    if (check_args(W, H, M, row_lo, row_hi) || T < 0) return 1;
    const long N = (long)W * H;
    float wd[2 * CPU_MAX_LABELS + 1];
    const int Tc = T < M - 1 ? T : M - 1;          /* offsets past M - 1 never meet a label */
    for (int d = -Tc; d <= Tc; ++d) wd[d + Tc] = band[d + T] - fbar;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(n_threads)
#endif
    for (int r = row_lo; r < row_hi; ++r) {
        float h[CPU_MAX_LABELS];
        for (int c = 0; c < W; ++c)
            for (int t = 0; t < 4; ++t) {
                const int rn = r + kDr[t], cn = c + kDc[t];
                if (rn < 0 || rn >= H || cn < 0 || cn >= W) continue;
                form_h(W, H, M, g, in, r, c, t, h);
                float S = 0.f;
                for (int x = 0; x < M; ++x) S += h[x];
                float *o = out + ((long)(t ^ 1) * N + (long)rn * W + cn) * M;
                const float base = fbar * S;
                for (int x = 0; x < M; ++x) o[x] = base;
                for (int d = -Tc; d <= Tc; ++d) {
                    const float w = wd[d + Tc];
                    const int lo = d < 0 ? -d : 0, hi = d > 0 ? M - d : M;
                    for (int x = lo; x < hi; ++x) o[x] += w * h[x + d];
                }
                normalise(M, o);
            }
    }
    return 0;
}

/* F[x_i][x_j] = f(x_i, x_j), M x M row-major */
int cpu_dense_iteration(int W, int H, int M, const float *g, const float *in, float *out,
                        const float *F, int row_lo, int row_hi, int n_threads) {
    if (check_args(W, H, M, row_lo, row_hi)) return 1;
    const long N = (long)W * H;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(n_threads)
#endif
    for (int r = row_lo; r < row_hi; ++r) {
        float h[CPU_MAX_LABELS];
        for (int c = 0; c < W; ++c)
            for (int t = 0; t < 4; ++t) {
                const int rn = r + kDr[t], cn = c + kDc[t];
                if (rn < 0 || rn >= H || cn < 0 || cn >= W) continue;
                form_h(W, H, M, g, in, r, c, t, h);
                float *o = out + ((long)(t ^ 1) * N + (long)rn * W + cn) * M;
                for (int x = 0; x < M; ++x) o[x] = 0.f;
                for (int y = 0; y < M; ++y) {
                    const float hy = h[y];
                    const float *Fy = F + (long)y * M;
                    for (int x = 0; x < M; ++x) o[x] += hy * Fy[x];
                }
                normalise(M, o);
            }
    }
    return 0;
}
