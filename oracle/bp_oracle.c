/*
 * Oracle for loopy belief propagation on a pairwise MRF -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, obviously correct: dense O(M^2) message updates in FP64
 * (sum-product) or exact 64-bit integers (min-sum), on an arbitrary directed
 * edge list.  It never splits the pairwise table into a constant plus a band;
 * it is the standard update that the O(mM) method must reproduce exactly.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this library; the product path never does.
 *
 * Model (Eq. 1): P(x) ~ prod_<ij> f(x_i, x_j) prod_i g_i(x_i).
 * Tables: F[xi*M + xj] = f(x_i, x_j); g[i*M + x] = g_i(x).
 * Messages: msg[e*M + x] = m_{src(e) -> dst(e)}(x).
 *
 * Schedules:
 *   0  synchronous: every message of iteration t+1 from those of iteration t.
 *   1  two-colour:  an iteration is two half-steps; half-step c recomputes
 *                   every message leaving a node of colour c from the current
 *                   messages (colour 0 first, then colour 1).
 */
#include <stdlib.h>
#include <string.h>

/* ---- incoming-edge lists (CSR by destination) ---------------------------- */
typedef struct {
    int *start; /* n_nodes + 1 */
    int *edge;  /* n_edges */
} in_lists;

static int build_in_lists(int n_nodes, int n_edges, const int *dst, in_lists *L) {
    L->start = (int *)calloc((size_t)n_nodes + 1, sizeof(int));
    L->edge = (int *)malloc((size_t)(n_edges > 0 ? n_edges : 1) * sizeof(int));
    int *fill = (int *)calloc((size_t)n_nodes + 1, sizeof(int));
    if (!L->start || !L->edge || !fill) { free(L->start); free(L->edge); free(fill); return -1; }
    for (int e = 0; e < n_edges; ++e) L->start[dst[e] + 1]++;
    for (int i = 0; i < n_nodes; ++i) L->start[i + 1] += L->start[i];
    for (int e = 0; e < n_edges; ++e) {
        int j = dst[e];
        L->edge[L->start[j] + fill[j]++] = e;
    }
    free(fill);
    return 0;
}

static void free_in_lists(in_lists *L) { free(L->start); free(L->edge); }

static int check_graph(int n_nodes, int M, int n_edges, const int *src, const int *dst) {
    if (n_nodes < 0 || M < 1 || n_edges < 0) return -1;
    for (int e = 0; e < n_edges; ++e)
        if (src[e] < 0 || src[e] >= n_nodes || dst[e] < 0 || dst[e] >= n_nodes || src[e] == dst[e])
            return -1;
    return 0;
}

/* ---- sum-product ---------------------------------------------------------- */

/* One message update, Eq. 2 with the explicit normalisation noted after it:
 *   m_new(x_j) = sum_{x_i} f(x_i, x_j) g_i(x_i) prod_{k in N(i)\j} m_ki(x_i),
 *   then divided by its sum over x_j.
 * `inc` holds the n_inc messages m_ki, k in N(i)\j, each of M entries.
 * Returns -1 if the unnormalised message sums to zero. */
int oracle_sum_edge_update(int M, const double *g_i, int n_inc, const double *const *inc,
                           const double *F, double *out) {
    double *h = (double *)malloc((size_t)M * sizeof(double));
    if (!h) return -1;
    for (int x = 0; x < M; ++x) {            /* h(x_i) = g(x_i) prod m_ki(x_i) (Eq. 5) */
        double p = g_i[x];
        for (int k = 0; k < n_inc; ++k) p *= inc[k][x];
        h[x] = p;
    }
    double Z = 0.0;
    for (int xj = 0; xj < M; ++xj) {         /* Eq. 2 / Eq. 4: full sum over x_i */
        double u = 0.0;
        for (int xi = 0; xi < M; ++xi) u += F[(size_t)xi * M + xj] * h[xi];
        out[xj] = u;
        Z += u;
    }
    free(h);
    if (!(Z > 0.0)) return -1;
    for (int xj = 0; xj < M; ++xj) out[xj] /= Z;
    return 0;
}

static int sum_update_edge(int e, int M, const int *src, const int *dst, const in_lists *L,
                           const double *g, const double *F, const double *msg, double *out,
                           const double **scratch) {
    int i = src[e], j = dst[e], n = 0;
    for (int p = L->start[i]; p < L->start[i + 1]; ++p) {
        int e2 = L->edge[p];
        if (src[e2] != j) scratch[n++] = msg + (size_t)e2 * M;
    }
    return oracle_sum_edge_update(M, g + (size_t)i * M, n, scratch, F, out);
}

int oracle_sum_product(int n_nodes, int M, int n_edges, const int *src, const int *dst,
                       const double *g, const double *F, const int *color, int schedule,
                       int n_iters, double *msg) {
    if (check_graph(n_nodes, M, n_edges, src, dst) || n_iters < 0) return -1;
    if (schedule != 0 && schedule != 1) return -1;
    if (schedule == 1 && !color) return -1;
    in_lists L;
    if (build_in_lists(n_nodes, n_edges, dst, &L)) return -1;
    size_t sz = (size_t)n_edges * M;
    double *next = (double *)malloc((sz ? sz : 1) * sizeof(double));
    const double **scratch = (const double **)malloc((size_t)(n_edges + 1) * sizeof(double *));
    int rc = (next && scratch) ? 0 : -1;
    for (int t = 0; t < n_iters && rc == 0; ++t) {
        if (schedule == 0) {
            for (int e = 0; e < n_edges && rc == 0; ++e)
                rc = sum_update_edge(e, M, src, dst, &L, g, F, msg, next + (size_t)e * M, scratch);
            if (rc == 0) memcpy(msg, next, sz * sizeof(double));
        } else {
            for (int c = 0; c < 2 && rc == 0; ++c) {
                for (int e = 0; e < n_edges && rc == 0; ++e)
                    if (color[src[e]] == c)
                        rc = sum_update_edge(e, M, src, dst, &L, g, F, msg, next + (size_t)e * M, scratch);
                for (int e = 0; e < n_edges && rc == 0; ++e)
                    if (color[src[e]] == c)
                        memcpy(msg + (size_t)e * M, next + (size_t)e * M, (size_t)M * sizeof(double));
            }
        }
    }
    free(next);
    free(scratch);
    free_in_lists(&L);
    return rc;
}

/* Beliefs, Eq. 3: b_i(x) = g_i(x) prod_{k in N(i)} m_ki(x) / Z_i. */
int oracle_sum_beliefs(int n_nodes, int M, int n_edges, const int *dst, const double *g,
                       const double *msg, double *belief) {
    for (int i = 0; i < n_nodes; ++i)
        for (int x = 0; x < M; ++x) belief[(size_t)i * M + x] = g[(size_t)i * M + x];
    for (int e = 0; e < n_edges; ++e) {
        int j = dst[e];
        if (j < 0 || j >= n_nodes) return -1;
        for (int x = 0; x < M; ++x) belief[(size_t)j * M + x] *= msg[(size_t)e * M + x];
    }
    for (int i = 0; i < n_nodes; ++i) {
        double Z = 0.0;
        for (int x = 0; x < M; ++x) Z += belief[(size_t)i * M + x];
        if (!(Z > 0.0)) return -1;
        for (int x = 0; x < M; ++x) belief[(size_t)i * M + x] /= Z;
    }
    return 0;
}

/* ---- min-sum (max-product in the negative-log domain), exact integers ------ */

/* One message update, Eq. 9 written with energies (max of -E == -min of E):
 *   m_new(x_j) = min_{x_i} [ V(x_i, x_j) + E_i(x_i) + sum_{k in N(i)\j} m_ki(x_i) ],
 *   then shifted so that its minimum is 0 (the normalisation of min-sum). */
int oracle_min_edge_update(int M, const long long *E_i, int n_inc, const long long *const *inc,
                           const long long *V, long long *out) {
    long long *h = (long long *)malloc((size_t)M * sizeof(long long));
    if (!h) return -1;
    for (int x = 0; x < M; ++x) {
        long long s = E_i[x];
        for (int k = 0; k < n_inc; ++k) s += inc[k][x];
        h[x] = s;
    }
    long long lo = 0;
    for (int xj = 0; xj < M; ++xj) {
        long long best = V[xj] + h[0];
        for (int xi = 1; xi < M; ++xi) {
            long long v = V[(size_t)xi * M + xj] + h[xi];
            if (v < best) best = v;
        }
        out[xj] = best;
        if (xj == 0 || best < lo) lo = best;
    }
    free(h);
    for (int xj = 0; xj < M; ++xj) out[xj] -= lo;
    return 0;
}

static int min_update_edge(int e, int M, const int *src, const int *dst, const in_lists *L,
                           const long long *E, const long long *V, const long long *msg,
                           long long *out, const long long **scratch) {
    int i = src[e], j = dst[e], n = 0;
    for (int p = L->start[i]; p < L->start[i + 1]; ++p) {
        int e2 = L->edge[p];
        if (src[e2] != j) scratch[n++] = msg + (size_t)e2 * M;
    }
    return oracle_min_edge_update(M, E + (size_t)i * M, n, scratch, V, out);
}

int oracle_min_sum(int n_nodes, int M, int n_edges, const int *src, const int *dst,
                   const long long *E, const long long *V, const int *color, int schedule,
                   int n_iters, long long *msg) {
    if (check_graph(n_nodes, M, n_edges, src, dst) || n_iters < 0) return -1;
    if (schedule != 0 && schedule != 1) return -1;
    if (schedule == 1 && !color) return -1;
    in_lists L;
    if (build_in_lists(n_nodes, n_edges, dst, &L)) return -1;
    size_t sz = (size_t)n_edges * M;
    long long *next = (long long *)malloc((sz ? sz : 1) * sizeof(long long));
    const long long **scratch = (const long long **)malloc((size_t)(n_edges + 1) * sizeof(long long *));
    int rc = (next && scratch) ? 0 : -1;
    for (int t = 0; t < n_iters && rc == 0; ++t) {
        if (schedule == 0) {
            for (int e = 0; e < n_edges && rc == 0; ++e)
                rc = min_update_edge(e, M, src, dst, &L, E, V, msg, next + (size_t)e * M, scratch);
            if (rc == 0) memcpy(msg, next, sz * sizeof(long long));
        } else {
            for (int c = 0; c < 2 && rc == 0; ++c) {
                for (int e = 0; e < n_edges && rc == 0; ++e)
                    if (color[src[e]] == c)
                        rc = min_update_edge(e, M, src, dst, &L, E, V, msg, next + (size_t)e * M, scratch);
                for (int e = 0; e < n_edges && rc == 0; ++e)
                    if (color[src[e]] == c)
                        memcpy(msg + (size_t)e * M, next + (size_t)e * M, (size_t)M * sizeof(long long));
            }
        }
    }
    free(next);
    free(scratch);
    free_in_lists(&L);
    return rc;
}

/* Min-sum beliefs (negative-log form of Eq. 3, unnormalised):
 *   B_i(x) = E_i(x) + sum_{k in N(i)} m_ki(x). */
int oracle_min_beliefs(int n_nodes, int M, int n_edges, const int *dst, const long long *E,
                       const long long *msg, long long *belief) {
    memcpy(belief, E, (size_t)n_nodes * M * sizeof(long long));
    for (int e = 0; e < n_edges; ++e) {
        int j = dst[e];
        if (j < 0 || j >= n_nodes) return -1;
        for (int x = 0; x < M; ++x) belief[(size_t)j * M + x] += msg[(size_t)e * M + x];
    }
    return 0;
}
