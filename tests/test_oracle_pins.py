"""Pins for the oracle: checks against things other than itself.

* brute-force enumeration of Eq. 1 on small trees, where BP is exact
  (sum-product marginals, min-sum min-marginals);
* textbook forward-backward and Viterbi recursions on chains;
* special cases with closed forms (f = 1 everywhere, the two-colour
  schedule on a three-node chain, T >= M - 1);
* structural invariants of the 4-connected grid.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import grid, stereo


# ---------------------------------------------------------------- helpers ----

def random_tree(n, rng):
    parent = [-1] + [int(rng.integers(0, k)) for k in range(1, n)]
    und = [(parent[k], k) for k in range(1, n)]
    src = [a for a, b in und] + [b for a, b in und]
    dst = [b for a, b in und] + [a for a, b in und]
    depth = [0] * n
    for k in range(1, n):
        depth[k] = depth[parent[k]] + 1
    return np.array(src), np.array(dst), und, np.array([d % 2 for d in depth])


def sym_positive(M, rng):
    A = rng.uniform(0.05, 1.0, (M, M))
    return 0.5 * (A + A.T)


def brute_marginals(n, M, und, g, F):
    P = np.zeros((n, M))
    for x in itertools.product(range(M), repeat=n):
        w = np.prod([g[i, x[i]] for i in range(n)]) * np.prod([F[x[a], x[b]] for a, b in und])
        for i in range(n):
            P[i, x[i]] += w
    return P / P.sum(axis=1, keepdims=True)


def brute_min_marginals(n, M, und, Eu, V):
    best = np.full((n, M), np.iinfo(np.int64).max)
    for x in itertools.product(range(M), repeat=n):
        e = sum(int(Eu[i, x[i]]) for i in range(n)) + sum(int(V[x[a], x[b]]) for a, b in und)
        for i in range(n):
            best[i, x[i]] = min(best[i, x[i]], e)
    return best


def forward_backward(g, F):
    """Exact chain marginals by the textbook alpha/beta recursions."""
    n, M = g.shape
    a = np.zeros((n, M))
    b = np.ones((n, M))
    a[0] = g[0] / g[0].sum()
    for t in range(1, n):
        a[t] = g[t] * (a[t - 1] @ F)
        a[t] /= a[t].sum()
    for t in range(n - 2, -1, -1):
        b[t] = F @ (g[t + 1] * b[t + 1])
        b[t] /= b[t].sum()
    p = a * b
    return p / p.sum(axis=1, keepdims=True)


def viterbi_min_marginals(Eu, V):
    """Exact chain min-marginals from forward and backward min-plus passes."""
    n, M = Eu.shape
    fw = np.zeros((n, M), dtype=np.int64)
    bw = np.zeros((n, M), dtype=np.int64)
    fw[0] = Eu[0]
    for t in range(1, n):
        fw[t] = Eu[t] + np.min(fw[t - 1][:, None] + V, axis=0)
    for t in range(n - 2, -1, -1):
        bw[t] = np.min(V + (Eu[t + 1] + bw[t + 1])[None, :], axis=1)
    return fw + bw


# ------------------------------------------------------------- trees (exact) --

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_sum_product_exact_on_trees(seed, schedule):
    rng = np.random.default_rng(seed)
    n, M = int(rng.integers(3, 8)), int(rng.integers(2, 4))
    src, dst, und, col = random_tree(n, rng)
    g = rng.uniform(0.05, 1.0, (n, M))
    F = sym_positive(M, rng)
    msg = oracle.sum_product(src, dst, g, F, n_iters=n, color=col, schedule=schedule)
    bel = oracle.sum_beliefs(dst, g, msg)
    np.testing.assert_allclose(bel, brute_marginals(n, M, und, g, F), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_min_sum_exact_on_trees(seed, schedule):
    rng = np.random.default_rng(100 + seed)
    n, M = int(rng.integers(3, 8)), int(rng.integers(2, 4))
    src, dst, und, col = random_tree(n, rng)
    Eu = rng.integers(0, 20, (n, M))
    A = rng.integers(0, 15, (M, M))
    V = np.minimum(A, A.T)
    msg = oracle.min_sum(src, dst, Eu, V, n_iters=n, color=col, schedule=schedule)
    bel = oracle.min_beliefs(dst, Eu, msg)
    ref = brute_min_marginals(n, M, und, Eu, V)
    # messages are shifted to min 0, so beliefs equal min-marginals up to a per-node constant
    np.testing.assert_array_equal(bel - bel.min(axis=1, keepdims=True),
                                  ref - ref.min(axis=1, keepdims=True))
    # and the MAP labels (lowest-label ties) agree with the brute-force MAP
    np.testing.assert_array_equal(oracle.map_labels(bel, maximise=False),
                                  np.argmin(ref, axis=1))


# ---------------------------------------------------------- chains (closed) ---

@pytest.mark.parametrize("W,H", [(12, 1), (1, 9)])
def test_grid_chain_matches_forward_backward(W, H):
    rng = np.random.default_rng(5)
    M = 6
    g = rng.uniform(0.05, 1.0, (H, W, M))
    F = stereo.pairwise_matrix(0.7, 2, M)
    _, bel = grid.grid_sum_product(g, F, n_iters=max(W, H))
    ref = forward_backward(g.reshape(-1, M), F)
    np.testing.assert_allclose(bel.reshape(-1, M), ref, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("W,H", [(15, 1), (1, 11)])
def test_grid_chain_matches_viterbi(W, H):
    rng = np.random.default_rng(6)
    M = 7
    Eu = rng.integers(0, 21, (H, W, M))
    V = stereo.pairwise_energy_matrix(10, 2, M)
    _, bel = grid.grid_min_sum(Eu, V, n_iters=max(W, H))
    ref = viterbi_min_marginals(Eu.reshape(-1, M), V)
    b = bel.reshape(-1, M)
    np.testing.assert_array_equal(b - b.min(1, keepdims=True), ref - ref.min(1, keepdims=True))


# ---------------------------------------------------------- special cases -----

def test_uniform_potential_gives_unary_beliefs_on_loopy_grid():
    """alpha = 0 makes f identically 1: every message is uniform and the
    beliefs are the normalised unaries, on any graph."""
    rng = np.random.default_rng(1)
    H, W, M = 5, 6, 5
    g = rng.uniform(0.05, 1.0, (H, W, M))
    planes, bel = grid.grid_sum_product(g, stereo.pairwise_matrix(0.0, 2, M), n_iters=4)
    np.testing.assert_allclose(bel, g / g.sum(-1, keepdims=True), rtol=1e-13)
    src, dst, side, rr, cc = grid.grid_edges(W, H)
    np.testing.assert_allclose(planes[side, rr, cc], 1.0 / M, rtol=1e-13)


def test_redblack_is_exact_on_three_chain_after_one_iteration():
    """On the chain 0-1-2 the colour-0 half-step sends the exact leaf
    messages, which the colour-1 half-step then uses: one two-colour
    iteration is exact, one synchronous iteration is not, two are."""
    rng = np.random.default_rng(2)
    M = 4
    g = rng.uniform(0.05, 1.0, (1, 3, M))
    F = stereo.pairwise_matrix(0.9, 1, M)
    ref = brute_marginals(3, M, [(0, 1), (1, 2)], g[0], F)
    _, b_rb = grid.grid_sum_product(g, F, n_iters=1, schedule="redblack")
    np.testing.assert_allclose(b_rb[0], ref, rtol=1e-12)
    _, b_s1 = grid.grid_sum_product(g, F, n_iters=1, schedule="sync")
    assert np.max(np.abs(b_s1[0] - ref)) > 1e-4
    _, b_s2 = grid.grid_sum_product(g, F, n_iters=2, schedule="sync")
    np.testing.assert_allclose(b_s2[0], ref, rtol=1e-12)


def test_truncated_potential_is_constant_plus_band():
    """The stereo potential has the sparse compatibility property: outside
    |d| <= T it equals fbar = exp(-alpha T) (Sec. 1)."""
    for alpha, T, M in [(1.0, 2, 16), (0.5, 4, 40), (0.3, 0, 5)]:
        F = stereo.pairwise_matrix(alpha, T, M)
        d = np.arange(-T, T + 1)
        band = np.exp(-alpha * np.abs(d))
        np.testing.assert_array_equal(F, stereo.compatibility_matrix(band, T, np.exp(-alpha * T), M))


def test_grid_structure():
    for W, H in [(1, 1), (1, 5), (7, 1), (6, 4), (13, 9)]:
        src, dst, side, rr, cc = grid.grid_edges(W, H)
        assert src.size == 2 * (H * (W - 1) + W * (H - 1))
        r1, c1 = src // W, src % W
        r2, c2 = dst // W, dst % W
        assert np.all(np.abs(r1 - r2) + np.abs(c1 - c2) == 1)
        pairs = set(zip(src.tolist(), dst.tolist()))
        assert len(pairs) == src.size and all((b, a) in pairs for a, b in pairs)
        for s, (dr, dc) in enumerate(grid.SIDE_OFFSETS):
            m = side == s
            assert np.all(r1[m] == r2[m] + dr) and np.all(c1[m] == c2[m] + dc)
        col = grid.redblack_colors(W, H)
        assert np.all(col[src] != col[dst])


def test_matching_cost_definition_matches_workload_generator():
    """The stereo unary of Sec. 6, stated independently here and in the
    workload module, gives the same cost volume and the same float32 g."""
    from paper_1010_0012_gb300 import workload as wl
    cfg = wl.small_config("t", 37, 11, 16, 2, noise_sigma=3.0, structure="voronoi")
    st = wl.make_stereo(cfg)
    np.testing.assert_array_equal(st.cost.astype(np.int64),
                                  stereo.matching_cost(st.left, st.right, cfg.M, cfg.Tu))
    np.testing.assert_array_equal(wl.unary_f32(st),
                                  stereo.unary_potential(st.left, st.right, cfg.M, cfg.beta,
                                                         cfg.Tu).astype(np.float32))
    # where the true disparity is inside the image and there is no noise, cost is zero there
    cfg0 = wl.small_config("t0", 40, 9, 16, 2, structure="rectangles")
    st0 = wl.make_stereo(cfg0)
    rr, cc = np.meshgrid(np.arange(9), np.arange(40), indexing="ij")
    inside = cc + st0.d_gt < 40
    assert np.all(st0.cost[rr[inside], cc[inside], st0.d_gt[inside]] == 0)


def test_sampled_updates_agree_with_full_iteration():
    rng = np.random.default_rng(3)
    H, W, M = 4, 5, 6
    g = rng.uniform(0.05, 1.0, (H, W, M))
    F = stereo.pairwise_matrix(0.8, 2, M)
    p0, _ = grid.grid_sum_product(g, F, n_iters=2)
    p1, _ = grid.grid_sum_product(g, F, n_iters=1, planes0=p0)
    samples = [(1, 2, 0), (0, 0, 1), (3, 4, 2), (2, 1, 3)]
    got = grid.sampled_sum_updates(g, F, p0, samples)
    for (r, c, t), m in zip(samples, got):
        dr, dc = grid.SIDE_OFFSETS[t]
        np.testing.assert_allclose(m, p1[grid.OPPOSITE[t], r + dr, c + dc], rtol=1e-14)


def test_sparse_lists_of_a_band_give_the_band_matrix():
    """A sparse-compatibility potential listing |x_i - x_j| <= T for every x_j
    is the truncated band potential."""
    M, T = 11, 2
    band = np.array([0.3, 0.7, 1.0, 0.6, 0.2])
    rowptr, cols, vals = [0], [], []
    for xj in range(M):
        for d in range(-T, T + 1):
            if 0 <= xj + d < M:
                cols.append(xj + d)
                vals.append(band[d + T])
        rowptr.append(len(cols))
    np.testing.assert_array_equal(stereo.sparse_compatibility_matrix(rowptr, cols, vals, 0.05, M),
                                  stereo.compatibility_matrix(band, T, 0.05, M))


@pytest.mark.parametrize("M", [2, 3, 7])
def test_two_node_mrf_closed_form(M):
    """Two nodes joined by one edge with an asymmetric table: after one
    iteration the message 0 -> 1 is sum_{x_0} f(x_0, x_1) g_0(x_0) (Eq. 2
    with no other incoming message), normalised, and the message 1 -> 0 is
    sum_{x_1} f(x_1, x_0) g_1(x_1): the table is indexed (sender, receiver).
    Node 1's belief is then its exact marginal g_1(x_1) sum_{x_0} g_0 f /Z,
    and min-sum gives the exact min-marginal E_1(x_1) + min_{x_0} [E_0 + V]."""
    rng = np.random.default_rng(M)
    src, dst = np.array([0, 1]), np.array([1, 0])
    g = rng.uniform(0.05, 1.0, (2, M))
    F = rng.uniform(0.1, 2.0, (M, M))                 # F[x_sender, x_receiver]
    msg = oracle.sum_product(src, dst, g, F, 1)
    m01 = g[0] @ F
    m10 = g[1] @ F
    np.testing.assert_allclose(msg[0], m01 / m01.sum(), rtol=1e-13)
    np.testing.assert_allclose(msg[1], m10 / m10.sum(), rtol=1e-13)
    bel = oracle.sum_beliefs(dst, g, msg)
    joint = g[0][:, None] * g[1][None, :] * F        # P(x_0, x_1) with the edge's f(x_0, x_1)
    np.testing.assert_allclose(bel[1], joint.sum(0) / joint.sum(), rtol=1e-12)

    Eu = rng.integers(0, 30, (2, M))
    V = rng.integers(0, 20, (M, M))                   # V[x_sender, x_receiver]
    msg = oracle.min_sum(src, dst, Eu, V, 1)
    u01 = np.min(Eu[0][:, None] + V, axis=0)
    np.testing.assert_array_equal(msg[0], u01 - u01.min())
    bel = oracle.min_beliefs(dst, Eu, msg)
    ref = Eu[1] + np.min(Eu[0][:, None] + V, axis=0)
    np.testing.assert_array_equal(bel[1] - bel[1].min(), ref - ref.min())
