"""Pins for the coarse-to-fine oracle."""
import numpy as np
import pytest

from oracle import grid, multiscale, stereo
from tests.test_oracle_pins import forward_backward, viterbi_min_marginals


def test_single_level_is_plain_bp():
    rng = np.random.default_rng(0)
    g = rng.uniform(0.05, 1.0, (6, 7, 5))
    F = stereo.pairwise_matrix(0.8, 1, 5)
    a = multiscale.multiscale_sum_product(g, F, [4])
    b = grid.grid_sum_product(g, F, 4)
    np.testing.assert_array_equal(a[1], b[1])


def test_coarse_unary_is_the_block_product_and_sum():
    u = np.arange(1, 3 * 3 * 2 + 1, dtype=np.float64).reshape(3, 3, 2)
    c = multiscale.coarsen(u, np.prod)
    assert c.shape == (2, 2, 2)
    np.testing.assert_array_equal(c[0, 0], u[0, 0] * u[0, 1] * u[1, 0] * u[1, 1])
    np.testing.assert_array_equal(c[0, 1], u[0, 2] * u[1, 2])
    np.testing.assert_array_equal(c[1, 0], u[2, 0] * u[2, 1])
    np.testing.assert_array_equal(c[1, 1], u[2, 2])
    e = multiscale.coarsen(u.astype(np.int64), np.sum)
    assert e[0, 1, 0] == u[0, 2, 0] + u[1, 2, 0]


def test_messages_start_from_the_parent_by_direction():
    Hc, Wc, M = 2, 2, 3
    pc = np.arange(4 * Hc * Wc * M, dtype=np.float64).reshape(4, Hc, Wc, M)
    fine = multiscale.upsample_messages(pc, 4, 4, -1.0)
    # (1, 2) sits in parent (0, 1), which has a left neighbour: from-left message copied
    np.testing.assert_array_equal(fine[0, 1, 2], pc[0, 0, 1])
    # (1, 1) sits in parent (0, 0), which has no left neighbour: uniform fill
    np.testing.assert_array_equal(fine[0, 1, 1], -1.0)
    # (2, 3) in parent (1, 1): up-neighbour exists, down does not
    np.testing.assert_array_equal(fine[2, 2, 3], pc[2, 1, 1])
    np.testing.assert_array_equal(fine[3, 2, 3], -1.0)


@pytest.mark.parametrize("W,H", [(13, 1), (1, 11)])
def test_coarse_start_does_not_change_the_exact_chain_result(W, H):
    """On a chain BP is exact after as many iterations as the chain is long,
    from any starting messages, so the coarse levels cannot change the result."""
    rng = np.random.default_rng(4)
    M = 5
    g = rng.uniform(0.05, 1.0, (H, W, M))
    F = stereo.pairwise_matrix(0.7, 1, M)
    _, bel = multiscale.multiscale_sum_product(g, F, [2, 3, max(W, H)])
    np.testing.assert_allclose(bel.reshape(-1, M), forward_backward(g.reshape(-1, M), F), rtol=1e-11)
    E = rng.integers(0, 20, (H, W, M))
    V = stereo.pairwise_energy_matrix(7, 1, M)
    _, b = multiscale.multiscale_min_sum(E, V, [3, 1, max(W, H)])
    ref = viterbi_min_marginals(E.reshape(-1, M), V)
    b = b.reshape(-1, M)
    np.testing.assert_array_equal(b - b.min(1, keepdims=True), ref - ref.min(1, keepdims=True))


def test_uniform_potential_at_every_level():
    rng = np.random.default_rng(3)
    g = rng.uniform(0.05, 1.0, (9, 10, 4))
    planes, bel = multiscale.multiscale_sum_product(g, stereo.pairwise_matrix(0.0, 1, 4), [2, 2, 2])
    np.testing.assert_allclose(bel, g / g.sum(-1, keepdims=True), rtol=1e-12)


def test_log_coarsening_is_the_block_product_up_to_scale():
    rng = np.random.default_rng(8)
    g = rng.uniform(0.1, 1.0, (5, 6, 4))
    prod = multiscale.coarsen(g, np.prod)
    lg = multiscale.coarsen_log(np.log(g))
    np.testing.assert_allclose(np.exp(lg), prod / prod.max(-1, keepdims=True), rtol=1e-13)
    assert np.all(lg.max(-1) == 0.0)


def test_per_node_unary_scale_does_not_change_bp():
    """The reason coarse unaries may be rescaled: scaling g_i by any positive
    constant leaves every normalised message and belief unchanged."""
    rng = np.random.default_rng(9)
    g = rng.uniform(0.05, 1.0, (4, 5, 6))
    F = stereo.pairwise_matrix(0.6, 2, 6)
    a = grid.grid_sum_product(g, F, 5)
    b = grid.grid_sum_product(g * rng.uniform(1e-3, 1e3, (4, 5, 1)), F, 5)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
    src, dst, side, rr, cc = grid.grid_edges(5, 4)
    np.testing.assert_allclose(a[0][side, rr, cc], b[0][side, rr, cc], rtol=1e-12)
