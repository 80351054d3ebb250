"""Pins for the FP64 gradient oracle.

The torch forward (dense Eq. 2 on message planes) must equal the C oracle's
edge-list BP, which is itself pinned against brute force; the autograd
gradient must equal central finite differences."""
import numpy as np
import pytest

from oracle import gradient, grid, stereo
from paper_1010_0012_gb300 import workload as wl


def _small(W=9, H=7, M=8, T=2, seed=11):
    cfg = wl.small_config("g", W, H, M, T, structure="planar", seed=seed)
    return wl.make_stereo(cfg)


@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_torch_forward_matches_c_oracle(schedule):
    import torch
    st = _small()
    M, T, alpha, beta = st.cfg.M, st.cfg.T, 0.8, 0.1
    cost = st.cost.astype(np.float64)
    fbar = np.exp(-alpha * T)
    planes_t, bel_t = gradient.sum_product_planes(torch.tensor(-beta * cost), alpha, fbar, T, 6,
                                                  schedule)
    g = np.exp(-beta * cost)
    planes_c, bel_c = grid.grid_sum_product(g, stereo.pairwise_matrix(alpha, T, M), 6, schedule)
    np.testing.assert_allclose(bel_t.numpy(), bel_c, rtol=1e-12, atol=1e-15)
    src, dst, side, rr, cc = grid.grid_edges(st.cfg.W, st.cfg.H)
    np.testing.assert_allclose(planes_t.numpy()[side, rr, cc], planes_c[side, rr, cc], rtol=1e-12)


@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_autograd_matches_finite_differences(schedule):
    st = _small(W=7, H=6, M=6, T=2, seed=4)
    alpha, beta, T = 0.9, 0.1, st.cfg.T
    fbar = float(np.exp(-alpha * T))
    cost = st.cost.astype(np.float64)
    ref = gradient.reference_gradient(cost, st.d_gt, alpha, fbar, beta, T, 8, schedule)
    fd = gradient.finite_difference(cost, st.d_gt, alpha, fbar, beta, T, 8, schedule)
    for k in ("d_alpha", "d_fbar", "d_beta"):
        assert abs(ref[k] - fd[k]) <= 1e-6 * max(1.0, abs(fd[k])), (k, ref[k], fd[k])


def test_dlogg_matches_finite_difference_on_one_entry():
    import torch
    st = _small(W=5, H=4, M=5, T=1, seed=8)
    alpha, beta, T = 1.0, 0.1, 1
    fbar = float(np.exp(-alpha * T))
    cost = st.cost.astype(np.float64)
    ref = gradient.reference_gradient(cost, st.d_gt, alpha, fbar, beta, T, 5)
    r, c, x = 2, 3, 1
    h = 1e-6

    def loss_at(delta):
        logg = torch.tensor(-beta * cost)
        logg[r, c, x] += delta
        with torch.no_grad():
            return float(gradient.nll_loss(logg, alpha, fbar, T, 5, st.d_gt))
    fd = (loss_at(h) - loss_at(-h)) / (2 * h)
    assert abs(ref["d_logg"][r, c, x] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_table_parameterisation_chain_rule_matches_alpha_gradient():
    """d/d alpha through f(d) = exp(-alpha |d|) (chain rule on d/d f(d)) equals
    the direct d/d alpha; d/d fbar and d/d log g agree between the two forms."""
    st = _small(W=6, H=5, M=7, T=2, seed=21)
    alpha, beta, T = 0.8, 0.1, 2
    fbar = float(np.exp(-alpha * T))
    cost = st.cost.astype(np.float64)
    d = np.arange(-T, T + 1)
    table = np.exp(-alpha * np.abs(d))
    a = gradient.reference_gradient(cost, st.d_gt, alpha, fbar, beta, T, 5)
    b = gradient.reference_gradient_table(cost, st.d_gt, table, fbar, beta, T, 5)
    assert abs(a["loss"] - b["loss"]) <= 1e-12 * abs(a["loss"])
    chain = float(np.sum(b["d_table"] * -np.abs(d) * table))
    assert abs(chain - a["d_alpha"]) <= 1e-10 * max(1.0, abs(a["d_alpha"]))
    assert abs(b["d_fbar"] - a["d_fbar"]) <= 1e-10 * max(1.0, abs(a["d_fbar"]))
    np.testing.assert_allclose(b["d_logg"], a["d_logg"], rtol=1e-10, atol=1e-13)
