"""Coarse-to-fine BP on the GPU against the multi-scale oracle (same levels,
same iterations): FP32 sum-product within 1e-5, int32 min-sum bit-exact."""
import numpy as np
import pytest

import oracle
from oracle import grid, multiscale
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _gpu(unary, dtype, table, T, fbar, iters, mode, schedule):
    import torch
    from paper_1010_0012_gb300 import bp
    Hh, W, M = unary.shape
    G = bp.BPGrid(W, Hh, M, dtype)
    G.set_unary(torch.from_numpy(unary).cuda())
    G.set_potential(table, T, fbar)
    bp.bp_iterate_multiscale(G.h, iters, mode, schedule)
    bel, mp = G.beliefs()
    pl = G.get_messages()
    G.sync()
    out = bel.cpu().numpy(), mp.cpu().numpy(), pl.cpu().numpy()
    G.close()
    return out


@pytest.mark.parametrize("W,Hh,M,T,iters", [(37, 23, 16, 2, [4, 3, 3]), (64, 48, 64, 3, [5, 3, 2, 2]),
                                             (21, 9, 128, 4, [3, 3])])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_multiscale_matches_oracle(W, Hh, M, T, iters, schedule):
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("ms", W, Hh, M, T, alpha=0.8, structure="voronoi", seed=W + M, noise_sigma=3.0)
    st, g, E = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, T)
    bel, mp, pl = _gpu(g, bp.BP_F32, tab, T, fbar, iters, bp.BP_SUM, schedule)
    F = H.oracle_F_from_table(tab, T, fbar, M)
    p64, b64 = multiscale.multiscale_sum_product(g.astype(np.float64), F, iters, schedule)
    assert H.node_rel_err(bel, b64) <= H.REL_TOL
    assert H.message_rel_err(pl, p64, W, Hh) <= H.REL_TOL
    tabi, ebar = wl.pair_table_i32(cfg.alpha, T)
    bel, mp, pl = _gpu(E, bp.BP_I32, tabi, T, ebar, iters, bp.BP_MAX, schedule)
    V = H.oracle_V_from_table(tabi, T, ebar, M)
    p64, b64 = multiscale.multiscale_min_sum(E.astype(np.int64), V, iters, schedule)
    np.testing.assert_array_equal(bel.astype(np.int64), b64)
    src, dst, side, rr, cc = grid.grid_edges(W, Hh)
    np.testing.assert_array_equal(pl.astype(np.int64)[side, rr, cc], p64[side, rr, cc])
    np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))


def test_one_level_is_bp_iterate():
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("ms1", 19, 17, 32, 3, structure="planar", seed=4)
    st, g, E = H.stereo_inputs(cfg)
    tabi, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
    a = _gpu(E, bp.BP_I32, tabi, cfg.T, ebar, [6], bp.BP_MAX, "sync")
    b = H.run_gpu_min(E, tabi, cfg.T, ebar, 6, "sync")
    np.testing.assert_array_equal(a[0], b[0])


def test_deep_pyramid_keeps_the_coarse_unaries_in_range():
    """Six levels on 1280 x 720 (the coarsest node covers 32 x 32 pixels, a
    product of 1024 unaries): every level must stay finite and the fine result
    must match the oracle's."""
    from paper_1010_0012_gb300 import bp
    import dataclasses
    cfg = dataclasses.replace(wl.CONFIGS["grid1280x720_m128"], W=160, H=96)
    st, g, E = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    iters = [4, 3, 3, 2, 2, 2]
    bel, mp, pl = _gpu(g, bp.BP_F32, tab, cfg.T, fbar, iters, bp.BP_SUM, "sync")
    assert np.all(np.isfinite(bel))
    F = H.oracle_F_from_table(tab, cfg.T, fbar, cfg.M)
    p64, b64 = multiscale.multiscale_sum_product(g.astype(np.float64), F, iters, "sync")
    assert H.node_rel_err(bel, b64) <= H.REL_TOL
