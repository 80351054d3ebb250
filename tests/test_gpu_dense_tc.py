"""The O(M^2) tensor-core baseline (Eq. 2 as a BF16 tcgen05 GEMM with FP32
accumulation) against the FP64 oracle.

Tolerance from the arithmetic: h and f are each rounded once to BF16
(relative error <= 2^-8 each), all terms are non-negative, so every
unnormalised entry is within 2^-7 relative and the normalised message within
2 * 2^-7 = 2^-6 of the exact one (FP32 accumulation adds far less)."""
import numpy as np
import pytest

from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -6 * 1.02


def _one_step(W, Hh, M, T, alpha, seed, fused=False):
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    planes0 = H.random_planes_sum(W, Hh, M, rng)
    tab, fbar = wl.pair_table_f32(alpha, T)
    kind = bp.BP_DENSE_BF16_TC_FUSED if fused else bp.BP_DENSE_BF16_TC
    bel, mp, msgs = H.run_gpu_sum(g, tab, T, fbar, 1, planes0=planes0, dense=kind)
    F = H.oracle_F_from_table(tab, T, fbar, M)
    p64, _ = grid.grid_sum_product(g.astype(np.float64), F, 1, planes0=planes0)
    src, dst, side, rr, cc = grid.grid_edges(W, Hh)
    a = msgs.astype(np.float64)[side, rr, cc]
    b = p64[side, rr, cc]
    rel = np.abs(a - b) / b
    return float(rel.max())


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("W,Hh,M,T", [(9, 7, 128, 4), (13, 5, 64, 3), (11, 6, 100, 4), (200, 100, 128, 4),
                                      (1, 37, 128, 2), (45, 1, 64, 2),
                                      # 256 labels: the K-block ring kernels (88 tiles, a ragged tail; 200 -> 256)
                                      (70, 40, 256, 8), (13, 9, 256, 4), (11, 6, 200, 6), (1, 41, 256, 3)])
def test_one_iteration_within_bf16_bound(W, Hh, M, T, fused):
    err = _one_step(W, Hh, M, T, 0.5, seed=W * Hh + M, fused=fused)
    assert err <= TOL, f"max relative error {err:.4e} > {TOL:.4e}"


@pytest.mark.parametrize("fused", [False, True])
def test_several_iterations_map_agrees_where_clear(fused):
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("tc", 40, 24, 128, 4, alpha=0.5, structure="slanted", seed=3)
    st, g, _ = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    bel, mp, _ = H.run_gpu_sum(g, tab, cfg.T, fbar, 8,
                               dense=bp.BP_DENSE_BF16_TC_FUSED if fused else bp.BP_DENSE_BF16_TC)
    F = H.oracle_F_from_table(tab, cfg.T, fbar, cfg.M)
    _, b64 = grid.grid_sum_product(g.astype(np.float64), F, 8)
    top2 = np.sort(b64, -1)[..., -2:]
    clear = (top2[..., 1] - top2[..., 0]) > 0.1 * top2[..., 1]
    assert clear.mean() > 0.5
    assert np.array_equal(mp[clear], np.argmax(b64, -1)[clear])
    assert H.node_rel_err(bel, b64) < 0.1


def test_unsupported_label_count_is_reported():
    from paper_1010_0012_gb300 import bp
    import torch
    G = bp.BPGrid(4, 4, 16, bp.BP_F32)
    G.set_unary(torch.ones((4, 4, 16), device="cuda"))
    tab, fbar = wl.pair_table_f32(1.0, 2)
    G.set_potential(tab, 2, fbar)
    with pytest.raises(bp.BPError) as ei:
        G.iterate_dense(1, bp.BP_DENSE_BF16_TC)
    assert ei.value.status == bp.BP_ERR_UNSUPPORTED
    G.close()


@pytest.mark.parametrize("M,T", [(128, 4), (256, 6)])
def test_fused_and_packed_forms_agree_bit_for_bit(M, T):
    """Both forms round the same h to BF16 and run the same MMAs, so the
    messages agree exactly."""
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(17 + M)
    W, Hh = 33, 21
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    p0 = H.random_planes_sum(W, Hh, M, rng)
    tab, fbar = wl.pair_table_f32(0.5, T)
    _, _, a = H.run_gpu_sum(g, tab, T, fbar, 2, planes0=p0, dense=bp.BP_DENSE_BF16_TC)
    _, _, b = H.run_gpu_sum(g, tab, T, fbar, 2, planes0=p0, dense=bp.BP_DENSE_BF16_TC_FUSED)
    src, dst, side, rr, cc = grid.grid_edges(W, Hh)
    np.testing.assert_array_equal(a[side, rr, cc], b[side, rr, cc])
