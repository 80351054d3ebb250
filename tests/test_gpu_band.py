"""Parity of the O(mM) CUDA kernels (Eq. 7, Eq. 11) with the dense oracle.

Sum-product: FP32 against FP64 within 1e-5 relative per node (beliefs) and per
message.  Min-sum: int32 against exact int64, bit for bit."""
import numpy as np
import pytest

from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


# ---------------------------------------------------------- benchmark configs --

def test_grid32_m16_sum_and_min_10_sync():
    cfg = wl.CONFIGS["grid32_m16"]
    st, g, E = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    H.check_sum_case(g, tab, cfg.T, fbar, cfg.iters, "sync")
    tabi, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
    H.check_min_case(E, tabi, cfg.T, ebar, cfg.iters, "sync")


@pytest.mark.parametrize("mode", ["sum", "min"])
def test_grid384x288_m16_50_redblack(mode):
    cfg = wl.CONFIGS["grid384x288_m16"]
    st, g, E = H.stereo_inputs(cfg)
    if mode == "sum":
        tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
        H.check_sum_case(g, tab, cfg.T, fbar, cfg.iters, "redblack")
    else:
        tabi, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
        H.check_min_case(E, tabi, cfg.T, ebar, cfg.iters, "redblack")


# ------------------------------------------------------- sizes and band widths --

CASES = [(2, 0), (2, 1), (3, 1), (3, 2), (16, 0), (16, 1), (16, 2), (16, 15), (17, 2), (17, 16),
         (31, 3), (64, 3), (64, 8), (128, 4), (128, 8), (256, 2), (256, 5)]


@pytest.mark.parametrize("M,T", CASES)
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_one_iteration_from_injected_state(M, T, schedule):
    """One update of every message from the same random state, both modes."""
    rng = np.random.default_rng(M * 100 + T)
    W, Hh = 7, 5
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    tab, fbar = wl.pair_table_f32(0.7, T)
    H.check_sum_case(g, tab, T, fbar, 1, schedule, planes0=H.random_planes_sum(W, Hh, M, rng))
    E = rng.integers(0, 21, (Hh, W, M)).astype(np.int32)
    tabi, ebar = wl.pair_table_i32(0.7, T)
    H.check_min_case(E, tabi, T, ebar, 1, schedule, planes0=H.random_planes_min(W, Hh, M, rng))


@pytest.mark.parametrize("M,T", [(16, 2), (17, 3), (64, 3), (128, 4), (256, 8)])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_several_iterations_stereo(M, T, schedule):
    cfg = wl.small_config("s", 23, 13, M, T, alpha=0.8, structure="planar", seed=M + T)
    st, g, E = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, T)
    H.check_sum_case(g, tab, T, fbar, 6, schedule)
    tabi, ebar = wl.pair_table_i32(cfg.alpha, T)
    H.check_min_case(E, tabi, T, ebar, 6, schedule)


@pytest.mark.parametrize("W,Hh", [(1, 1), (1, 9), (11, 1), (2, 2), (3, 1), (1, 2)])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_degenerate_grids(W, Hh, schedule):
    rng = np.random.default_rng(W * 10 + Hh)
    M, T = 16, 2
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    tab, fbar = wl.pair_table_f32(1.0, T)
    H.check_sum_case(g, tab, T, fbar, 4, schedule)
    E = rng.integers(0, 21, (Hh, W, M)).astype(np.int32)
    tabi, ebar = wl.pair_table_i32(1.0, T)
    H.check_min_case(E, tabi, T, ebar, 4, schedule)


# ------------------------------------------------------------- general tables --

def test_asymmetric_table_and_f_below_fbar_sum():
    """Sum-product accepts any table (Sec. 4); d = x_i - x_j orientation."""
    rng = np.random.default_rng(9)
    M, T, W, Hh = 32, 3, 9, 6
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    tab = rng.uniform(0.01, 1.0, 2 * T + 1).astype(np.float32)
    fbar = 0.3     # some f(d) below fbar: negative band weights
    H.check_sum_case(g, tab, T, fbar, 3, "sync", planes0=H.random_planes_sum(W, Hh, M, rng))


def test_asymmetric_table_min():
    rng = np.random.default_rng(10)
    M, T, W, Hh = 32, 3, 9, 6
    E = rng.integers(0, 30, (Hh, W, M)).astype(np.int32)
    tab = rng.integers(0, 12, 2 * T + 1).astype(np.int32)
    H.check_min_case(E, tab, T, 12, 3, "redblack", planes0=H.random_planes_min(W, Hh, M, rng))


def test_pruned_potential_fbar_zero():
    """Eq. 8: fbar = 0 leaves only the band; exact when the table's fbar is 0."""
    rng = np.random.default_rng(11)
    M, T, W, Hh = 16, 2, 8, 8
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    tab, _ = wl.pair_table_f32(1.0, T)
    H.check_sum_case(g, tab, T, 0.0, 5, "sync")


@pytest.mark.parametrize("M,T", [(40, 12), (64, 63), (600, 3), (700, 20)])
def test_wide_band_and_large_label_count_generic_path(M, T):
    """T > 8 or M > 512 run on the shared-memory kernels."""
    rng = np.random.default_rng(M + T)
    W, Hh = 5, 4
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    tab, fbar = wl.pair_table_f32(0.2, T)
    H.check_sum_case(g, tab, T, fbar, 2, "sync", planes0=H.random_planes_sum(W, Hh, M, rng))
    E = rng.integers(0, 21, (Hh, W, M)).astype(np.int32)
    tabi, ebar = wl.pair_table_i32(0.5, T)
    H.check_min_case(E, tabi, T, ebar, 2, "redblack", planes0=H.random_planes_min(W, Hh, M, rng))


def test_t_beyond_label_range_is_dense():
    """T >= M - 1: the band covers all pairs, so Eq. 7 needs no fbar term."""
    rng = np.random.default_rng(12)
    M, T = 6, 9
    g = rng.uniform(0.05, 1.0, (4, 5, M)).astype(np.float32)
    tab = rng.uniform(0.1, 1.0, 2 * T + 1).astype(np.float32)
    H.check_sum_case(g, tab, T, 0.77, 3, "sync")


# ------------------------------------------------------------------ layouts --

@pytest.mark.parametrize("M,T", [(16, 2), (32, 4), (64, 3), (128, 4), (256, 8)])
def test_every_layout_agrees(M, T):
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(M)
    W, Hh = 9, 7
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    E = rng.integers(0, 21, (Hh, W, M)).astype(np.int32)
    tab, fbar = wl.pair_table_f32(0.6, T)
    tabi, ebar = wl.pair_table_i32(0.6, T)
    layouts = {(32, 1), (16, 2), (8, 1), (4, 2), (16, 1), (8, 2), (4, 1), (2, 2), (32, 2), (16, 4)}
    Mp = 4
    while Mp < M:
        Mp *= 2
    for L, C in sorted(layouts):
        if L * 4 * C != Mp:
            continue
        H.check_sum_case(g, tab, T, fbar, 3, "sync", layout=(L, C), persistent=0)
        H.check_min_case(E, tabi, T, ebar, 3, "sync", layout=(L, C), persistent=0)


# ------------------------------------------------------------- dense baselines --

@pytest.mark.parametrize("M,T", [(16, 2), (33, 3), (128, 4)])
def test_dense_cuda_core_baseline(M, T):
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("d", 12, 9, M, T, alpha=0.7, structure="planar", seed=M)
    st, g, E = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, T)
    H.check_sum_case(g, tab, T, fbar, 4, dense=bp.BP_DENSE_CUDA_CORE)
    tabi, ebar = wl.pair_table_i32(cfg.alpha, T)
    H.check_min_case(E, tabi, T, ebar, 4, dense=bp.BP_DENSE_CUDA_CORE)


# ------------------------------------------------------------------ errors -----

def test_max_mode_rejects_potential_below_fbar():
    from paper_1010_0012_gb300 import bp
    G = bp.BPGrid(4, 4, 8, bp.BP_I32)
    with pytest.raises(bp.BPError) as ei:
        G.set_potential(np.array([0, 5, 0], dtype=np.int32), 1, 4)   # E(0) = 5 > Ebar = 4
    assert ei.value.status == bp.BP_ERR_POTENTIAL
    with pytest.raises(bp.BPError) as ei:
        G.iterate(1)
    assert ei.value.status == bp.BP_ERR_STATE
    G.close()


def test_mode_dtype_mismatch_is_an_argument_error():
    from paper_1010_0012_gb300 import bp
    G = bp.BPGrid(4, 4, 8, bp.BP_F32)
    tab, fbar = wl.pair_table_f32(1.0, 2)
    G.set_potential(tab, 2, fbar)
    import torch
    G.set_unary(torch.ones((4, 4, 8), device="cuda"))
    with pytest.raises(bp.BPError) as ei:
        G.iterate(1, bp.BP_MAX)
    assert ei.value.status == bp.BP_ERR_ARG
    G.close()


# ------------------------------------------- per-launch vs persistent issue --

@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("M,T", [(16, 2), (33, 3), (64, 8), (128, 4), (256, 5)])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_both_issue_forms_match_the_oracle(persistent, M, T, schedule):
    """The same iterations issued one launch per (half-)iteration, or as one
    persistent launch with grid barriers between them."""
    cfg = wl.small_config("p", 29, 17, M, T, alpha=0.8, structure="planar", seed=M * 7 + T)
    st, g, E = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, T)
    H.check_sum_case(g, tab, T, fbar, 7, schedule, persistent=persistent)
    tabi, ebar = wl.pair_table_i32(cfg.alpha, T)
    H.check_min_case(E, tabi, T, ebar, 7, schedule, persistent=persistent)


def test_persistent_issue_is_one_launch_per_call():
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.CONFIGS["grid384x288_m16"]
    st, g, E = H.stereo_inputs(cfg)
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_I32)
    G.set_unary(torch.from_numpy(E).cuda())
    tabi, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
    G.set_potential(tabi, cfg.T, ebar)
    bp.bp_set_persistent(G.h, 1)
    G.reset()
    G.iterate(0, bp.BP_MAX)
    n0 = G.launches
    G.iterate(50, bp.BP_MAX, "redblack")
    assert G.launches - n0 == 1
    bp.bp_set_persistent(G.h, 0)
    n1 = G.launches
    G.iterate(50, bp.BP_MAX, "redblack")
    assert G.launches - n1 == 100
    G.sync()
    G.close()


@pytest.mark.parametrize("ebar", [16000, 16001, 90000])
@pytest.mark.parametrize("T", [3, 8])
def test_min_sum_16_bit_pairs_boundary_and_large_energies(ebar, T):
    """The 16-bit pair form of the min-sum band serves Ebar - min E(d) <= 16000
    (16000: pairs; 16001 and 90000: int32).  Large unaries and incoming
    messages make h exceed the clamp; every message must still equal the
    oracle's exactly."""
    rng = np.random.default_rng(ebar + T)
    M, W, Hh = 64, 9, 7
    tab = rng.integers(0, ebar + 1, 2 * T + 1).astype(np.int32)
    tab[T] = 0
    E = rng.integers(0, 60000, (Hh, W, M)).astype(np.int32)
    planes = H.random_planes_min(W, Hh, M, rng, hi=ebar)
    H.check_min_case(E, tab, T, ebar, 3, "sync", planes0=planes)
    H.check_min_case(E, tab, T, ebar, 2, "redblack", planes0=planes)
