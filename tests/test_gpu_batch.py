"""Batched O(mM) BP: many MRFs of uneven size, label count and band width in
one persistent launch, against the oracle run on each MRF alone."""
import numpy as np
import pytest

import oracle
from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _mrfs(n=7, seed=3, label_counts=(16, 32, 64, 100, 128, 256)):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        M = int(rng.choice(label_counts))
        T = int(rng.integers(0, 9))
        W, Hh = int(rng.integers(3, 23)), int(rng.integers(2, 17))
        alpha = float(rng.uniform(0.25, 1.0))
        cfg = wl.small_config(f"b{k}", W, Hh, M, T, alpha=alpha, structure="planar", seed=100 + k)
        out.append((cfg, wl.make_stereo(cfg)))
    return out


def _run_batch(mrfs, dtype, iters, family=None, tile=None, calls=1):
    import torch
    from paper_1010_0012_gb300 import bp
    descs, keep = [], []
    for cfg, st in mrfs:
        if dtype == bp.BP_F32:
            un = torch.from_numpy(wl.unary_f32(st)).cuda()
            tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
        else:
            un = torch.from_numpy(wl.unary_i32(st)).cuda()
            tab, fbar = wl.pair_table_i32(cfg.alpha, cfg.T)
        keep.append(un)
        descs.append((un, tab, cfg.T, fbar))
    b = bp.bp_batch_create(descs, dtype)
    if family is not None:
        bp.bp_batch_set_tiling(b, family, tile)
    bp.bp_batch_reset_messages(b)
    for _ in range(calls):
        bp.bp_batch_iterate(b, iters, bp.BP_SUM if dtype == bp.BP_F32 else bp.BP_MAX)
    outs = []
    for k, (cfg, st) in enumerate(mrfs):
        bel = torch.empty((cfg.H, cfg.W, cfg.M), dtype=torch.float32 if dtype == bp.BP_F32 else torch.int32,
                          device="cuda")
        mp = torch.empty((cfg.H, cfg.W), dtype=torch.int32, device="cuda")
        pl = torch.empty((4, cfg.H, cfg.W, cfg.M), dtype=bel.dtype, device="cuda")
        bp.bp_batch_beliefs(b, k, bel, mp)
        bp.bp_batch_get_messages(b, k, pl)
        outs.append((bel, mp, pl))
    bp.bp_batch_sync(b)
    res = [(x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy()) for x, y, z in outs]
    launches = bp.bp_batch_launch_count(b)
    bp.bp_batch_destroy(b)
    return res, launches


def _check_sum(mrfs, res, iters):
    for (cfg, st), (bel, mp, pl) in zip(mrfs, res):
        g = wl.unary_f32(st)
        tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
        F = H.oracle_F_from_table(tab, cfg.T, fbar, cfg.M)
        p64, b64 = grid.grid_sum_product(g.astype(np.float64), F, iters)
        assert H.node_rel_err(bel, b64) <= H.REL_TOL, cfg
        assert H.message_rel_err(pl, p64, cfg.W, cfg.H) <= H.REL_TOL, cfg
        H.check_sum_map(mp, bel, b64)


def _check_min(mrfs, res, iters):
    for (cfg, st), (bel, mp, pl) in zip(mrfs, res):
        E = wl.unary_i32(st)
        tab, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
        V = H.oracle_V_from_table(tab, cfg.T, ebar, cfg.M)
        p64, b64 = grid.grid_min_sum(E.astype(np.int64), V, iters)
        src, dst, side, rr, cc = grid.grid_edges(cfg.W, cfg.H)
        np.testing.assert_array_equal(pl.astype(np.int64)[side, rr, cc], p64[side, rr, cc])
        np.testing.assert_array_equal(bel.astype(np.int64), b64)
        np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))


@pytest.mark.parametrize("family,tile", [(1, 512), (2, 2048), (1, 65536)])
def test_batch_sum_matches_oracle(family, tile):
    from paper_1010_0012_gb300 import bp
    mrfs = _mrfs()
    res, _ = _run_batch(mrfs, bp.BP_F32, 6, family, tile)
    _check_sum(mrfs, res, 6)


@pytest.mark.parametrize("family,tile", [(1, 512), (2, 4096)])
def test_batch_min_matches_oracle_bit_exact(family, tile):
    from paper_1010_0012_gb300 import bp
    mrfs = _mrfs(seed=4)
    res, _ = _run_batch(mrfs, bp.BP_I32, 6, family, tile)
    _check_min(mrfs, res, 6)


def test_graph_replay_continues_the_iteration():
    """Two calls of 3 iterations (the second a replay of the captured graph
    with the other start buffer) equal 6 iterations."""
    from paper_1010_0012_gb300 import bp
    mrfs = _mrfs(n=5, seed=5)
    res, launches = _run_batch(mrfs, bp.BP_I32, 3, 2, 1024, calls=2)
    _check_min(mrfs, res, 6)


def test_one_launch_per_iterate_call():
    from paper_1010_0012_gb300 import bp
    import torch
    mrfs = _mrfs(n=4, seed=6)
    descs = []
    for cfg, st in mrfs:
        un = torch.from_numpy(wl.unary_i32(st)).cuda()
        tab, e = wl.pair_table_i32(cfg.alpha, cfg.T)
        descs.append((un, tab, cfg.T, e))
    b = bp.bp_batch_create(descs, bp.BP_I32)
    bp.bp_batch_iterate(b, 1, bp.BP_MAX)        # materialises the start state
    n0 = bp.bp_batch_launch_count(b)
    bp.bp_batch_iterate(b, 30, bp.BP_MAX)
    assert bp.bp_batch_launch_count(b) - n0 == 1
    bp.bp_batch_sync(b)
    bp.bp_batch_destroy(b)


def test_barrier_time_out_is_reported_and_the_context_survives():
    """The barrier waits for one block that does not exist; every wait runs
    out after 50 ms, the kernel ends, bp_batch_sync reports BP_ERR_TIMEOUT and
    the same batch then runs correctly."""
    import torch
    from paper_1010_0012_gb300 import bp
    mrfs = _mrfs(n=4, seed=7)
    descs = []
    for cfg, st in mrfs:
        un = torch.from_numpy(wl.unary_i32(st)).cuda()
        tab, e = wl.pair_table_i32(cfg.alpha, cfg.T)
        descs.append((un, tab, cfg.T, e))
    b = bp.bp_batch_create(descs, bp.BP_I32)
    bp.bp_batch_set_wait_limit(b, 0.05, 1)
    bp.bp_batch_reset_messages(b)
    bp.bp_batch_iterate(b, 4, bp.BP_MAX)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_batch_sync(b)
    assert ei.value.status == bp.BP_ERR_TIMEOUT
    bp.bp_batch_set_wait_limit(b, 2.0, 0)
    bp.bp_batch_reset_messages(b)
    bp.bp_batch_iterate(b, 4, bp.BP_MAX)
    bp.bp_batch_sync(b)
    for k, (cfg, st) in enumerate(mrfs):
        bel = torch.empty((cfg.H, cfg.W, cfg.M), dtype=torch.int32, device="cuda")
        bp.bp_batch_beliefs(b, k, bel)
        bp.bp_batch_sync(b)
        tab, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
        V = H.oracle_V_from_table(tab, cfg.T, ebar, cfg.M)
        _, b64 = grid.grid_min_sum(wl.unary_i32(st).astype(np.int64), V, 4)
        np.testing.assert_array_equal(bel.cpu().numpy().astype(np.int64), b64)
    bp.bp_batch_destroy(b)


def H_padded(M):
    mp = 16
    while mp < M:
        mp *= 2
    return mp


@pytest.mark.parametrize("dtype_name", ["i32", "f32"])
def test_classes_with_different_lane_layouts_in_one_launch(dtype_name):
    """Each (Mp, T) class on its own family and item size: the launch mixes
    both lane layouts and stays exact (min-sum bit for bit, sum-product
    within 1e-5 of the FP64 oracle)."""
    import torch
    from paper_1010_0012_gb300 import bp
    mrfs = _mrfs(n=8, seed=21)
    dtype = bp.BP_I32 if dtype_name == "i32" else bp.BP_F32
    descs, keep = [], []
    for cfg, st in mrfs:
        if dtype == bp.BP_F32:
            un = torch.from_numpy(wl.unary_f32(st)).cuda()
            tab, fb = wl.pair_table_f32(cfg.alpha, cfg.T)
        else:
            un = torch.from_numpy(wl.unary_i32(st)).cuda()
            tab, fb = wl.pair_table_i32(cfg.alpha, cfg.T)
        keep.append(un)
        descs.append((un, tab, cfg.T, fb))
    b = bp.bp_batch_create(descs, dtype)
    n = bp.bp_batch_class_count(b)
    assert n >= 2
    for k in range(n):
        Mp, T, _, _ = bp.bp_batch_get_class_tiling(b, k)
        bp.bp_batch_set_class_tiling(b, Mp, T, 1 + k % 2, 512 * (1 + k))
    got = [bp.bp_batch_get_class_tiling(b, k) for k in range(n)]
    assert [g[2:] for g in got] == [(1 + k % 2, 512 * (1 + k)) for k in range(n)]
    with pytest.raises(bp.BPError) as ei:
        bp.bp_batch_set_class_tiling(b, 48, 3, 1, 4096)
    assert ei.value.status == bp.BP_ERR_ARG
    with pytest.raises(bp.BPError) as ei:
        bp.bp_batch_get_class_tiling(b, n)
    assert ei.value.status == bp.BP_ERR_ARG
    bp.bp_batch_reset_messages(b)
    bp.bp_batch_iterate(b, 3, bp.BP_MAX if dtype == bp.BP_I32 else bp.BP_SUM)
    bp.bp_batch_iterate(b, 3, bp.BP_MAX if dtype == bp.BP_I32 else bp.BP_SUM)
    res = []
    for k, (cfg, st) in enumerate(mrfs):
        bel = torch.empty((cfg.H, cfg.W, cfg.M), dtype=torch.float32 if dtype == bp.BP_F32 else torch.int32,
                          device="cuda")
        mp = torch.empty((cfg.H, cfg.W), dtype=torch.int32, device="cuda")
        pl = torch.empty((4, cfg.H, cfg.W, cfg.M), dtype=bel.dtype, device="cuda")
        bp.bp_batch_beliefs(b, k, bel, mp)
        bp.bp_batch_get_messages(b, k, pl)
        res.append((bel, mp, pl))
    bp.bp_batch_sync(b)
    res = [(x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy()) for x, y, z in res]
    bp.bp_batch_destroy(b)
    if dtype == bp.BP_I32:
        _check_min(mrfs, res, 6)
    else:
        _check_sum(mrfs, res, 6)


def test_autotune_picks_a_candidate_and_stays_exact(tmp_path, monkeypatch):
    import torch
    from paper_1010_0012_gb300 import bp
    monkeypatch.setenv("BP_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    mrfs = _mrfs(n=6, seed=8)
    descs = []
    for cfg, st in mrfs:
        un = torch.from_numpy(wl.unary_i32(st)).cuda()
        tab, e = wl.pair_table_i32(cfg.alpha, cfg.T)
        descs.append((un, tab, cfg.T, e))
    b = bp.bp_batch_create(descs, bp.BP_I32)
    ms = bp.bp_batch_autotune(b, bp.BP_MAX, 2)
    assert ms > 0
    fam, tile = bp.bp_batch_get_tiling(b)
    assert fam in (1, 2) and tile in (16384, 65536, 262144)
    classes = [bp.bp_batch_get_class_tiling(b, k) for k in range(bp.bp_batch_class_count(b))]
    want = sorted({(H_padded(cfg.M), min(cfg.T, cfg.M - 1)) for cfg, st in mrfs})
    assert [c[:2] for c in classes] == want
    assert all(f in (1, 2) and t in (16384, 65536, 262144) for _, _, f, t in classes)
    assert (tmp_path / "tune.txt").read_text().strip()
    bp.bp_batch_iterate(b, 5, bp.BP_MAX)
    bp.bp_batch_sync(b)
    cfg, st = mrfs[0]
    bel = torch.empty((cfg.H, cfg.W, cfg.M), dtype=torch.int32, device="cuda")
    bp.bp_batch_beliefs(b, 0, bel)
    bp.bp_batch_sync(b)
    tab, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
    V = H.oracle_V_from_table(tab, cfg.T, ebar, cfg.M)
    _, b64 = grid.grid_min_sum(wl.unary_i32(st).astype(np.int64), V, 5)
    np.testing.assert_array_equal(bel.cpu().numpy().astype(np.int64), b64)
    # a second autotune reads the cache
    b2 = bp.bp_batch_create(descs, bp.BP_I32)
    bp.bp_batch_autotune(b2, bp.BP_MAX, 2)
    assert bp.bp_batch_get_tiling(b2) == (fam, tile)
    assert [bp.bp_batch_get_class_tiling(b2, k) for k in range(bp.bp_batch_class_count(b2))] == classes
    bp.bp_batch_destroy(b)
    bp.bp_batch_destroy(b2)


def test_batch_rejects_potential_below_fbar_in_max_mode():
    import torch
    from paper_1010_0012_gb300 import bp
    un = torch.zeros((4, 5, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(bp.BPError) as ei:
        bp.bp_batch_create([(un, np.array([0, 9, 0], dtype=np.int32), 1, 5)], bp.BP_I32)
    assert ei.value.status == bp.BP_ERR_POTENTIAL


@pytest.mark.parametrize("family", [1, 2])
def test_batch_min_power_of_two_labels_bit_exact(family):
    """Every MRF with M a power of two: the batch runs the kernel variant
    without padded-label masks (the others above include M = 100)."""
    mrfs = _mrfs(n=6, seed=11, label_counts=(16, 32, 64, 128, 256))
    res, _ = _run_batch(mrfs, H.bp().BP_I32, 6, family=family, tile=2048)
    _check_min(mrfs, res, 6)


@pytest.mark.parametrize("family", [1, 2])
def test_batch_sum_power_of_two_labels(family):
    mrfs = _mrfs(n=6, seed=12, label_counts=(16, 32, 64, 128, 256))
    res, _ = _run_batch(mrfs, H.bp().BP_F32, 6, family=family, tile=2048)
    _check_sum(mrfs, res, 6)
