"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (the handle's default layout and grid, CUDA-graph issue of one launch
per synchronous iteration; the batch with its autotuned tiling):

* 1280 x 720, M = 128, T = 4, 100 sum-product iterations;
* the 64-MRF batch (W 128..640, H 128..480, M in 32..256, T 2..8) after 30
  iterations, min-sum int32 and sum-product FP32.

The oracle cannot run these grids whole.  It recomputes sampled message
updates one by one (Eq. 2 / Eq. 9) from the GPU's own state one iteration
earlier, and sampled beliefs (Eq. 3) from the final state.  A property
that holds at any size is checked everywhere: every sum-product message
sums to 1, every min-sum message has minimum 0."""
import numpy as np
import pytest

import oracle
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

SIDE = ((0, -1), (0, 1), (-1, 0), (1, 0))   # (dr, dc) of the neighbour on side s


def _sample_edges(W, Hh, n, rng):
    """n directed edges (r, c, t): node (r, c) sends towards side t."""
    out = []
    while len(out) < n:
        r, c, t = int(rng.integers(0, Hh)), int(rng.integers(0, W)), int(rng.integers(0, 4))
        dr, dc = SIDE[t]
        if 0 <= r + dr < Hh and 0 <= c + dc < W:
            out.append((r, c, t))
    return out


def _edge_inputs(node_planes, r, c, t, W, Hh):
    """Incoming messages of (r, c) ([4][M], by side) from every present side but t."""
    inc = []
    for s in range(4):
        dr, dc = SIDE[s]
        if s != t and 0 <= r + dr < Hh and 0 <= c + dc < W:
            inc.append(node_planes[s])
    return inc


def _node_inputs(planes, r, c, W, Hh):
    return _edge_inputs(planes, r, c, -1, W, Hh)


def _sampled(planes_dev, idx):
    """Host copies of planes[:, r, c] for the sampled nodes (dict by (r, c))."""
    import torch
    rs = torch.tensor([i[0] for i in idx], device=planes_dev.device)
    cs = torch.tensor([i[1] for i in idx], device=planes_dev.device)
    sub = planes_dev[:, rs, cs].cpu().numpy()            # [4][n][M]
    return {(int(r), int(c)): sub[:, k] for k, (r, c) in enumerate(idx)}


def _check_sum_edges(prev, nxt, g, F, edges, W, Hh):
    worst = 0.0
    for (r, c, t) in edges:
        inc = [m.astype(np.float64) for m in _edge_inputs(prev[(r, c)], r, c, t, W, Hh)]
        ref = oracle.sum_edge_update(g[r, c], inc, F)
        dr, dc = SIDE[t]
        got = nxt[(r + dr, c + dc)][t ^ 1].astype(np.float64)
        worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(ref)))
    assert worst <= H.REL_TOL, worst


def _check_min_edges(prev, nxt, E, V, edges, W, Hh):
    for (r, c, t) in edges:
        inc = [m.astype(np.int64) for m in _edge_inputs(prev[(r, c)], r, c, t, W, Hh)]
        ref = oracle.min_edge_update(E[r, c], inc, V)
        dr, dc = SIDE[t]
        np.testing.assert_array_equal(nxt[(r + dr, c + dc)][t ^ 1].astype(np.int64), ref)


def _edge_nodes(edges):
    """Sender and receiver nodes of the sampled edges."""
    nodes = set()
    for (r, c, t) in edges:
        dr, dc = SIDE[t]
        nodes.add((r, c))
        nodes.add((r + dr, c + dc))
    return sorted(nodes)


def _present_mask(W, Hh, torch):
    """[4][H][W] True where the slot has a neighbour."""
    m = torch.ones((4, Hh, W), dtype=torch.bool, device="cuda")
    m[0, :, 0] = False
    m[1, :, W - 1] = False
    m[2, 0, :] = False
    m[3, Hh - 1, :] = False
    return m


def test_grid1280x720_m128_100_sync_sampled():
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.CONFIGS["grid1280x720_m128"]
    st = wl.make_stereo(cfg)
    g = wl.unary_f32(st)
    tab, fbar = wl.pair_table_f32(cfg.alpha, cfg.T)
    F = H.oracle_F_from_table(tab, cfg.T, fbar, cfg.M)
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32)
    G.set_unary(torch.from_numpy(g).cuda())
    G.set_potential(tab, cfg.T, fbar)
    G.reset()
    G.iterate(cfg.iters - 1, bp.BP_SUM, "sync")
    p_prev = G.get_messages()
    G.iterate(1, bp.BP_SUM, "sync")
    p_last = G.get_messages()
    bel, mp = G.beliefs()
    G.sync()
    rng = np.random.default_rng(2024)
    edges = _sample_edges(cfg.W, cfg.H, 300, rng)
    nodes = _edge_nodes(edges)
    prev, last = _sampled(p_prev, nodes), _sampled(p_last, nodes)
    _check_sum_edges(prev, last, g, F, edges, cfg.W, cfg.H)

    # every present message of the final state sums to 1
    sums = p_last.sum(-1)
    present = _present_mask(cfg.W, cfg.H, torch)
    assert float((sums[present] - 1).abs().max()) <= 1e-5
    assert bool(torch.isfinite(p_last).all())

    # sampled beliefs (Eq. 3) and MAP labels of the final state
    bn = [(int(rng.integers(0, cfg.H)), int(rng.integers(0, cfg.W))) for _ in range(200)]
    fin = _sampled(p_last, bn)
    bel_s = bel[torch.tensor([x[0] for x in bn], device="cuda"), torch.tensor([x[1] for x in bn], device="cuda")]
    bel_s = bel_s.cpu().numpy()
    mp_s = mp[torch.tensor([x[0] for x in bn], device="cuda"), torch.tensor([x[1] for x in bn], device="cuda")]
    mp_s = mp_s.cpu().numpy()
    for k, (r, c) in enumerate(bn):
        inc = [m.astype(np.float64) for m in _node_inputs(fin[(r, c)], r, c, cfg.W, cfg.H)]
        b64 = oracle.sum_beliefs(np.zeros(len(inc), np.int32), g[r, c][None].astype(np.float64), np.stack(inc))[0]
        assert np.max(np.abs(bel_s[k] - b64)) / np.max(b64) <= H.REL_TOL
        srt = np.sort(b64)
        if (srt[-1] - srt[-2]) > 1e-4 * srt[-1]:
            assert mp_s[k] == oracle.map_labels(b64[None], maximise=True)[0]
    G.close()


@pytest.fixture(scope="module")
def batch64():
    return wl.make_batch(n=64)


@pytest.mark.parametrize("mode", ["min", "sum"])
def test_batch64_30_iterations_sampled(mode, batch64):
    import torch
    from paper_1010_0012_gb300 import bp
    items = batch64
    dtype = bp.BP_I32 if mode == "min" else bp.BP_F32
    bmode = bp.BP_MAX if mode == "min" else bp.BP_SUM
    descs, unaries, tables = [], [], []
    for it in items:
        if mode == "min":
            un = wl.unary_i32(it.stereo)
            tab, fb = wl.pair_table_i32(it.cfg.alpha, it.cfg.T)
        else:
            un = wl.unary_f32(it.stereo)
            tab, fb = wl.pair_table_f32(it.cfg.alpha, it.cfg.T)
        unaries.append(un)
        tables.append((tab, fb))
        descs.append((torch.from_numpy(un).cuda(), tab, it.cfg.T, fb))
    torch.cuda.synchronize()
    b = bp.bp_batch_create(descs, dtype)
    del descs
    bp.bp_batch_autotune(b, bmode, 8)          # as bench.py; leaves the uniform state
    bp.bp_batch_reset_messages(b)
    bp.bp_batch_iterate(b, 29, bmode)
    rng = np.random.default_rng(7 if mode == "min" else 8)
    picks = sorted(rng.choice(len(items), size=8, replace=False).tolist())
    tdt = torch.int32 if mode == "min" else torch.float32
    prev_dev = {}
    for k in picks:
        cfg = items[k].cfg
        pl = torch.empty((4, cfg.H, cfg.W, cfg.M), dtype=tdt, device="cuda")
        bp.bp_batch_get_messages(b, k, pl)
        prev_dev[k] = pl
    bp.bp_batch_iterate(b, 1, bmode)
    for k in picks:
        cfg = items[k].cfg
        pl = torch.empty((4, cfg.H, cfg.W, cfg.M), dtype=tdt, device="cuda")
        bp.bp_batch_get_messages(b, k, pl)
        bp.bp_batch_sync(b)
        edges = _sample_edges(cfg.W, cfg.H, 40, rng)
        nodes = _edge_nodes(edges)
        prev, last = _sampled(prev_dev[k], nodes), _sampled(pl, nodes)
        tab, fb = tables[k]
        present = _present_mask(cfg.W, cfg.H, torch)
        if mode == "min":
            V = H.oracle_V_from_table(tab, cfg.T, fb, cfg.M)
            _check_min_edges(prev, last, unaries[k], V, edges, cfg.W, cfg.H)
            assert int(pl.min(-1).values[present].abs().max()) == 0
        else:
            F = H.oracle_F_from_table(tab, cfg.T, fb, cfg.M)
            _check_sum_edges(prev, last, unaries[k], F, edges, cfg.W, cfg.H)
            assert float((pl.sum(-1)[present] - 1).abs().max()) <= 1e-5
    bp.bp_batch_destroy(b)
