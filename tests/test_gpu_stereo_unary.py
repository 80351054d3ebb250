"""The stereo unary formed on the device from the image pair (Sec. 6):
bp_set_unary_stereo against bp_set_unary of the same cost table (bit for
bit), and against the oracle's FP64 unary (Sec. 6's definition written out)
through the beliefs of the uniform state, which are the normalised unary."""
import numpy as np
import pytest

import oracle
from oracle import stereo
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _pair(cfg):
    import torch
    st = wl.make_stereo(cfg)
    return st, torch.from_numpy(st.left).cuda(), torch.from_numpy(st.right).cuda()


def _grids(cfg, dtype):
    """Two handles: the unary through bp_set_unary and through the images."""
    import torch
    from paper_1010_0012_gb300 import bp
    st, L, R = _pair(cfg)
    if dtype == bp.BP_F32:
        un, table = wl.unary_f32(st), wl.unary_table_f32(cfg)
        tab, fb = wl.pair_table_f32(cfg.alpha, cfg.T)
    else:
        un, table = wl.unary_i32(st), wl.unary_table_i32(cfg)
        tab, fb = wl.pair_table_i32(cfg.alpha, cfg.T)
    A = bp.BPGrid(cfg.W, cfg.H, cfg.M, dtype)
    A.set_unary(torch.from_numpy(un).cuda())
    B = bp.BPGrid(cfg.W, cfg.H, cfg.M, dtype)
    B.set_unary_stereo(L, R, table, cfg.Tu)
    for G in (A, B):
        G.set_potential(tab, cfg.T, fb)
        G.reset()
    return st, A, B


# W < M (labels past the right edge at every pixel), M not a multiple of 4
# (padded labels), M past the fast path's range, a ragged grid
SHAPES = [(23, 7, 16, 2), (9, 5, 37, 3), (40, 11, 64, 4), (13, 6, 130, 2), (70, 3, 600, 1)]


@pytest.mark.parametrize("W,Hh,M,T", SHAPES)
@pytest.mark.parametrize("mode", ["sum", "min"])
def test_stereo_unary_equals_the_uploaded_unary_bit_for_bit(W, Hh, M, T, mode):
    from paper_1010_0012_gb300 import bp
    dtype = bp.BP_F32 if mode == "sum" else bp.BP_I32
    cfg = wl.small_config("su", W, Hh, M, T, seed=W + M, noise_sigma=3.0)
    st, A, B = _grids(cfg, dtype)
    for n in (0, 3):
        A.iterate(n, None, "sync")
        B.iterate(n, None, "sync")
        ba, ma = A.beliefs()
        bb, mb = B.beliefs()
        A.sync()
        B.sync()
        assert np.array_equal(ba.cpu().numpy(), bb.cpu().numpy()), n
        assert np.array_equal(ma.cpu().numpy(), mb.cpu().numpy()), n
    assert np.array_equal(A.get_messages().cpu().numpy(), B.get_messages().cpu().numpy())
    A.close()
    B.close()


@pytest.mark.parametrize("W,Hh,M", [(23, 7, 16), (9, 5, 37), (13, 6, 130)])
def test_stereo_unary_matches_the_oracle_definition(W, Hh, M):
    """Uniform messages: the sum-product beliefs are g / sum_x g, and the
    min-sum beliefs are E_u itself, with g and E_u from Sec. 6's matching
    cost as the oracle writes it (FP64 exp)."""
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("so", W, Hh, M, 2, seed=3 * M, noise_sigma=3.0)
    st, A, B = _grids(cfg, bp.BP_F32)
    B.iterate(0, bp.BP_SUM, "sync")
    bel, mp = B.beliefs()
    B.sync()
    g64 = stereo.unary_potential(st.left, st.right, M, cfg.beta, cfg.Tu)
    b64 = g64 / g64.sum(-1, keepdims=True)
    assert H.node_rel_err(bel.cpu().numpy(), b64) <= H.REL_TOL
    A.close()
    B.close()
    st, A, B = _grids(cfg, bp.BP_I32)
    B.iterate(0, bp.BP_MAX, "sync")
    bel, mp = B.beliefs()
    B.sync()
    cost = stereo.matching_cost(st.left, st.right, M, cfg.Tu).astype(np.int64)
    q = int(round(wl.Q_ENERGY * cfg.beta))
    np.testing.assert_array_equal(bel.cpu().numpy().astype(np.int64), q * cost)
    np.testing.assert_array_equal(mp.cpu().numpy(), oracle.map_labels(q * cost, maximise=False))
    A.close()
    B.close()


def test_stereo_unary_argument_checks():
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("sa", 8, 4, 8, 1)
    st, L, R = _pair(cfg)
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32)
    with pytest.raises(ValueError):
        G.set_unary_stereo(L, R, np.ones(5, np.float32), 5)          # table of Tu entries, not Tu + 1
    with pytest.raises(bp.BPError) as ei:
        G.set_unary_stereo(L, R, np.ones(257, np.float32), 256)
    assert ei.value.status == bp.BP_ERR_ARG
    bad = np.ones(21, np.float32)
    bad[4] = -1.0
    with pytest.raises(bp.BPError) as ei:
        G.set_unary_stereo(L, R, bad, 20)
    assert ei.value.status == bp.BP_ERR_ARG
    bad[4] = np.inf
    with pytest.raises(bp.BPError) as ei:
        G.set_unary_stereo(L, R, bad, 20)
    assert ei.value.status == bp.BP_ERR_ARG
    G.close()
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_I32)
    with pytest.raises(bp.BPError) as ei:
        G.set_unary_stereo(L, R, np.full(21, 1 << 26, np.int32), 20)
    assert ei.value.status == bp.BP_ERR_ARG
    G.set_unary_stereo(L, R, np.arange(21, dtype=np.int32), 20)
    G.close()


def test_stereo_unary_at_the_benchmark_size():
    """1280 x 720, M = 128: the device-formed unary gives the uploaded unary's
    beliefs bit for bit after two synchronous iterations."""
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.CONFIGS["grid1280x720_m128"]
    st, A, B = _grids(cfg, bp.BP_F32)
    A.iterate(2, bp.BP_SUM, "sync")
    B.iterate(2, bp.BP_SUM, "sync")
    ba, ma = A.beliefs()
    bb, mb = B.beliefs()
    A.sync()
    B.sync()
    assert bool(torch.equal(ba, bb)) and bool(torch.equal(ma, mb))
    A.close()
    B.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_stereo_unary_from_host_images(pinned):
    """Host images (pinned or pageable) are copied by the library itself and
    give the device images' unary bit for bit, also when the host buffers are
    overwritten right after the call returns (the next call's images)."""
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("sh", 37, 11, 24, 2, seed=91, noise_sigma=3.0)
    st, L, R = _pair(cfg)
    other = wl.make_stereo(wl.small_config("sh2", 37, 11, 24, 2, seed=92, noise_sigma=3.0))
    table = wl.unary_table_f32(cfg)
    hl, hr = torch.from_numpy(st.left.copy()), torch.from_numpy(st.right.copy())
    if pinned:
        hl, hr = hl.pin_memory(), hr.pin_memory()
    tab, fb = wl.pair_table_f32(cfg.alpha, cfg.T)
    out = []
    for source in ("device", "host"):
        G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32)
        G.set_potential(tab, cfg.T, fb)
        if source == "device":
            G.set_unary_stereo(L, R, table, cfg.Tu)
        else:
            G.set_unary_stereo(hl, hr, table, cfg.Tu)
            G.sync()                       # the copies have run; reuse the host buffers
            hl.copy_(torch.from_numpy(other.left))
            hr.copy_(torch.from_numpy(other.right))
        G.reset()
        G.iterate(2, bp.BP_SUM, "sync")
        bel, mp = G.beliefs()
        G.sync()
        out.append((bel.cpu().numpy(), mp.cpu().numpy()))
        G.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
