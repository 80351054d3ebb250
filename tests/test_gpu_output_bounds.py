"""Every call that writes into a caller's buffer writes that buffer whole and
nothing around it.  With compute-sanitizer closed, this is the check for
out-of-range writes that needs no fault: the output is a view in the middle
of a larger device buffer filled with a canary pattern, and after the call the
margins must still hold the canary while no element of the view may.

Outputs covered: beliefs and MAP (linear, log and int32), message planes,
the adjoint's d log g, the batch's beliefs and planes, and the factor graph's
beliefs and messages.  The shapes have padded label counts (M not a multiple
of the kernels' label groups), so an unpadding bug would show."""
import math

import numpy as np
import pytest

from paper_1010_0012_gb300 import workload as wl

pytestmark = pytest.mark.gpu

CANARY = 0x5A5AA5A5          # as float32 about 1.5e16: no belief, message or adjoint
PAD = 4096                   # canary elements on each side (16 KB)


class Guarded:
    def __init__(self, shape, dtype):
        import torch
        self.n = math.prod(shape)
        self.full = torch.full((self.n + 2 * PAD,), CANARY, dtype=torch.int32, device="cuda")
        inner = self.full[PAD:PAD + self.n]
        self.view = (inner.view(torch.float32) if dtype == torch.float32 else inner).view(shape)

    def check(self, what):
        torch_full = self.full
        assert bool((torch_full[:PAD] == CANARY).all()), f"{what}: write before the buffer"
        assert bool((torch_full[PAD + self.n:] == CANARY).all()), f"{what}: write past the buffer"
        assert not bool((torch_full[PAD:PAD + self.n] == CANARY).any()), f"{what}: element not written"


def _tensors(dtype_name):
    import torch
    return torch.float32 if dtype_name == "f32" else torch.int32


@pytest.mark.parametrize("dtype_name", ["f32", "i32"])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_grid_outputs_stay_in_their_buffers(dtype_name, schedule):
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("ob", 7, 5, 13, 2, seed=17, noise_sigma=3.0)
    st = wl.make_stereo(cfg)
    dtype = bp.BP_F32 if dtype_name == "f32" else bp.BP_I32
    td = _tensors(dtype_name)
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, dtype)
    if dtype == bp.BP_F32:
        G.set_unary(torch.from_numpy(wl.unary_f32(st)).cuda())
        tab, fb = wl.pair_table_f32(cfg.alpha, cfg.T)
    else:
        G.set_unary(torch.from_numpy(wl.unary_i32(st)).cuda())
        tab, fb = wl.pair_table_i32(cfg.alpha, cfg.T)
    G.set_potential(tab, cfg.T, fb)
    G.reset()
    G.iterate(3, None, schedule)
    bel, mp = Guarded((cfg.H, cfg.W, cfg.M), td), Guarded((cfg.H, cfg.W), torch.int32)
    planes = Guarded((4, cfg.H, cfg.W, cfg.M), td)
    bp.bp_beliefs(G.h, bel.view, mp.view)
    # absent neighbours' planes are written too (uniform messages), so the
    # whole [4][H][W][M] view is output
    bp.bp_get_messages(G.h, planes.view)
    G.sync()
    bel.check("bp_beliefs")
    mp.check("bp_beliefs map")
    planes.check("bp_get_messages")
    G.close()


def test_log_beliefs_and_adjoint_stay_in_their_buffers():
    import torch
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("oa", 9, 6, 21, 3, seed=5, noise_sigma=3.0)
    st = wl.make_stereo(cfg)
    logg = torch.from_numpy(np.log(wl.unary_f32(st).astype(np.float64)).astype(np.float32)).cuda()
    tab, fb = wl.pair_table_f32(cfg.alpha, cfg.T)
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32)
    bp.bp_set_unary_log(G.h, logg)
    bp.bp_set_potential(G.h, tab, cfg.T, fb, bp.BP_F32)
    bp.bp_set_checkpoint_interval(G.h, 2)
    bp.bp_reset_messages(G.h)
    bp.bp_iterate(G.h, 5, bp.BP_SUM | bp.BP_LOG | bp.BP_RECORD, bp.BP_SYNC)
    logb = Guarded((cfg.H, cfg.W, cfg.M), torch.float32)
    bp.bp_beliefs(G.h, logb.view)
    dlogb = torch.from_numpy(np.random.default_rng(3).standard_normal((cfg.H, cfg.W, cfg.M)).astype(np.float32)).cuda()
    dlogg = Guarded((cfg.H, cfg.W, cfg.M), torch.float32)
    dtab, dfbar = bp.bp_backward(G.h, dlogb, dlogg.view, 2 * cfg.T + 1)
    G.sync()
    logb.check("bp_beliefs (log)")
    dlogg.check("bp_backward d log g")
    assert np.all(np.isfinite(dtab)) and np.isfinite(dfbar)
    G.close()


@pytest.mark.parametrize("dtype_name", ["f32", "i32"])
def test_batch_outputs_stay_in_their_buffers(dtype_name):
    import torch
    from paper_1010_0012_gb300 import bp
    dtype = bp.BP_F32 if dtype_name == "f32" else bp.BP_I32
    td = _tensors(dtype_name)
    cfgs = [wl.small_config("b0", 11, 6, 13, 2, seed=1), wl.small_config("b1", 5, 9, 37, 4, seed=2)]
    descs, keep = [], []
    for cfg in cfgs:
        st = wl.make_stereo(cfg)
        if dtype == bp.BP_F32:
            un = torch.from_numpy(wl.unary_f32(st)).cuda()
            tab, fb = wl.pair_table_f32(cfg.alpha, cfg.T)
        else:
            un = torch.from_numpy(wl.unary_i32(st)).cuda()
            tab, fb = wl.pair_table_i32(cfg.alpha, cfg.T)
        keep.append(un)
        descs.append((un, tab, cfg.T, fb))
    b = bp.bp_batch_create(descs, dtype)
    bp.bp_batch_reset_messages(b)
    bp.bp_batch_iterate(b, 3, bp.BP_SUM if dtype == bp.BP_F32 else bp.BP_MAX)
    outs = []
    for k, cfg in enumerate(cfgs):
        bel, mp = Guarded((cfg.H, cfg.W, cfg.M), td), Guarded((cfg.H, cfg.W), torch.int32)
        planes = Guarded((4, cfg.H, cfg.W, cfg.M), td)
        bp.bp_batch_beliefs(b, k, bel.view, mp.view)
        bp.bp_batch_get_messages(b, k, planes.view)
        outs.append((k, bel, mp, planes))
    bp.bp_batch_sync(b)
    for k, bel, mp, planes in outs:
        bel.check(f"bp_batch_beliefs {k}")
        mp.check(f"bp_batch_beliefs map {k}")
        planes.check(f"bp_batch_get_messages {k}")
    bp.bp_batch_destroy(b)


@pytest.mark.parametrize("dtype_name", ["f32", "i32"])
def test_factor_graph_outputs_stay_in_their_buffers(dtype_name):
    import torch
    from paper_1010_0012_gb300 import bp
    dtype = bp.BP_F32 if dtype_name == "f32" else bp.BP_I32
    td = _tensors(dtype_name)
    rng = np.random.default_rng(11)
    nv, M = 10, 7
    factors = [(0, 1, 2), (2, 3, 4), (4, 5, 6), (6, 7, 8), (1, 8, 9)]
    flat = rng.choice(M * M * M, size=40, replace=False)
    trip = np.stack([flat // (M * M), (flat // M) % M, flat % M], axis=1).astype(np.int32)
    if dtype == bp.BP_F32:
        unary = rng.uniform(0.1, 1.0, (nv, M)).astype(np.float32)
        vals, fbar = rng.uniform(0.3, 1.0, len(trip)).astype(np.float32), 0.1
    else:
        unary = rng.integers(0, 20, (nv, M)).astype(np.int32)
        vals, fbar = rng.integers(0, 8, len(trip)).astype(np.int32), 9
    g = bp.bp_fg_create(nv, M, factors, dtype)
    bp.bp_fg_set_unary(g, torch.from_numpy(unary).cuda())
    bp.bp_fg_set_factor(g, trip, vals, fbar, dtype)
    bp.bp_fg_reset_messages(g)
    bp.bp_fg_iterate(g, 3, bp.BP_SUM if dtype == bp.BP_F32 else bp.BP_MAX)
    bel, mp = Guarded((nv, M), td), Guarded((nv,), torch.int32)
    msg = Guarded((len(factors), 3, M), td)
    bp.bp_fg_beliefs(g, bel.view, mp.view)
    bp.bp_fg_get_messages(g, msg.view)
    bp.bp_fg_sync(g)
    bel.check("bp_fg_beliefs")
    mp.check("bp_fg_beliefs map")
    msg.check("bp_fg_get_messages")
    bp.bp_fg_destroy(g)
