"""The allocation-free tensor-core iteration (bp_iterate_dense_tc_noalloc).

It exists for callers that cannot allocate device memory themselves (their
memory is planned by another component, or allocation is forbidden after
start-up), so its scratch is a fixed array inside the library.  This file is
collected last on purpose: a failure here leaves every other test already run.
The call must give what the handle-based bp_iterate_dense(BP_DENSE_BF16_TC)
gives, within the BF16 tolerance of the tensor-core tests, on two calls in a
row (the second call reuses the array the first one left behind), and it must
stay within that bound of the FP64 oracle too."""
import numpy as np
import pytest

from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -6 * 1.02     # the tensor-core tests' bound (BF16 h and f, FP32 accumulation)


def _handle_path(g, p0, tab, T, fbar, W, Hh, M, n):
    from paper_1010_0012_gb300 import bp
    G = bp.BPGrid(W, Hh, M, bp.BP_F32)
    G.set_unary(g)
    G.set_potential(tab, T, fbar)
    G.set_messages(p0)
    out = []
    for _ in range(n):
        G.iterate_dense(1, bp.BP_DENSE_BF16_TC)
        out.append(G.get_messages())
    G.sync()
    G.close()
    return out


def _rel(a, b, W, Hh):
    src, dst, side, rr, cc = grid.grid_edges(W, Hh)
    x = a.cpu().numpy().astype(np.float64)[side, rr, cc]
    y = b[side, rr, cc] if isinstance(b, np.ndarray) else b.cpu().numpy().astype(np.float64)[side, rr, cc]
    assert np.all(np.isfinite(x))
    return float(np.max(np.abs(x - y) / y))


def _absent_slots_are_zero(out, W, Hh):
    o = out.cpu().numpy()
    assert np.all(o[0, :, 0, :] == 0.0)        # no left neighbour in column 0
    assert np.all(o[1, :, W - 1, :] == 0.0)    # no right neighbour in the last column
    assert np.all(o[2, 0, :, :] == 0.0)        # no upper neighbour in row 0
    assert np.all(o[3, Hh - 1, :, :] == 0.0)   # no lower neighbour in the last row


@pytest.mark.parametrize("W,Hh,M,T,on_stream", [(24, 16, 128, 4, False), (37, 21, 64, 3, False),
                                                (19, 13, 64, 70, True)])
def test_no_alloc_matches_handle_path_and_oracle_twice(W, Hh, M, T, on_stream):
    """T = 70 >= M covers the clamp of the band to the M - 1 label differences
    that exist (a 141-entry table of which the middle 127 values are read)."""
    import torch
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(W + Hh + M + T)
    g_np = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    p0_np = H.random_planes_sum(W, Hh, M, rng)
    g = torch.from_numpy(g_np).cuda()
    p0 = torch.from_numpy(p0_np).cuda()
    tab, fbar = wl.pair_table_f32(0.5, T)
    ref1, ref2 = _handle_path(g, p0, tab, T, fbar, W, Hh, M, 2)

    out1 = torch.empty_like(p0)
    out2 = torch.empty_like(p0)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream() if on_stream else None
    bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, p0, out1, tab, T, fbar, stream=stream)
    bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, out1, out2, tab, T, fbar, stream=stream)
    torch.cuda.synchronize()

    assert _rel(out1, ref1, W, Hh) <= TOL
    assert _rel(out2, ref2, W, Hh) <= TOL
    _absent_slots_are_zero(out1, W, Hh)
    _absent_slots_are_zero(out2, W, Hh)

    # the first call against the FP64 oracle directly, from the same inputs
    F = H.oracle_F_from_table(tab, T, fbar, M)
    p64, _ = grid.grid_sum_product(g_np.astype(np.float64), F, 1, planes0=p0_np)
    assert _rel(out1, p64, W, Hh) <= TOL


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1010_0012_gb300 import bp
    W, Hh, M = 256, 256, 128          # 4*W*H*M*2 = 64 MiB > 32 MiB
    g = torch.ones((Hh, W, M), device="cuda")
    p = torch.ones((4, Hh, W, M), device="cuda")
    q = torch.empty_like(p)
    tab, fbar = wl.pair_table_f32(0.5, 4)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, p, q, tab, 4, fbar)
    assert ei.value.status == bp.BP_ERR_ARG
    assert "32 MiB" in str(ei.value)


def test_no_alloc_rejects_misaligned_and_overlapping_buffers():
    """Both are refused on the host before any launch, so nothing faults."""
    import torch
    from paper_1010_0012_gb300 import bp
    W, Hh, M = 8, 8, 64
    n = 4 * Hh * W * M
    g = torch.ones((Hh, W, M), device="cuda")
    big = torch.ones(2 * n + 8, device="cuda")
    p = big[:n].view(4, Hh, W, M)
    q_odd = big[n + 1:2 * n + 1].view(4, Hh, W, M)       # contiguous view 4 bytes past a 16-byte boundary
    tab, fbar = wl.pair_table_f32(0.5, 3)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, p, q_odd, tab, 3, fbar)
    assert ei.value.status == bp.BP_ERR_ARG and "aligned" in str(ei.value)
    q_overlap = big[n // 2:n // 2 + n].view(4, Hh, W, M)  # aligned, but half of it is the input
    with pytest.raises(bp.BPError) as ei:
        bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, p, q_overlap, tab, 3, fbar)
    assert ei.value.status == bp.BP_ERR_ARG and "overlap" in str(ei.value)
