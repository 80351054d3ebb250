"""The allocation-free tensor-core iteration (bp_iterate_dense_tc_noalloc).

It exists for callers that cannot allocate device memory themselves (their
memory is planned by another component, or allocation is forbidden after
start-up), so its scratch is a fixed array inside the library.  This file is
collected last on purpose: a failure here leaves every other test already run.
The call must give what the handle-based bp_iterate_dense(BP_DENSE_BF16_TC)
gives, within the BF16 tolerance of the tensor-core tests, on two calls in a
row (the second call reuses the array the first one left behind)."""
import numpy as np
import pytest

from oracle import grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
TOL = 2.0 ** -6 * 1.02     # the tensor-core tests' bound


@pytest.mark.parametrize("W,Hh,M,T", [(24, 16, 128, 4), (37, 21, 64, 3)])
def test_no_alloc_matches_handle_path_twice(W, Hh, M, T):
    import torch
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(W + Hh + M)
    g = torch.from_numpy(rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)).cuda()
    p0 = torch.from_numpy(H.random_planes_sum(W, Hh, M, rng)).cuda()
    tab, fbar = wl.pair_table_f32(0.5, T)

    G = bp.BPGrid(W, Hh, M, bp.BP_F32)
    G.set_unary(g)
    G.set_potential(tab, T, fbar)
    G.set_messages(p0)
    G.iterate_dense(1, bp.BP_DENSE_BF16_TC)
    ref1 = G.get_messages()
    G.iterate_dense(1, bp.BP_DENSE_BF16_TC)
    ref2 = G.get_messages()
    G.sync()
    G.close()

    out1 = torch.empty_like(p0)
    out2 = torch.empty_like(p0)
    torch.cuda.synchronize()
    bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, p0, out1, tab, T, fbar)
    bp.bp_iterate_dense_tc_noalloc(W, Hh, M, g, out1, out2, tab, T, fbar)
    torch.cuda.synchronize()

    src, dst, side, rr, cc = grid.grid_edges(W, Hh)
    for got, ref in ((out1, ref1), (out2, ref2)):
        a = got.cpu().numpy().astype(np.float64)[side, rr, cc]
        b = ref.cpu().numpy().astype(np.float64)[side, rr, cc]
        assert np.all(np.isfinite(a))
        assert float(np.max(np.abs(a - b) / b)) <= TOL


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
