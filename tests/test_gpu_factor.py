"""Factor-graph BP with sparse three-variable factors (Sec. 7) against the
dense factor-BP oracle: FP32 sum-product within 1e-5, int32 min-sum exact;
and the O(M^3) comparison kernel against the same oracle."""
import numpy as np
import pytest

from oracle import factor
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def random_graph(n_vars, n_factors, rng):
    fs = []
    while len(fs) < n_factors:
        v = rng.choice(n_vars, size=3, replace=False)
        fs.append(tuple(int(x) for x in v))
    return np.array(fs, np.int32)


def random_triplets(M, C, rng):
    flat = rng.choice(M * M * M, size=C, replace=False)
    return np.stack([flat // (M * M), (flat // M) % M, flat % M], axis=1).astype(np.int32)


def _gpu(unary, factors, trip, vals, fbar, iters, dtype, dense=False):
    import torch
    from paper_1010_0012_gb300 import bp
    nv, M = unary.shape
    g = bp.bp_fg_create(nv, M, factors, dtype)
    bp.bp_fg_set_unary(g, torch.from_numpy(unary).cuda())
    bp.bp_fg_set_factor(g, trip, vals, fbar, dtype)
    bp.bp_fg_reset_messages(g)
    mode = bp.BP_SUM if dtype == bp.BP_F32 else bp.BP_MAX
    (bp.bp_fg_iterate_dense if dense else bp.bp_fg_iterate)(g, iters, mode)
    bel = torch.empty((nv, M), dtype=torch.float32 if dtype == bp.BP_F32 else torch.int32, device="cuda")
    mp = torch.empty((nv,), dtype=torch.int32, device="cuda")
    msg = torch.empty((len(factors), 3, M), dtype=bel.dtype, device="cuda")
    bp.bp_fg_beliefs(g, bel, mp)
    bp.bp_fg_get_messages(g, msg)
    bp.bp_fg_sync(g)
    out = bel.cpu().numpy(), mp.cpu().numpy(), msg.cpu().numpy()
    bp.bp_fg_destroy(g)
    return out


@pytest.mark.parametrize("M,C", [(4, 20), (8, 60), (16, 300), (33, 500)])
@pytest.mark.parametrize("dense", [False, True])
def test_factor_sum_matches_oracle(M, C, dense):
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(M + C)
    nv, nf = 40, 30
    fs = random_graph(nv, nf, rng)
    g = rng.uniform(0.05, 1.0, (nv, M)).astype(np.float32)
    trip = random_triplets(M, C, rng)
    vals = rng.uniform(0.2, 3.0, C).astype(np.float32)
    fbar = 0.15
    bel, mp, msg = _gpu(g, fs, trip, vals, fbar, 5, bp.BP_F32, dense)
    F = factor.dense_table(trip, vals.astype(np.float64), fbar, M)
    m64, b64 = factor.sum_product(g.astype(np.float64), fs, F, 5)
    assert H.node_rel_err(bel, b64) <= H.REL_TOL
    assert float(np.max(np.abs(msg - m64).max(-1) / np.abs(m64).max(-1))) <= H.REL_TOL


@pytest.mark.parametrize("M,C", [(4, 20), (8, 60), (16, 300), (33, 500)])
@pytest.mark.parametrize("dense", [False, True])
def test_factor_min_sum_bit_exact(M, C, dense):
    import oracle
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(100 + M + C)
    nv, nf = 40, 30
    fs = random_graph(nv, nf, rng)
    E = rng.integers(0, 25, (nv, M)).astype(np.int32)
    trip = random_triplets(M, C, rng)
    ebar = 12
    vals = rng.integers(0, ebar + 1, C).astype(np.int32)
    bel, mp, msg = _gpu(E, fs, trip, vals, ebar, 5, bp.BP_I32, dense)
    V = factor.dense_table(trip, vals.astype(np.int64), ebar, M, dtype=np.int64)
    m64, b64 = factor.min_sum(E.astype(np.int64), fs, V, 5)
    np.testing.assert_array_equal(msg.astype(np.int64), m64)
    np.testing.assert_array_equal(bel.astype(np.int64), b64)
    np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))


def test_factor_rejects_energy_above_ebar_and_bad_factors():
    import torch
    from paper_1010_0012_gb300 import bp
    g = bp.bp_fg_create(5, 4, [(0, 1, 2)], bp.BP_I32)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_fg_set_factor(g, [(0, 0, 0)], [9], 5, bp.BP_I32)
    assert ei.value.status == bp.BP_ERR_POTENTIAL
    bp.bp_fg_destroy(g)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_fg_create(5, 4, [(0, 1, 1)], bp.BP_I32)
    assert ei.value.status == bp.BP_ERR_ARG


@pytest.mark.parametrize("hub_degree", [5, 9, 16])
def test_factor_hub_variable_degrees(hub_degree):
    """One variable in hub_degree factors (the largest degree bound the
    variable-to-factor kernel is compiled for is 16), the others in few:
    sum-product within 1e-5 and min-sum exact against the dense oracle."""
    import oracle
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(hub_degree)
    M, nv = 12, 3 + 2 * hub_degree
    fs = np.array([(0, 1 + 2 * i, 2 + 2 * i) for i in range(hub_degree)] + [(1, 2, 3)], np.int32)
    trip = random_triplets(M, 150, rng)
    g = rng.uniform(0.05, 1.0, (nv, M)).astype(np.float32)
    vals = rng.uniform(0.2, 3.0, len(trip)).astype(np.float32)
    bel, mp, msg = _gpu(g, fs, trip, vals, 0.15, 4, bp.BP_F32)
    F = factor.dense_table(trip, vals.astype(np.float64), 0.15, M)
    m64, b64 = factor.sum_product(g.astype(np.float64), fs, F, 4)
    assert H.node_rel_err(bel, b64) <= H.REL_TOL
    E = rng.integers(0, 25, (nv, M)).astype(np.int32)
    vi = rng.integers(0, 13, len(trip)).astype(np.int32)
    bel, mp, msg = _gpu(E, fs, trip, vi, 12, 4, bp.BP_I32)
    V = factor.dense_table(trip, vi.astype(np.int64), 12, M, dtype=np.int64)
    m64, b64 = factor.min_sum(E.astype(np.int64), fs, V, 4)
    np.testing.assert_array_equal(msg.astype(np.int64), m64)
    np.testing.assert_array_equal(bel.astype(np.int64), b64)
    np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))


def second_difference_triplets(M, alpha=1.0):
    """The benchmark's smoothness potential: f = exp(-alpha |x0 - 2 x1 + x2|)
    where the second difference is at most 1.  Its middle slot's lists run
    from 3 to ~3M entries, so the balanced deal splits long lists across lanes."""
    x0, x1, x2 = np.meshgrid(np.arange(M), np.arange(M), np.arange(M), indexing="ij")
    d2 = np.abs(x0 - 2 * x1 + x2)
    keep = d2 <= 1
    trip = np.stack([x0[keep], x1[keep], x2[keep]], 1).astype(np.int32)
    return trip, d2[keep]


@pytest.mark.parametrize("M", [32, 70])
def test_factor_uneven_lists_sum_and_min_sum(M):
    """Uneven lists (split across lane pairs) and, at M = 70, 3 chunks of 32
    labels served by the 4-chunk kernel: sum-product within 1e-5 of the FP64
    oracle, min-sum bit for bit."""
    import oracle
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(M)
    nv, nf = 30, 24
    fs = random_graph(nv, nf, rng)
    trip, d2 = second_difference_triplets(M)
    vals = np.exp(-d2.astype(np.float64)).astype(np.float32)
    fbar = float(np.float32(np.exp(-2.0)))
    g = rng.uniform(0.05, 1.0, (nv, M)).astype(np.float32)
    bel, mp, msg = _gpu(g, fs, trip, vals, fbar, 4, bp.BP_F32)
    F = factor.dense_table(trip, vals.astype(np.float64), fbar, M)
    m64, b64 = factor.sum_product(g.astype(np.float64), fs, F, 4)
    assert H.node_rel_err(bel, b64) <= H.REL_TOL
    assert float(np.max(np.abs(msg - m64).max(-1) / np.abs(m64).max(-1))) <= H.REL_TOL
    E = rng.integers(0, 25, (nv, M)).astype(np.int32)
    ebar = 4
    vi = (2 * d2).astype(np.int32)
    bel, mp, msg = _gpu(E, fs, trip, vi, ebar, 4, bp.BP_I32)
    V = factor.dense_table(trip, vi.astype(np.int64), ebar, M, dtype=np.int64)
    m64, b64 = factor.min_sum(E.astype(np.int64), fs, V, 4)
    np.testing.assert_array_equal(msg.astype(np.int64), m64)
    np.testing.assert_array_equal(bel.astype(np.int64), b64)
    np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))
