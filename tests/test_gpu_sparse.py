"""General sparse compatibility (Sec. 4, Sec. 7): arbitrary per-label lists of
compatible states, including potentials that are not a function of
x_i - x_j, against the dense oracle built from the same lists."""
import numpy as np
import pytest

import oracle
from oracle import grid, stereo
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def random_pattern(M, max_per_row, rng, integer=False, ebar=40):
    rowptr, cols, vals = [0], [], []
    for xj in range(M):
        k = int(rng.integers(0, max_per_row + 1))
        xs = rng.choice(M, size=k, replace=False)
        cols.extend(int(x) for x in xs)
        if integer:
            vals.extend(int(v) for v in rng.integers(0, ebar + 1, k))
        else:
            vals.extend(float(v) for v in rng.uniform(0.05, 2.0, k))
        rowptr.append(len(cols))
    return (np.array(rowptr, np.int32), np.array(cols, np.int32),
            np.array(vals, np.int32 if integer else np.float32))


KERNELS = ["lists", "registers"]


def _run(M, dtype, planes0, unary, pattern, fbar, iters, schedule, kernel="auto"):
    """kernel: "lists", "registers" (the call asserts that it is the one that
    runs) or "auto"."""
    import torch
    from paper_1010_0012_gb300 import bp
    Hh, W, _ = unary.shape
    G = bp.BPGrid(W, Hh, M, dtype)
    G.set_unary(torch.from_numpy(unary).cuda())
    bp.bp_set_potential_sparse(G.h, *pattern, fbar, dtype)
    if kernel != "auto":
        want = bp.BP_SPARSE_LISTS if kernel == "lists" else bp.BP_SPARSE_REGISTERS
        bp.bp_set_sparse_kernel(G.h, want)
        assert bp.bp_get_sparse_kernel(G.h)[0] == want
    G.reset()
    if planes0 is not None:
        G.set_messages(torch.from_numpy(planes0).cuda())
    G.iterate(iters, bp.BP_SUM if dtype == bp.BP_F32 else bp.BP_MAX, schedule)
    bel, mp = G.beliefs()
    pl = G.get_messages()
    G.sync()
    out = bel.cpu().numpy(), mp.cpu().numpy(), pl.cpu().numpy()
    G.close()
    return out


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("M,k", [(16, 5), (37, 9), (128, 9), (256, 4)])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
def test_sparse_sum_matches_oracle(M, k, schedule, kernel):
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(M + k)
    W, Hh = 11, 7
    g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
    pat = random_pattern(M, k, rng)
    fbar = 0.12
    p0 = H.random_planes_sum(W, Hh, M, rng)
    bel, mp, pl = _run(M, bp.BP_F32, p0, g, pat, fbar, 3, schedule, kernel)
    F = stereo.sparse_compatibility_matrix(*[x.astype(np.float64) if i == 2 else x for i, x in enumerate(pat)],
                                           fbar, M)
    p64, b64 = grid.grid_sum_product(g.astype(np.float64), F, 3, schedule, planes0=p0)
    assert H.node_rel_err(bel, b64) <= H.REL_TOL
    assert H.message_rel_err(pl, p64, W, Hh) <= H.REL_TOL


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("M,k", [(16, 5), (64, 7), (200, 6)])
@pytest.mark.parametrize("schedule", ["sync", "redblack"])
@pytest.mark.parametrize("ebar", [40, 16382, 16383])
def test_sparse_min_matches_oracle_bit_exact(M, k, schedule, kernel, ebar):
    """Ebar <= 16382 runs the register kernel's 16-bit form (h - min h clamped
    to Ebar + 1); 16382 with unaries up to 4 Ebar makes the clamp bite.
    16383 runs the 32-bit form."""
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(10 * M + k + ebar)
    W, Hh = 9, 8
    E = rng.integers(0, 30 if ebar == 40 else 4 * ebar, (Hh, W, M)).astype(np.int32)
    pat = random_pattern(M, k, rng, integer=True, ebar=ebar)
    p0 = H.random_planes_min(W, Hh, M, rng)
    if kernel == "registers":
        # the schedule that runs is the one of the form Ebar selects
        G = bp.BPGrid(W, Hh, M, bp.BP_I32)
        bp.bp_set_potential_sparse(G.h, *pat, ebar, bp.BP_I32)
        wf = bp.bp_get_sparse_kernel(G.h)[2]
        G.close()
        assert wf == bp.bp_sparse_schedule(M, pat[0], pat[1], 8 if ebar <= 16382 else 16)["wavefronts"]
    bel, mp, pl = _run(M, bp.BP_I32, p0, E, pat, ebar, 4, schedule, kernel)
    V = stereo.sparse_compatibility_matrix(pat[0], pat[1], pat[2].astype(np.int64), ebar, M, dtype=np.int64)
    p64, b64 = grid.grid_min_sum(E.astype(np.int64), V, 4, schedule, planes0=p0)
    src, dst, side, rr, cc = grid.grid_edges(W, Hh)
    np.testing.assert_array_equal(pl.astype(np.int64)[side, rr, cc], p64[side, rr, cc])
    np.testing.assert_array_equal(bel.astype(np.int64), b64)
    np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))


@pytest.mark.parametrize("kernel", KERNELS)
def test_band_written_as_lists_equals_the_band_kernel(kernel):
    """The truncated potential as a sparse pattern (|x_i - x_j| <= T) gives the
    band kernel's messages (integer: bit for bit)."""
    from paper_1010_0012_gb300 import bp
    cfg = wl.small_config("sb", 21, 13, 64, 3, alpha=0.7, structure="planar", seed=2)
    st, g, E = H.stereo_inputs(cfg)
    tabi, ebar = wl.pair_table_i32(cfg.alpha, cfg.T)
    rowptr, cols, vals = [0], [], []
    for xj in range(cfg.M):
        for d in range(-cfg.T, cfg.T + 1):
            if 0 <= xj + d < cfg.M:
                cols.append(xj + d)
                vals.append(int(tabi[d + cfg.T]))
        rowptr.append(len(cols))
    pat = (np.array(rowptr, np.int32), np.array(cols, np.int32), np.array(vals, np.int32))
    bel_s, _, pl_s = _run(cfg.M, bp.BP_I32, None, E, pat, ebar, 6, "sync", kernel)
    bel_b, _, pl_b = H.run_gpu_min(E, tabi, cfg.T, ebar, 6, "sync")
    np.testing.assert_array_equal(bel_s, bel_b)
    src, dst, side, rr, cc = grid.grid_edges(cfg.W, cfg.H)
    np.testing.assert_array_equal(pl_s[side, rr, cc], pl_b[side, rr, cc])


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("dtype_name", ["f32", "i32"])
def test_empty_pattern_leaves_only_the_constant_term(dtype_name, kernel):
    """No compatible pair at all: every pair has fbar (Ebar), so every
    message is uniform (1/M, or 0 for min-sum), whatever the inputs."""
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(5)
    M, W, Hh = 24, 6, 5
    rowptr = np.zeros(M + 1, np.int32)
    if dtype_name == "f32":
        g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
        bel, mp, pl = _run(M, bp.BP_F32, None, g, (rowptr, np.zeros(0, np.int32), np.zeros(0, np.float32)),
                           0.3, 2, "sync", kernel)
        src, dst, side, rr, cc = grid.grid_edges(W, Hh)
        np.testing.assert_allclose(pl[side, rr, cc][:, :M], 1.0 / M, rtol=1e-6)
        b64 = g.astype(np.float64) / g.astype(np.float64).sum(-1, keepdims=True)
        assert H.node_rel_err(bel, b64) <= H.REL_TOL
    else:
        E = rng.integers(0, 30, (Hh, W, M)).astype(np.int32)
        bel, mp, pl = _run(M, bp.BP_I32, None, E, (rowptr, np.zeros(0, np.int32), np.zeros(0, np.int32)),
                           7, 2, "sync", kernel)
        src, dst, side, rr, cc = grid.grid_edges(W, Hh)
        assert int(np.abs(pl[side, rr, cc][:, :M]).max()) == 0
        np.testing.assert_array_equal(bel.astype(np.int64), E.astype(np.int64))


def test_sparse_max_mode_rejects_energy_above_ebar():
    import torch
    from paper_1010_0012_gb300 import bp
    G = bp.BPGrid(4, 4, 8, bp.BP_I32)
    rowptr = np.array([0, 1, 1, 1, 1, 1, 1, 1, 1], np.int32)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_set_potential_sparse(G.h, rowptr, np.array([3], np.int32), np.array([9], np.int32), 5, bp.BP_I32)
    assert ei.value.status == bp.BP_ERR_POTENTIAL
    with pytest.raises(bp.BPError) as ei:
        bp.bp_set_potential_sparse(G.h, rowptr, np.array([8], np.int32), np.array([1], np.int32), 5, bp.BP_I32)
    assert ei.value.status == bp.BP_ERR_ARG
    G.close()


@pytest.mark.parametrize("dtype_name", ["f32", "i32"])
def test_sparse_long_rows_at_the_largest_label_count(dtype_name):
    """M = 300 (padded to 512 labels: 16 receiver labels per lane), rows from
    empty up to every label (the dense row), against the dense oracle."""
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(300)
    M, W, Hh = 300, 5, 4
    lens = rng.integers(0, 40, M)
    lens[[0, 7, M - 1]] = [M, 0, M]
    rowptr, cols = [0], []
    for xj in range(M):
        cols.extend(int(x) for x in rng.choice(M, size=int(lens[xj]), replace=False))
        rowptr.append(len(cols))
    rowptr, cols = np.array(rowptr, np.int32), np.array(cols, np.int32)
    if dtype_name == "f32":
        vals = rng.uniform(0.05, 2.0, len(cols)).astype(np.float32)
        g = rng.uniform(0.05, 1.0, (Hh, W, M)).astype(np.float32)
        bel, mp, pl = _run(M, bp.BP_F32, None, g, (rowptr, cols, vals), 0.1, 2, "sync")
        F = stereo.sparse_compatibility_matrix(rowptr, cols, vals.astype(np.float64), 0.1, M)
        p64, b64 = grid.grid_sum_product(g.astype(np.float64), F, 2, "sync")
        assert H.node_rel_err(bel, b64) <= H.REL_TOL
        assert H.message_rel_err(pl, p64, W, Hh) <= H.REL_TOL
    else:
        ebar = 25
        vals = rng.integers(0, ebar + 1, len(cols)).astype(np.int32)
        E = rng.integers(0, 30, (Hh, W, M)).astype(np.int32)
        bel, mp, pl = _run(M, bp.BP_I32, None, E, (rowptr, cols, vals), ebar, 2, "sync")
        V = stereo.sparse_compatibility_matrix(rowptr, cols, vals.astype(np.int64), ebar, M, dtype=np.int64)
        p64, b64 = grid.grid_min_sum(E.astype(np.int64), V, 2, "sync")
        np.testing.assert_array_equal(bel.astype(np.int64), b64)


def test_sparse_rejects_more_than_512_labels():
    from paper_1010_0012_gb300 import bp
    G = bp.BPGrid(3, 3, 600, bp.BP_F32)
    rowptr = np.zeros(601, np.int32)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_set_potential_sparse(G.h, rowptr, np.zeros(0, np.int32), np.zeros(0, np.float32), 0.5, bp.BP_F32)
    assert ei.value.status == bp.BP_ERR_UNSUPPORTED
    G.close()


def test_kernel_choice_follows_the_pattern():
    """The register kernel runs by default where the pattern has a schedule;
    a pattern without one (here M = 300: 512 padded labels) runs on the lists,
    and asking for registers there is refused."""
    import torch
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(4)
    G = bp.BPGrid(5, 4, 128, bp.BP_F32)
    G.set_unary(torch.ones((4, 5, 128), device="cuda"))
    with pytest.raises(bp.BPError) as ei:
        bp.bp_get_sparse_kernel(G.h)
    assert ei.value.status == bp.BP_ERR_STATE
    pat = random_pattern(128, 9, rng)
    bp.bp_set_potential_sparse(G.h, *pat, 0.1, bp.BP_F32)
    kind, steps, wf = bp.bp_get_sparse_kernel(G.h)
    assert kind == bp.BP_SPARSE_REGISTERS and 9 <= steps <= 12 and wf > 0
    bp.bp_set_sparse_kernel(G.h, bp.BP_SPARSE_LISTS)
    assert bp.bp_get_sparse_kernel(G.h) == (bp.BP_SPARSE_LISTS, 0, 0)
    G.close()
    G = bp.BPGrid(3, 3, 300, bp.BP_F32)
    pat = random_pattern(300, 3, rng)
    bp.bp_set_potential_sparse(G.h, *pat, 0.1, bp.BP_F32)
    assert bp.bp_get_sparse_kernel(G.h)[0] == bp.BP_SPARSE_LISTS
    with pytest.raises(bp.BPError) as ei:
        bp.bp_set_sparse_kernel(G.h, bp.BP_SPARSE_REGISTERS)
    assert ei.value.status == bp.BP_ERR_UNSUPPORTED
    G.close()

