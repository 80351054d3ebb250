"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import grid, stereo
from paper_1010_0012_gb300 import workload as wl

REL_TOL = 1e-5   # per-node relative error of FP32 sum-product vs FP64


def bp():
    from paper_1010_0012_gb300 import bp as _bp
    return _bp


def torch():
    import torch as _t
    return _t


def oracle_F_from_table(table, T, fbar, M):
    """Dense M x M table of the sparse-compatibility potential, from the same
    float32 values the GPU receives."""
    return stereo.compatibility_matrix(np.asarray(table, dtype=np.float64), T, float(fbar), M)


def oracle_V_from_table(table, T, ebar, M):
    return stereo.compatibility_matrix(np.asarray(table, dtype=np.int64), T, int(ebar), M, dtype=np.int64)


def run_gpu_sum(g32, table, T, fbar, iters, schedule="sync", planes0=None, layout=None, dense=None,
                log=False, persistent=None):
    B = bp()
    t = torch()
    H, W, M = g32.shape
    G = B.BPGrid(W, H, M, B.BP_F32)
    if layout is not None:
        B.bp_set_layout(G.h, *layout)
    if persistent is not None:
        B.bp_set_persistent(G.h, persistent)
    G.set_unary(t.from_numpy(np.ascontiguousarray(g32)).cuda())
    G.set_potential(table, T, fbar)
    G.reset()
    if planes0 is not None:
        G.set_messages(t.from_numpy(np.ascontiguousarray(planes0, dtype=np.float32)).cuda())
    if dense is not None:
        G.iterate_dense(iters, dense)
    else:
        G.iterate(iters, B.BP_SUM | (B.BP_LOG if log else 0), schedule)
    bel, mp = G.beliefs()
    msgs = G.get_messages()
    G.sync()
    out = (bel.cpu().numpy(), mp.cpu().numpy(), msgs.cpu().numpy())
    G.close()
    return out


def run_gpu_min(E32, table, T, ebar, iters, schedule="sync", planes0=None, layout=None, dense=None,
                persistent=None):
    B = bp()
    t = torch()
    H, W, M = E32.shape
    G = B.BPGrid(W, H, M, B.BP_I32)
    if layout is not None:
        B.bp_set_layout(G.h, *layout)
    if persistent is not None:
        B.bp_set_persistent(G.h, persistent)
    G.set_unary(t.from_numpy(np.ascontiguousarray(E32, dtype=np.int32)).cuda())
    G.set_potential(table, T, ebar)
    G.reset()
    if planes0 is not None:
        G.set_messages(t.from_numpy(np.ascontiguousarray(planes0, dtype=np.int32)).cuda())
    if dense is not None:
        G.iterate_dense(iters, dense)
    else:
        G.iterate(iters, B.BP_MAX, schedule)
    bel, mp = G.beliefs()
    msgs = G.get_messages()
    G.sync()
    out = (bel.cpu().numpy(), mp.cpu().numpy(), msgs.cpu().numpy())
    G.close()
    return out


def node_rel_err(b32, b64):
    """max over nodes of max_x |b32 - b64| / max_x b64."""
    b32 = np.asarray(b32, dtype=np.float64)
    den = np.max(np.abs(b64), axis=-1)
    return float(np.max(np.max(np.abs(b32 - b64), axis=-1) / den))


def message_rel_err(p32, p64, W, H):
    src, dst, side, rr, cc = grid.grid_edges(W, H)
    if src.size == 0:
        return 0.0
    a = np.asarray(p32, dtype=np.float64)[side, rr, cc]
    b = np.asarray(p64)[side, rr, cc]
    return float(np.max(np.max(np.abs(a - b), axis=-1) / np.max(np.abs(b), axis=-1)))


def check_sum_map(map_gpu, bel_gpu, bel64, gap=1e-4):
    """MAP parity where floating point decides an argmax: the GPU label is the
    argmax of the GPU beliefs (lowest label on ties), and equals the oracle's
    wherever the oracle's top-two beliefs differ by more than `gap` (relative)."""
    np.testing.assert_array_equal(map_gpu, np.argmax(bel_gpu, axis=-1))
    top2 = np.sort(bel64, axis=-1)[..., -2:]
    clear = (top2[..., 1] - top2[..., 0]) > gap * top2[..., 1]
    ref = np.argmax(bel64, axis=-1)
    assert np.array_equal(map_gpu[clear], ref[clear])


def check_sum_case(g32, table, T, fbar, iters, schedule="sync", planes0=None, layout=None, dense=None,
                   log=False, tol=REL_TOL, persistent=None):
    H, W, M = g32.shape
    F = oracle_F_from_table(table, T, fbar, M)
    bel, mp, msgs = run_gpu_sum(g32, table, T, fbar, iters, schedule, planes0, layout, dense, log, persistent)
    p64, b64 = grid.grid_sum_product(g32.astype(np.float64), F, iters,
                                     "sync" if dense is not None else schedule, planes0=planes0)
    if log:
        bel = np.exp(bel.astype(np.float64))
    e_b = node_rel_err(bel, b64)
    e_m = message_rel_err(msgs, p64, W, H)
    assert e_b <= tol, f"belief rel err {e_b:.3e} > {tol}"
    assert e_m <= tol, f"message rel err {e_m:.3e} > {tol}"
    check_sum_map(mp, bel, b64)
    return e_b, e_m


def check_min_case(E, table, T, ebar, iters, schedule="sync", planes0=None, layout=None, dense=None,
                   persistent=None):
    H, W, M = E.shape
    V = oracle_V_from_table(table, T, ebar, M)
    bel, mp, msgs = run_gpu_min(E, table, T, ebar, iters, schedule, planes0, layout, dense, persistent)
    p64, b64 = grid.grid_min_sum(E.astype(np.int64), V, iters, "sync" if dense is not None else schedule,
                                 planes0=planes0)
    src, dst, side, rr, cc = grid.grid_edges(W, H)
    np.testing.assert_array_equal(msgs.astype(np.int64)[side, rr, cc], p64[side, rr, cc])
    np.testing.assert_array_equal(bel.astype(np.int64), b64)
    np.testing.assert_array_equal(mp, oracle.map_labels(b64, maximise=False))


def stereo_inputs(cfg):
    st = wl.make_stereo(cfg)
    return st, wl.unary_f32(st), wl.unary_i32(st)


def random_planes_sum(W, H, M, rng):
    p = rng.uniform(0.05, 1.0, (4, H, W, M))
    return (p / p.sum(-1, keepdims=True)).astype(np.float32)


def random_planes_min(W, H, M, rng, hi=30):
    p = rng.integers(0, hi, (4, H, W, M))
    return (p - p.min(-1, keepdims=True)).astype(np.int32)
