"""The CPU throughput baselines (FP32 O(mM) Eq. 7 and O(M^2) Eq. 2, OpenMP)
against the FP64 oracle: one synchronous iteration from random messages,
every message within FP32 rounding, on full grids and on a band of rows."""
import numpy as np
import pytest

import cpu_baselines as cb
import oracle
from oracle import grid, stereo


def _case(W, H, M, T, seed):
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.05, 1.0, (H, W, M)).astype(np.float32)
    planes = rng.uniform(0.1, 1.0, (4, H, W, M)).astype(np.float32)
    band = np.exp(-0.6 * np.abs(np.arange(-T, T + 1))).astype(np.float32)
    fbar = float(np.float32(np.exp(-0.6 * (T + 1))))
    return g, planes, band, fbar


def _oracle_step(g, planes, band, T, fbar):
    H, W, M = g.shape
    src, dst, side, rr, cc = grid.grid_edges(W, H)
    F = stereo.compatibility_matrix(band.astype(np.float64), T, fbar, M)
    msg0 = grid.planes_to_edges(planes.astype(np.float64), W, H)
    out = oracle.sum_product(src, dst, g.reshape(-1, M).astype(np.float64), F, 1, msg0=msg0)
    return grid.edges_to_planes(out, W, H, np.nan), F


def _check(got, ref, mask):
    assert np.all(np.isfinite(ref[mask].reshape(-1, ref.shape[-1])))
    rel = np.abs(got[mask] - ref[mask]).max(-1) / np.abs(ref[mask]).max(-1)
    assert float(rel.max()) <= 1e-5


@pytest.mark.parametrize("W,H,M,T", [(13, 9, 16, 2), (8, 11, 4, 0), (7, 5, 10, 9), (9, 6, 33, 4)])
@pytest.mark.parametrize("kind", ["band", "dense"])
def test_cpu_iteration_matches_oracle(W, H, M, T, kind):
    g, planes, band, fbar = _case(W, H, M, T, W * 100 + M)
    ref, F = _oracle_step(g, planes, band, T, fbar)
    out = np.full_like(planes, np.nan)
    if kind == "band":
        cb.band_iteration(g, planes, out, band, T, fbar)
    else:
        cb.dense_iteration(g, planes, out, F.astype(np.float32))
    present = np.isfinite(ref[..., 0])
    _check(out, ref, present)
    assert np.all(np.isnan(out[~present]))           # absent slots untouched


@pytest.mark.parametrize("kind", ["band", "dense"])
def test_cpu_iteration_on_a_band_of_rows(kind):
    W, H, M, T = 12, 10, 16, 3
    g, planes, band, fbar = _case(W, H, M, T, 7)
    ref, F = _oracle_step(g, planes, band, T, fbar)
    out = np.full_like(planes, np.nan)
    rows = (3, 6)
    if kind == "band":
        cb.band_iteration(g, planes, out, band, T, fbar, rows=rows, n_threads=2)
    else:
        cb.dense_iteration(g, planes, out, F.astype(np.float32), rows=rows, n_threads=2)
    # the nodes of rows 3..5 send into rows 2..6; a message is written iff its sender is in the band
    src, dst, side, rr, cc = grid.grid_edges(W, H)
    sent = np.zeros((4, H, W), bool)
    sent[side, rr, cc] = (src // W >= rows[0]) & (src // W < rows[1])
    _check(out, ref, sent)
    assert np.all(np.isnan(out[~sent]))
    assert int(sent.sum()) == cb.messages_sent(W, H, rows)


def test_cpu_band_equals_dense_when_the_band_covers_every_pair():
    W, H, M = 6, 5, 8
    T = M - 1
    g, planes, band, fbar = _case(W, H, M, T, 3)
    F = stereo.compatibility_matrix(band.astype(np.float64), T, fbar, M).astype(np.float32)
    a = np.zeros_like(planes)
    b = np.zeros_like(planes)
    cb.band_iteration(g, planes, a, band, T, fbar)
    cb.dense_iteration(g, planes, b, F)
    np.testing.assert_allclose(a, b, rtol=2e-6, atol=0)


def test_cpu_baselines_reject_bad_arguments():
    g = np.ones((4, 4, 8), np.float32)
    p = np.ones((4, 4, 4, 8), np.float32)
    with pytest.raises(ValueError):
        cb.band_iteration(g, p, p.copy(), np.ones(5, np.float32), 2, 0.1, rows=(3, 9))
    with pytest.raises(ValueError):
        cb.dense_iteration(g, p, p.astype(np.float64), np.ones((8, 8), np.float32))
    assert cb.threads() >= 1
