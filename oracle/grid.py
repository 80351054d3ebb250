"""4-connected grid graphs for the oracle -- TEST INFRASTRUCTURE.

The stereo lattice of Sec. 6: node (r, c) of an H x W image is connected to
(r, c-1), (r, c+1), (r-1, c), (r+1, c) where those exist.  Nodes outside the
grid are absent (no message, i.e. a factor 1 in Eq. 2 / a term 0 in Eq. 9).

Message-plane layout used by the CUDA library (and mirrored here only to
compare results): planes[s][r][c][x] is the message INTO node (r, c) from its
neighbour on side s, s = 0 left (r, c-1), 1 right (r, c+1), 2 up (r-1, c),
3 down (r+1, c); label x innermost.
"""
from __future__ import annotations

import numpy as np

import oracle as _o

SIDE_OFFSETS = ((0, -1), (0, 1), (-1, 0), (1, 0))   # (dr, dc) of the sender, per side


def node_id(r, c, W):
    return r * W + c


def grid_edges(W: int, H: int):
    """Directed edges of the 4-connected grid as (src, dst, side, r, c).

    Edge e carries the message from src to dst = (r, c); `side` is the side of
    dst on which src sits, so the message lives in planes[side][r][c]."""
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    valid = np.zeros((H, W, 4), dtype=bool)
    for s, (dr, dc) in enumerate(SIDE_OFFSETS):
        valid[:, :, s] = (rr + dr >= 0) & (rr + dr < H) & (cc + dc >= 0) & (cc + dc < W)
    r, c, side = np.nonzero(valid)                     # ordered by (r, c, side)
    dr = np.asarray([o[0] for o in SIDE_OFFSETS])[side]
    dc = np.asarray([o[1] for o in SIDE_OFFSETS])[side]
    as32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    return (as32(node_id(r + dr, c + dc, W)), as32(node_id(r, c, W)), as32(side), as32(r),
            as32(c))


def redblack_colors(W: int, H: int):
    """Checkerboard colouring (r + c) mod 2 (the bipartite schedule of [2])."""
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return ((rr + cc) % 2).reshape(-1).astype(np.int32)


def edges_to_planes(msg, W, H, fill):
    """[n_edges][M] messages -> [4][H][W][M] planes (absent slots = fill)."""
    src, dst, side, rr, cc = grid_edges(W, H)
    M = msg.shape[1]
    planes = np.full((4, H, W, M), fill, dtype=msg.dtype)
    planes[side, rr, cc] = msg
    return planes


def planes_to_edges(planes, W, H):
    src, dst, side, rr, cc = grid_edges(W, H)
    return np.ascontiguousarray(planes[side, rr, cc])


def grid_sum_product(g, F, n_iters, schedule="sync", planes0=None):
    """Dense sum-product BP on the H x W grid.  g: [H][W][M].

    Returns (planes [4][H][W][M], beliefs [H][W][M]) in float64."""
    H, W, M = g.shape
    src, dst, side, rr, cc = grid_edges(W, H)
    msg0 = None if planes0 is None else planes_to_edges(np.asarray(planes0, dtype=np.float64), W, H)
    color = redblack_colors(W, H) if schedule == "redblack" else None
    msg = _o.sum_product(src, dst, g.reshape(H * W, M), F, n_iters, msg0=msg0, color=color,
                         schedule=schedule)
    bel = _o.sum_beliefs(dst, g.reshape(H * W, M), msg).reshape(H, W, M)
    return edges_to_planes(msg, W, H, 0.0), bel


def grid_min_sum(Eu, V, n_iters, schedule="sync", planes0=None):
    """Dense min-sum BP on the grid with int64 energies.  Eu: [H][W][M].

    Returns (planes [4][H][W][M], beliefs [H][W][M]) in int64."""
    H, W, M = Eu.shape
    src, dst, side, rr, cc = grid_edges(W, H)
    msg0 = None if planes0 is None else planes_to_edges(np.asarray(planes0, dtype=np.int64), W, H)
    color = redblack_colors(W, H) if schedule == "redblack" else None
    msg = _o.min_sum(src, dst, np.asarray(Eu).reshape(H * W, M), V, n_iters, msg0=msg0,
                     color=color, schedule=schedule)
    bel = _o.min_beliefs(dst, np.asarray(Eu).reshape(H * W, M), msg).reshape(H, W, M)
    return edges_to_planes(msg, W, H, 0), bel


def grid_incoming(planes, r, c, exclude_side=None):
    """The messages into (r, c), optionally without the one from `exclude_side`."""
    H, W = planes.shape[1], planes.shape[2]
    out = []
    for s, (dr, dc) in enumerate(SIDE_OFFSETS):
        if s == exclude_side:
            continue
        if 0 <= r + dr < H and 0 <= c + dc < W:
            out.append(planes[s, r, c])
    return out


# Outgoing message from (r, c) towards its neighbour on side t of (r, c): it is
# stored in the neighbour's plane on the opposite side, and Eq. 5 leaves out the
# message that came from that neighbour (plane t of (r, c)).
OPPOSITE = (1, 0, 3, 2)


def sampled_sum_updates(g, F, planes, samples):
    """One-by-one Eq. 2 updates for sampled outgoing messages.

    samples: iterable of (r, c, t): the message from (r, c) to its neighbour on
    side t.  Returns a list of [M] float64 results (same order)."""
    out = []
    for r, c, t in samples:
        inc = grid_incoming(planes, r, c, exclude_side=t)
        out.append(_o.sum_edge_update(g[r, c], inc, F))
    return out


def sampled_min_updates(Eu, V, planes, samples):
    out = []
    for r, c, t in samples:
        inc = grid_incoming(planes, r, c, exclude_side=t)
        out.append(_o.min_edge_update(Eu[r, c], inc, V))
    return out


__all__ = ["grid_edges", "redblack_colors", "edges_to_planes", "planes_to_edges",
           "grid_sum_product", "grid_min_sum", "sampled_sum_updates", "sampled_min_updates",
           "OPPOSITE", "SIDE_OFFSETS"]
