"""Coarse-to-fine (multi-scale) BP on the grid -- TEST INFRASTRUCTURE.

The multi-scale message passing of [2], which Sec. 2 and Sec. 6 name as
combinable with the O(mM) update.  Reading used here (the paper gives no
details): level l+1 has one node per 2 x 2 block of level l (ceil(W/2) x
ceil(H/2)); its unary is the product of the block's unaries (the sum of their
energies for min-sum); the pairwise potential is the same at every level.  BP
runs first on the coarsest level from uniform messages; the messages of each
finer level start as the final messages of the coarser one, copied by
direction: the message into (r, c) from side s starts as the message into
(r // 2, c // 2) from side s, or uniform where the coarse node has no
neighbour on that side.  Then BP runs on that level, down to the given grid.
Coarse unaries are kept scaled to maximum 1 per node (formed in logs); a
per-node scale of g changes no message and no belief.
"""
from __future__ import annotations

import numpy as np

from . import grid


def coarse_shape(H, W):
    return (H + 1) // 2, (W + 1) // 2


def coarsen(u, combine):
    """Block 2 x 2 combination of a [H][W][M] unary: `combine` is np.prod
    (potentials) or np.sum (energies) over the block's existing nodes."""
    H, W, M = u.shape
    Hc, Wc = coarse_shape(H, W)
    out = np.empty((Hc, Wc, M), dtype=u.dtype)
    for r in range(Hc):
        for c in range(Wc):
            block = u[2 * r:2 * r + 2, 2 * c:2 * c + 2].reshape(-1, M)
            out[r, c] = combine(block, axis=0)
    return out


def upsample_messages(planes_c, H, W, fill):
    """Initial fine planes [4][H][W][M] from the coarse ones, by direction."""
    _, Hc, Wc, M = planes_c.shape
    out = np.full((4, H, W, M), fill, dtype=planes_c.dtype)
    for s, (dr, dc) in enumerate(grid.SIDE_OFFSETS):
        for r in range(H):
            for c in range(W):
                pr, pc = r // 2, c // 2
                if 0 <= pr + dr < Hc and 0 <= pc + dc < Wc:
                    out[s, r, c] = planes_c[s, pr, pc]
    return out


def coarsen_log(lu):
    """Coarse log-unary: the block sum of log g (the log of the block product),
    minus its maximum over labels -- the product scaled to maximum 1 per node,
    which BP does not see and which keeps products of thousands of unaries
    representable."""
    s = coarsen(lu, np.sum)
    return s - s.max(axis=-1, keepdims=True)


def multiscale_sum_product(g, F, iters, schedule="sync"):
    """iters[k] iterations at level len(iters)-1-k (coarsest first).  Returns
    the finest planes and beliefs (float64)."""
    levels = len(iters)
    pyr = [np.asarray(g, dtype=np.float64)]
    lu = np.log(pyr[0])
    for _ in range(levels - 1):
        lu = coarsen_log(lu)
        pyr.append(np.exp(lu))
    planes = None
    for k, lvl in enumerate(range(levels - 1, -1, -1)):
        u = pyr[lvl]
        H, W, M = u.shape
        p0 = None if planes is None else upsample_messages(planes, H, W, 1.0 / M)
        planes, bel = grid.grid_sum_product(u, F, iters[k], schedule, planes0=p0)
    return planes, bel


def multiscale_min_sum(Eu, V, iters, schedule="sync"):
    levels = len(iters)
    pyr = [np.asarray(Eu, dtype=np.int64)]
    for _ in range(levels - 1):
        pyr.append(coarsen(pyr[-1], np.sum))
    planes = None
    for k, lvl in enumerate(range(levels - 1, -1, -1)):
        u = pyr[lvl]
        H, W, M = u.shape
        p0 = None if planes is None else upsample_messages(planes, H, W, 0)
        planes, bel = grid.grid_min_sum(u, V, iters[k], schedule, planes0=p0)
    return planes, bel
