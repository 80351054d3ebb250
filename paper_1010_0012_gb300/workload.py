"""Seeded synthetic stereo workloads (random-dot stereograms).

This module only builds inputs: image pairs, ground-truth disparities and
the per-pixel matching-cost volume of the stereo model of Sec. 6.  It holds
none of the belief-propagation arithmetic, and both the CUDA path and the
CPU oracle take their inputs from here.

Stereo model (Sec. 6): pixel i at (r, c) with disparity x_i expects
R(r, c) ~ L(r, c + x_i).  The unary potential is
g(x_i) = exp(-beta * min(|R(r,c) - L(r,c+x_i)|, T_u)); the pairwise
potential is f(x_i, x_j) = exp(-alpha * min(|x_i - x_j|, T)) (Sec. 1 and 6).
Where c + x_i falls outside the image the matching cost is the maximum
penalty T_u.

Integer (min-sum) energies use a positive scaling Q = 10 of -log P:
E_u = round(Q*beta) * cost and V(d) = round(Q*alpha) * min(|d|, T), so the
MAP labelling is that of the real-valued model at these alpha and beta.

The Tsukuba pair used in Sec. 6 is not available; these random-dot pairs
with the shapes of the five benchmark workloads stand in for it.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

Q_ENERGY = 10          # integer energy scale for min-sum
T_U = 20               # unary truncation (maximum matching penalty)
BETA = 0.1             # unary sharpness


@dataclass(frozen=True)
class GridConfig:
    """One single-grid workload."""
    name: str
    W: int
    H: int
    M: int
    T: int
    alpha: float
    iters: int
    schedule: str                  # "sync" | "redblack"
    structure: str                 # disparity structure, see _disparity()
    seed: int
    beta: float = BETA
    Tu: int = T_U
    noise_sigma: float = 0.0
    modes: tuple = ("sum", "min")


# The five benchmark workloads.  Seeds are 1000 + workload index.
CONFIGS = {
    "grid32_m16": GridConfig("grid32_m16", 32, 32, 16, 2, 1.0, 10, "sync",
                             "rectangles", 1001),
    "grid384x288_m16": GridConfig("grid384x288_m16", 384, 288, 16, 2, 1.0, 50,
                                  "redblack", "voronoi", 1002, noise_sigma=3.0),
    "grid1280x720_m128": GridConfig("grid1280x720_m128", 1280, 720, 128, 4, 0.5,
                                    100, "sync", "slanted", 1003, modes=("sum",)),
    "grid256_m64_grad": GridConfig("grid256_m64_grad", 256, 256, 64, 3, 1.0, 30,
                                   "sync", "planar", 1005, modes=("sum",)),
}
BATCH_SEED = 1004


@dataclass
class Stereo:
    """A stereo problem: images, ground truth and the matching-cost volume."""
    cfg: GridConfig
    left: np.ndarray        # uint8 [H][W]
    right: np.ndarray       # uint8 [H][W]
    d_gt: np.ndarray        # int32 [H][W]
    cost: np.ndarray        # uint8 [H][W][M], min(|R - L(shifted)|, Tu), Tu off-image

    @property
    def shape(self):
        return self.cfg.H, self.cfg.W, self.cfg.M


def _disparity(structure: str, H: int, W: int, M: int, rng: np.random.Generator) -> np.ndarray:
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    if structure == "rectangles":
        d = np.full((H, W), int(rng.integers(0, M)), dtype=np.int64)
        for _ in range(3):
            h = int(rng.integers(max(1, H // 6), max(2, H // 2)))
            w = int(rng.integers(max(1, W // 6), max(2, W // 2)))
            r0 = int(rng.integers(0, H - h + 1))
            c0 = int(rng.integers(0, W - w + 1))
            d[r0:r0 + h, c0:c0 + w] = int(rng.integers(0, M))
        return d.astype(np.int32)
    if structure in ("voronoi", "planar"):
        n = 8
        pr = rng.uniform(0, H, n)
        pc = rng.uniform(0, W, n)
        dist = (rr[None] - pr[:, None, None]) ** 2 + (cc[None] - pc[:, None, None]) ** 2
        region = np.argmin(dist, axis=0)
        if structure == "voronoi":
            vals = rng.integers(0, M, n)
            return vals[region].astype(np.int32)
        # piecewise planar: each region a plane with a gentle slant
        d0 = rng.uniform(0, M - 1, n)
        a = rng.uniform(-0.5, 0.5, n) * (M - 1) / max(W - 1, 1)
        b = rng.uniform(-0.5, 0.5, n) * (M - 1) / max(H - 1, 1)
        d = d0[region] + a[region] * (cc - pc[region]) + b[region] * (rr - pr[region])
        return np.clip(np.rint(d), 0, M - 1).astype(np.int32)
    if structure == "slanted":
        frac = rng.uniform(0.3, 0.7)
        a = frac * (M - 1) / max(W - 1, 1)
        b = (1.0 - frac) * (M - 1) / max(H - 1, 1)
        d = a * cc + b * rr
        return np.clip(np.rint(d), 0, M - 1).astype(np.int32)
    raise ValueError(f"unknown disparity structure {structure!r}")


def _images(d_gt: np.ndarray, noise_sigma: float, rng: np.random.Generator):
    H, W = d_gt.shape
    left = rng.integers(0, 256, (H, W), dtype=np.int64)
    cc = np.arange(W)[None, :] + d_gt
    inside = cc < W
    fresh = rng.integers(0, 256, (H, W), dtype=np.int64)
    rows = np.broadcast_to(np.arange(H)[:, None], (H, W))
    right = np.where(inside, left[rows, np.minimum(cc, W - 1)], fresh)
    if noise_sigma > 0:
        left = left + rng.normal(0.0, noise_sigma, (H, W))
        right = right + rng.normal(0.0, noise_sigma, (H, W))
    left = np.clip(np.rint(left), 0, 255).astype(np.uint8)
    right = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return left, right


def cost_volume(left: np.ndarray, right: np.ndarray, M: int, Tu: int = T_U) -> np.ndarray:
    """Truncated absolute matching cost min(|R(r,c) - L(r,c+x)|, Tu), Tu off-image.

    Returns uint8 [H][W][M] (costs never exceed Tu <= 255)."""
    H, W = left.shape
    L = left.astype(np.int16)
    R = right.astype(np.int16)
    cost = np.full((H, W, M), Tu, dtype=np.uint8)
    for x in range(min(M, W)):
        diff = np.abs(R[:, :W - x] - L[:, x:])
        cost[:, :W - x, x] = np.minimum(diff, Tu).astype(np.uint8)
    return cost


def make_stereo(cfg: GridConfig, seed: Optional[int] = None) -> Stereo:
    rng = np.random.Generator(np.random.PCG64(cfg.seed if seed is None else seed))
    d_gt = _disparity(cfg.structure, cfg.H, cfg.W, cfg.M, rng)
    left, right = _images(d_gt, cfg.noise_sigma, rng)
    return Stereo(cfg, left, right, d_gt, cost_volume(left, right, cfg.M, cfg.Tu))


def small_config(name: str, W: int, H: int, M: int, T: int, alpha: float = 1.0,
                 iters: int = 10, schedule: str = "sync", structure: str = "rectangles",
                 seed: int = 7, noise_sigma: float = 0.0) -> GridConfig:
    """A test-sized workload with the same recipe."""
    return GridConfig(name, W, H, M, T, alpha, iters, schedule, structure, seed,
                      noise_sigma=noise_sigma)


# ---------------------------------------------------------------------------
# Unary and pairwise tables handed to both sides.  Each is the potential of the
# stereo model evaluated once in float64 and rounded once to the type the GPU
# path stores (float32 or int32), so both sides see identical inputs.

def unary_table_f32(cfg: GridConfig) -> np.ndarray:
    """g as a function of the matching cost k = 0..Tu: exp(-beta * k) in
    float64, rounded once to float32."""
    return np.exp(-cfg.beta * np.arange(cfg.Tu + 1, dtype=np.float64)).astype(np.float32)


def unary_table_i32(cfg: GridConfig) -> np.ndarray:
    """E_u as a function of the matching cost k = 0..Tu: round(Q*beta) * k."""
    return int(round(Q_ENERGY * cfg.beta)) * np.arange(cfg.Tu + 1, dtype=np.int32)


def unary_f32(stereo: Stereo) -> np.ndarray:
    """g = exp(-beta * cost) as float32 [H][W][M] (FP64 exp, one rounding)."""
    return unary_table_f32(stereo.cfg)[stereo.cost]


def unary_i32(stereo: Stereo) -> np.ndarray:
    """E_u = round(Q*beta) * cost as int32 [H][W][M]."""
    return unary_table_i32(stereo.cfg)[stereo.cost]


def pair_table_f32(alpha: float, T: int):
    """Band table f(d) = exp(-alpha*min(|d|,T)), d = -T..T, and fbar = exp(-alpha*T)."""
    d = np.arange(-T, T + 1)
    table = np.exp(-alpha * np.minimum(np.abs(d), T).astype(np.float64)).astype(np.float32)
    fbar = float(np.float32(np.exp(-alpha * float(T))))
    return table, fbar


def pair_table_i32(alpha: float, T: int):
    """Band energies V(d) = round(Q*alpha)*min(|d|,T), d = -T..T, and Vbar = round(Q*alpha)*T."""
    q = int(round(Q_ENERGY * alpha))
    d = np.arange(-T, T + 1)
    return (q * np.minimum(np.abs(d), T)).astype(np.int32), q * T


# ---------------------------------------------------------------------------
# Batch of uneven MRFs (64 problems of different size, label count and band).

@dataclass
class BatchItem:
    cfg: GridConfig
    stereo: Stereo


def make_batch(n: int = 64, seed: int = BATCH_SEED, w_range=(128, 640), h_range=(128, 480),
               m_choices=(32, 64, 128, 256), t_range=(2, 8), alpha_range=(0.25, 1.0),
               iters: int = 30) -> List[BatchItem]:
    rng = np.random.Generator(np.random.PCG64(seed))
    items = []
    for k in range(n):
        W = int(rng.integers(w_range[0], w_range[1] + 1))
        H = int(rng.integers(h_range[0], h_range[1] + 1))
        M = int(rng.choice(np.asarray(m_choices)))
        T = int(rng.integers(t_range[0], t_range[1] + 1))
        alpha = float(rng.uniform(*alpha_range))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        cfg = GridConfig(f"batch{k}", W, H, M, T, alpha, iters, "sync", "planar", sub_seed)
        items.append(BatchItem(cfg, make_stereo(cfg)))
    return items


def directed_edges(W: int, H: int) -> int:
    """Number of directed messages on a 4-connected W x H grid."""
    return 2 * (H * (W - 1) + W * (H - 1))
