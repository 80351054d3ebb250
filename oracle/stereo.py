"""The stereo MRF's potentials, written from their definitions -- TEST INFRASTRUCTURE.

Every table here is the full M x M (or per-pixel M-vector) object the paper
defines; nothing is split into a constant and a band.

  f(x_i, x_j) = exp(-alpha * min(|x_i - x_j|, T))              (Sec. 1, Sec. 6)
  g_i(x)      = exp(-beta * min(|R(r,c) - L(r,c+x)|, T_u))      (Sec. 6)

with the integer (min-sum) energies V = q_a * min(|d|, T), E_u = q_b * cost,
a positive scaling of -log f and -log g.
"""
from __future__ import annotations

import numpy as np


def pairwise_matrix(alpha: float, T: int, M: int) -> np.ndarray:
    """F[x_i, x_j] = exp(-alpha * min(|x_i - x_j|, T)), float64."""
    xi = np.arange(M)[:, None]
    xj = np.arange(M)[None, :]
    return np.exp(-alpha * np.minimum(np.abs(xi - xj), T).astype(np.float64))


def pairwise_energy_matrix(q: int, T: int, M: int) -> np.ndarray:
    """V[x_i, x_j] = q * min(|x_i - x_j|, T), int64."""
    xi = np.arange(M)[:, None]
    xj = np.arange(M)[None, :]
    return (q * np.minimum(np.abs(xi - xj), T)).astype(np.int64)


def compatibility_matrix(band, T: int, fbar, M: int, dtype=np.float64) -> np.ndarray:
    """A general sparse-compatibility potential (Sec. 4): f(x_i, x_j) is
    band[x_i - x_j + T] when |x_i - x_j| <= T and the constant fbar otherwise."""
    band = np.asarray(band)
    F = np.full((M, M), fbar, dtype=dtype)
    for xi in range(M):
        for xj in range(M):
            d = xi - xj
            if -T <= d <= T:
                F[xi, xj] = band[d + T]
    return F


def matching_cost(left: np.ndarray, right: np.ndarray, M: int, Tu: int) -> np.ndarray:
    """cost[r, c, x] = min(|R(r,c) - L(r,c+x)|, Tu), and Tu where c + x >= W (Sec. 6)."""
    H, W = left.shape
    Lp = np.concatenate([left.astype(np.int64), np.full((H, M), -1, dtype=np.int64)], axis=1)
    cols = np.arange(W)[:, None] + np.arange(M)[None, :]          # [W][M]
    shifted = Lp[:, cols]                                          # [H][W][M] = L(r, c+x)
    d = np.abs(right.astype(np.int64)[:, :, None] - shifted)
    cost = np.minimum(d, Tu)
    cost[shifted < 0] = Tu
    return cost


def unary_potential(left, right, M, beta, Tu) -> np.ndarray:
    """g[r, c, x] = exp(-beta * cost[r, c, x]), float64."""
    return np.exp(-beta * matching_cost(left, right, M, Tu).astype(np.float64))


def sparse_compatibility_matrix(rowptr, cols, vals, fbar, M, dtype=np.float64) -> np.ndarray:
    """A sparse-compatibility potential given per receiver label x_j by the
    list of compatible sender labels x_i and their values (Sec. 4): F[x_i, x_j]
    is that value when x_i is listed for x_j, fbar otherwise."""
    F = np.full((M, M), fbar, dtype=dtype)
    for xj in range(M):
        for p in range(rowptr[xj], rowptr[xj + 1]):
            F[cols[p], xj] = vals[p]
    return F
