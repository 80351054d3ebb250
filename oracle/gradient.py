"""FP64 reference gradient of unrolled sum-product BP -- TEST INFRASTRUCTURE.

The forward pass is plain dense sum-product BP (Eq. 2 with normalisation,
beliefs Eq. 3) on the 4-connected grid, written with float64 torch CPU ops so
that torch's autograd provides the exact reverse-mode derivative of the
unrolled iteration.  Central finite differences in float64 give a second,
independent derivative.

Parameters (the reading used throughout): the pairwise potential is
f(x_i, x_j) = exp(-alpha |x_i - x_j|) for |x_i - x_j| <= T and a free constant
fbar otherwise (its value exp(-alpha T) at the evaluation point); the unary is
g = exp(-beta * cost).  The loss is -sum_i log b_i(x_i*) at the ground-truth
label x_i*.
"""
from __future__ import annotations

import numpy as np
import torch

_DT = torch.float64


def _pair_matrix(alpha, fbar, T, M):
    xi = torch.arange(M, dtype=_DT)[:, None]
    xj = torch.arange(M, dtype=_DT)[None, :]
    d = (xi - xj).abs()
    return torch.where(d <= T, torch.exp(-alpha * d), fbar * torch.ones_like(d))


def _present(H, W):
    """Which message slots exist: planes into (r, c) from left/right/up/down."""
    rr = torch.arange(H)[:, None].expand(H, W)
    cc = torch.arange(W)[None, :].expand(H, W)
    return torch.stack([cc >= 1, cc <= W - 2, rr >= 1, rr <= H - 2])[..., None]


def _normalise(u):
    return u / u.sum(-1, keepdim=True)


def _as64(v):
    if isinstance(v, torch.Tensor):
        if v.dtype != _DT:
            raise TypeError("the FP64 oracle takes float64 tensors")
        return v
    return torch.tensor(float(v), dtype=_DT)


def sum_product_planes(logg, alpha, fbar, T, n_iters, schedule="sync"):
    """Dense sum-product on the grid; returns the [4][H][W][M] message planes
    (absent slots hold 1) and the normalised beliefs [H][W][M]."""
    logg, alpha, fbar = _as64(logg), _as64(alpha), _as64(fbar)
    H, W, M = logg.shape
    g = torch.exp(logg)
    F = _pair_matrix(alpha, fbar, T, M)
    present = _present(H, W)
    ones = torch.ones((H, W, M), dtype=_DT)
    planes = torch.where(present, torch.full((4, H, W, M), 1.0 / M, dtype=_DT), 1.0)
    parity = (torch.arange(H)[:, None] + torch.arange(W)[None, :]) % 2

    def all_new(P):
        P0, P1, P2, P3 = P[0], P[1], P[2], P[3]
        to_right = _normalise((g * P0 * P2 * P3) @ F)      # from (r,c) to (r,c+1): leaves out P1
        to_left = _normalise((g * P1 * P2 * P3) @ F)       # to (r,c-1): leaves out P0
        to_down = _normalise((g * P0 * P1 * P2) @ F)       # to (r+1,c): leaves out P3
        to_up = _normalise((g * P0 * P1 * P3) @ F)         # to (r-1,c): leaves out P2
        n0 = torch.cat([ones[:, :1], to_right[:, :-1]], dim=1)
        n1 = torch.cat([to_left[:, 1:], ones[:, -1:]], dim=1)
        n2 = torch.cat([ones[:1], to_down[:-1]], dim=0)
        n3 = torch.cat([to_up[1:], ones[-1:]], dim=0)
        return torch.stack([n0, n1, n2, n3])

    for _ in range(n_iters):
        if schedule == "sync":
            planes = all_new(planes)
        elif schedule == "redblack":
            for p in (0, 1):
                # half-step p: every message leaving a node of parity p, i.e.
                # every slot whose receiving node has parity 1 - p
                new = all_new(planes)
                planes = torch.where((parity == 1 - p)[None, ..., None], new, planes)
        else:
            raise ValueError(schedule)
    b = g * planes.prod(dim=0)
    return planes, b / b.sum(-1, keepdim=True)


def nll_loss(logg, alpha, fbar, T, n_iters, d_gt, schedule="sync"):
    """-sum_i log b_i(x_i*) after n_iters iterations."""
    _, bel = sum_product_planes(logg, alpha, fbar, T, n_iters, schedule)
    idx = torch.as_tensor(np.asarray(d_gt), dtype=torch.long)[..., None]
    return -torch.log(torch.gather(bel, -1, idx)).sum()


def reference_gradient(cost, d_gt, alpha, fbar, beta, T, n_iters, schedule="sync"):
    """Loss and its exact FP64 gradient: dict with loss, d_alpha, d_fbar, d_beta
    and d_logg ([H][W][M], the derivative with respect to log g)."""
    cost_t = torch.as_tensor(np.asarray(cost), dtype=_DT)
    a = torch.tensor(float(alpha), dtype=_DT, requires_grad=True)
    fb = torch.tensor(float(fbar), dtype=_DT, requires_grad=True)
    b = torch.tensor(float(beta), dtype=_DT, requires_grad=True)
    logg = (-b * cost_t).detach().requires_grad_(True)
    loss = nll_loss(logg, a, fb, T, n_iters, d_gt, schedule)
    d_logg, d_a, d_fb = torch.autograd.grad(loss, [logg, a, fb])
    d_b = float((d_logg * -cost_t).sum())
    return {"loss": float(loss.detach()), "d_alpha": float(d_a), "d_fbar": float(d_fb), "d_beta": d_b,
            "d_logg": d_logg.numpy()}


def loss_value(cost, d_gt, alpha, fbar, beta, T, n_iters, schedule="sync"):
    cost_t = torch.as_tensor(np.asarray(cost), dtype=_DT)
    with torch.no_grad():
        logg = -torch.tensor(float(beta), dtype=_DT) * cost_t
        return float(nll_loss(logg, torch.tensor(float(alpha), dtype=_DT),
                              torch.tensor(float(fbar), dtype=_DT), T, n_iters, d_gt, schedule))


def finite_difference(cost, d_gt, alpha, fbar, beta, T, n_iters, schedule="sync", rel_step=1e-6):
    """Central differences in FP64 for d/d alpha, d/d fbar, d/d beta."""
    theta = {"alpha": alpha, "fbar": fbar, "beta": beta}
    out = {}
    for k in theta:
        h = rel_step * max(1.0, abs(theta[k]))
        up = dict(theta)
        dn = dict(theta)
        up[k] += h
        dn[k] -= h
        lp = loss_value(cost, d_gt, up["alpha"], up["fbar"], up["beta"], T, n_iters, schedule)
        lm = loss_value(cost, d_gt, dn["alpha"], dn["fbar"], dn["beta"], T, n_iters, schedule)
        out["d_" + k] = (lp - lm) / (2 * h)
    return out


def _pair_matrix_from_table(table, fbar, T, M):
    """F[x_i, x_j] = table[x_i - x_j + T] for |x_i - x_j| <= T, fbar otherwise."""
    xi = torch.arange(M)[:, None]
    xj = torch.arange(M)[None, :]
    d = xi - xj
    inside = d.abs() <= T
    idx = (d + T).clamp(0, 2 * T)
    return torch.where(inside, table[idx], fbar * torch.ones((M, M), dtype=_DT))


def reference_gradient_table(cost, d_gt, table, fbar, beta, T, n_iters, schedule="sync"):
    """Exact FP64 gradient with the band values f(d) themselves as parameters:
    dict with loss, d_table [2T+1], d_fbar, d_logg."""
    cost_t = torch.as_tensor(np.asarray(cost), dtype=_DT)
    tab = torch.tensor(np.asarray(table, dtype=np.float64), requires_grad=True)
    fb = torch.tensor(float(fbar), dtype=_DT, requires_grad=True)
    logg = (-float(beta) * cost_t).detach().requires_grad_(True)
    H, W, M = logg.shape
    F = _pair_matrix_from_table(tab, fb, T, M)
    loss = _nll_with_matrix(logg, F, n_iters, d_gt, schedule)
    d_logg, d_tab, d_fb = torch.autograd.grad(loss, [logg, tab, fb])
    return {"loss": float(loss.detach()), "d_table": d_tab.numpy(), "d_fbar": float(d_fb),
            "d_logg": d_logg.numpy()}


def _nll_with_matrix(logg, F, n_iters, d_gt, schedule):
    """The same unrolled dense iteration as sum_product_planes, for a given F."""
    H, W, M = logg.shape
    g = torch.exp(logg)
    present = _present(H, W)
    ones = torch.ones((H, W, M), dtype=_DT)
    planes = torch.where(present, torch.full((4, H, W, M), 1.0 / M, dtype=_DT), 1.0)
    parity = (torch.arange(H)[:, None] + torch.arange(W)[None, :]) % 2

    def all_new(P):
        P0, P1, P2, P3 = P[0], P[1], P[2], P[3]
        to_right = _normalise((g * P0 * P2 * P3) @ F)
        to_left = _normalise((g * P1 * P2 * P3) @ F)
        to_down = _normalise((g * P0 * P1 * P2) @ F)
        to_up = _normalise((g * P0 * P1 * P3) @ F)
        return torch.stack([torch.cat([ones[:, :1], to_right[:, :-1]], dim=1),
                            torch.cat([to_left[:, 1:], ones[:, -1:]], dim=1),
                            torch.cat([ones[:1], to_down[:-1]], dim=0),
                            torch.cat([to_up[1:], ones[-1:]], dim=0)])

    for _ in range(n_iters):
        if schedule == "sync":
            planes = all_new(planes)
        else:
            for p in (0, 1):
                planes = torch.where((parity == 1 - p)[None, ..., None], all_new(planes), planes)
    b = g * planes.prod(dim=0)
    bel = b / b.sum(-1, keepdim=True)
    idx = torch.as_tensor(np.asarray(d_gt), dtype=torch.long)[..., None]
    return -torch.log(torch.gather(bel, -1, idx)).sum()
