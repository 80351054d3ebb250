"""torch.autograd.Function around the recorded log-domain forward and the
hand-written adjoint of the library (bp_iterate with BP_SUM|BP_LOG|BP_RECORD,
bp_beliefs, bp_backward).

BPFunction maps (log g, band table f(d), fbar) to the normalised log-beliefs
after K unrolled synchronous sum-product iterations.  Its backward calls
bp_backward, which recomputes each checkpoint segment and runs the adjoint
kernel; the parameter gradients (dL/df(d), dL/dfbar) come back in FP64.
With the table (and fbar) on the GPU the backward calls bp_backward_device:
the gradients stay on the device and no host wait interrupts autograd, so
the rest of the backward graph is queued while the reverse pass runs.
The library does all of the BP arithmetic; this module only moves tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bp


class BPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, logg, table, fbar, grid, T, n_iters, every):
        if logg.dtype != torch.float32 or not logg.is_cuda:
            raise TypeError("logg must be a float32 CUDA tensor [H][W][M]")
        h = grid.h
        bp.bp_set_unary_log(h, logg.detach().contiguous())
        if table.is_cuda:
            # the library takes the table on the host: one copy for the table
            # and fbar, in float64 so that both values arrive unchanged
            fb = fbar.detach().reshape(1).to(device=table.device, dtype=torch.float64) \
                if isinstance(fbar, torch.Tensor) else torch.tensor([float(fbar)], dtype=torch.float64, device=table.device)
            vals = torch.cat([table.detach().reshape(-1).double(), fb]).cpu().numpy()
            tab_h, fbar_h = vals[:-1].astype(np.float32), float(vals[-1])
        else:
            tab_h, fbar_h = table.detach().cpu().numpy().astype(np.float32), float(fbar)
        bp.bp_set_potential(h, tab_h, T, fbar_h, bp.BP_F32)
        bp.bp_set_checkpoint_interval(h, every)
        bp.bp_reset_messages(h)
        bp.bp_iterate(h, n_iters, bp.BP_SUM | bp.BP_LOG | bp.BP_RECORD, bp.BP_SYNC)
        logb = torch.empty_like(logg)
        bp.bp_beliefs(h, logb)
        if not grid.on_current_stream():
            bp.bp_sync(h)          # the handle's own stream: order it before torch's next work
        ctx.grid = grid
        ctx.T = T
        ctx.table_meta = (table.dtype, table.device)
        ctx.fbar_meta = (fbar.dtype, fbar.device, fbar.shape) if isinstance(fbar, torch.Tensor) else None
        return logb

    @staticmethod
    def backward(ctx, dlogb):
        dlogg = torch.empty_like(dlogb)
        tdt, tdev = ctx.table_meta
        n = 2 * ctx.T + 1
        h = ctx.grid.h
        if tdev.type == "cuda" and (ctx.fbar_meta is None or ctx.fbar_meta[1].type == "cuda"):
            # parameters on the GPU: the float64 gradients stay there and
            # nothing waits for the reverse pass
            dt = torch.empty(n, dtype=torch.float64, device=dlogb.device)
            df = torch.empty(1, dtype=torch.float64, device=dlogb.device)
            bp.bp_backward_device(h, dlogb.detach().float().contiguous(), dlogg, dt, df)
            if not ctx.grid.on_current_stream():
                bp.bp_sync(h)
            g_tab = dt.to(device=tdev, dtype=tdt)
            g_fbar = None
            if ctx.fbar_meta is not None:
                g_fbar = df.reshape(ctx.fbar_meta[2]).to(device=ctx.fbar_meta[1], dtype=ctx.fbar_meta[0])
            return dlogg, g_tab, g_fbar, None, None, None, None
        dtab, dfbar = bp.bp_backward(h, dlogb.detach().float().contiguous(), dlogg, n)
        g_tab = torch.as_tensor(dtab, dtype=torch.float64).to(device=tdev, dtype=tdt)
        g_fbar = None
        if ctx.fbar_meta is not None:
            g_fbar = torch.tensor(dfbar, dtype=torch.float64).reshape(ctx.fbar_meta[2]).to(
                device=ctx.fbar_meta[1], dtype=ctx.fbar_meta[0])
        return dlogg, g_tab, g_fbar, None, None, None, None


def log_beliefs(logg, table, fbar, grid, T, n_iters, every=5):
    """Normalised log-beliefs after n_iters log-domain iterations (differentiable
    in logg, table and fbar)."""
    return BPFunction.apply(logg, table, fbar, grid, T, n_iters, every)


class _NegScaledCost(torch.autograd.Function):
    """log g = -beta * cost.  The forward multiplies in FP32: the product of
    two FP32 numbers is exact in FP64, so rounding it once to FP32 gives what
    an FP64 product rounded to FP32 gives.  The backward keeps the chain rule
    to beta, a sum over every node and label, in FP64 (products and sum)."""

    @staticmethod
    def forward(ctx, cost, beta):
        ctx.save_for_backward(cost, beta)
        return torch.mul(cost, beta.to(device=cost.device, dtype=cost.dtype)).neg_()

    @staticmethod
    def backward(ctx, dlogg):
        cost, beta = ctx.saved_tensors
        g = -torch.dot(dlogg.reshape(-1).double(), cost.reshape(-1).double())
        return None, g.to(device=beta.device, dtype=beta.dtype)


_OFFSETS = {}


def _neg_abs_offsets(T, device):
    """-|d| for d = -T..T as float32 on `device`, made once per (T, device)."""
    key = (int(T), str(device))
    t = _OFFSETS.get(key)
    if t is None:
        t = -torch.arange(-T, T + 1, dtype=torch.float32, device=device).abs()
        _OFFSETS[key] = t
    return t


def stereo_nll(cost, d_gt, alpha, fbar, beta, T, n_iters, grid, every=5):
    """-sum_i log b_i(x_i*) of the stereo model (Sec. 6) with parameters
    alpha, fbar, beta as tensors: log g = -beta cost, f(d) = exp(-alpha |d|)
    for |d| <= T and fbar outside.  Autograd's chain rule maps the library's
    dL/d log g, dL/df(d), dL/dfbar to dL/d beta, d alpha, d fbar."""
    dev = cost.device
    # the chain rule to beta sums dL/d log g * cost over every node: that
    # reduction stays in FP64 (the library's log g is FP32)
    logg = _NegScaledCost.apply(cost.float().contiguous(), beta)
    # alpha * (-|d|) is -alpha * |d| exactly (IEEE products are sign-symmetric)
    table = torch.exp(alpha * _neg_abs_offsets(T, alpha.device))
    logb = log_beliefs(logg, table, fbar, grid, T, n_iters, every)
    idx = torch.as_tensor(d_gt, dtype=torch.long, device=dev)[..., None]
    return -torch.gather(logb, -1, idx).sum()
