"""FP32 calibration of the fit constants: the linear fit without its integer
shift and clamp, behind torch.autograd.Functions whose forward and backward
run in libsvt.so's kernels (include/svt.h, "FP32 calibration relaxation").

    data = CalibData(x, sector, theta, n_sectors, w)   # sorts the tracks by sector on the GPU
    loss = calib_loss(F, q, data)                      # L, differentiable in F and q
    y = fit_fp32(F, q, data)                           # y = F[s] x + q[s], tracks in sector order

The integer path is untouched by all of this.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .api import _p, _stream


def _f32(t):
    return t.detach().to(torch.float32).contiguous()


class CalibData:
    """Tracks in sector order with the device-side sector index."""

    def __init__(self, x, sector, theta, n_sectors: int, w=None, device="cuda"):
        L = N.load()
        x = torch.as_tensor(x, dtype=torch.float32, device=device).contiguous()
        sector = torch.as_tensor(sector, dtype=torch.int32, device=device).contiguous()
        theta = torch.as_tensor(theta, dtype=torch.float32, device=device).contiguous()
        n = int(sector.numel())
        self.n, self.n_sectors = n, int(n_sectors)
        self.index = torch.empty(L.svt_calib_index_size(n, self.n_sectors), dtype=torch.uint8,
                                 device=device)
        self.perm = torch.empty(max(n, 1), dtype=torch.int32, device=device)
        status = torch.empty(1, dtype=torch.int64, device=device)
        st = _stream(None)
        N.check(L.svt_calib_index(_p(sector), n, self.n_sectors, _p(self.index),
                                  self.index.numel(), _p(self.perm), _p(status), st),
                "svt_calib_index")
        key = int(status.cpu().numpy().view(np.uint64)[0])
        if key != N.STATUS_OK:
            raise N.SvtError(f"bad sector at track {key >> 8}")
        self.x = torch.empty((max(n, 1), 6), dtype=torch.float32, device=device)
        self.theta = torch.empty((max(n, 1), 3), dtype=torch.float32, device=device)
        N.check(L.svt_calib_gather(_p(x), 6, _p(self.perm), n, _p(self.x), st), "svt_calib_gather")
        N.check(L.svt_calib_gather(_p(theta), 3, _p(self.perm), n, _p(self.theta), st),
                "svt_calib_gather")
        self.w = (torch.ones(3) if w is None else torch.as_tensor(w)).to(device, torch.float32).contiguous()
        # zero-filled once: the fused pass keeps its tickets here
        self.workspace = torch.zeros(L.svt_calib_workspace_size(n, self.n_sectors), dtype=torch.uint8,
                                     device=device)


class FitFP32(torch.autograd.Function):
    """y = F[s] x + q[s] for the tracks of a CalibData (sector order)."""

    @staticmethod
    def forward(ctx, F, q, data: CalibData):
        L = N.load()
        F32, q32 = _f32(F), _f32(q)
        y = torch.empty((max(data.n, 1), 6), dtype=torch.float32, device=F.device)
        N.check(L.svt_calib_forward(_p(data.x), data.n, data.n_sectors, _p(data.index), _p(F32),
                                    _p(q32), _p(y), _stream(None)), "svt_calib_forward")
        ctx.data = data
        ctx.save_for_backward(F32)
        return y[: data.n]

    @staticmethod
    def backward(ctx, gy):
        L = N.load()
        data = ctx.data
        (F32,) = ctx.saved_tensors
        gy = gy.to(torch.float32).contiguous()
        dF = torch.empty_like(F32)
        dq = torch.empty((data.n_sectors, 6), dtype=torch.float32, device=F32.device)
        N.check(L.svt_calib_backward(_p(data.x), _p(gy), data.n, data.n_sectors, _p(data.index),
                                     _p(F32), _p(dF), _p(dq), None, _p(data.workspace),
                                     data.workspace.numel(), _stream(None)), "svt_calib_backward")
        return dF, dq, None


class CalibLoss(torch.autograd.Function):
    """L(F, q) of a CalibData (mean squared parameter error weighted by w,
    plus the mean chi-square of the three chi rows).  When F or q needs a
    gradient, the forward makes one fused pass (svt_calib_loss_grad) that
    reads the tracks once and yields L together with dL/dF and dL/dq; the
    backward then only scales them by the upstream gradient
    (svt_calib_grad_scale)."""

    @staticmethod
    def forward(ctx, F, q, data: CalibData):
        L = N.load()
        F32, q32 = _f32(F), _f32(q)
        loss = torch.empty(1, dtype=torch.float32, device=F.device)
        ctx.data = data
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            dF = torch.empty_like(F32)
            dq = torch.empty_like(q32)
            N.check(L.svt_calib_loss_grad(_p(data.x), _p(data.theta), _p(data.w), data.n,
                                          data.n_sectors, _p(data.index), _p(F32), _p(q32),
                                          _p(loss), _p(dF), _p(dq), None, _p(data.workspace),
                                          data.workspace.numel(), _stream(None)),
                    "svt_calib_loss_grad")
            ctx.save_for_backward(dF, dq)
        else:
            N.check(L.svt_calib_loss(_p(data.x), _p(data.theta), _p(data.w), data.n,
                                     data.n_sectors, _p(data.index), _p(F32), _p(q32), _p(loss),
                                     _p(data.workspace), data.workspace.numel(), _stream(None)),
                    "svt_calib_loss")
        return loss[0]

    @staticmethod
    def backward(ctx, gL):
        L = N.load()
        dF, dq = ctx.saved_tensors
        g = gL.to(torch.float32).contiguous().reshape(1)
        out_F = torch.empty_like(dF)
        out_q = torch.empty_like(dq)
        N.check(L.svt_calib_grad_scale(_p(g), _p(dF), _p(dq), ctx.data.n_sectors, _p(out_F),
                                       _p(out_q), _stream(None)), "svt_calib_grad_scale")
        return out_F, out_q, None


class CalibLossUnfused(torch.autograd.Function):
    """The same loss with the forward and the backward as separate passes
    (svt_calib_loss, then svt_calib_loss_backward, which reads the tracks
    again): for callers that evaluate the loss far more often than its
    gradient."""

    @staticmethod
    def forward(ctx, F, q, data: CalibData):
        L = N.load()
        F32, q32 = _f32(F), _f32(q)
        loss = torch.empty(1, dtype=torch.float32, device=F.device)
        N.check(L.svt_calib_loss(_p(data.x), _p(data.theta), _p(data.w), data.n, data.n_sectors,
                                 _p(data.index), _p(F32), _p(q32), _p(loss), _p(data.workspace),
                                 data.workspace.numel(), _stream(None)), "svt_calib_loss")
        ctx.data = data
        ctx.save_for_backward(F32, q32)
        return loss[0]

    @staticmethod
    def backward(ctx, gL):
        L = N.load()
        data = ctx.data
        F32, q32 = ctx.saved_tensors
        g = gL.to(torch.float32).contiguous().reshape(1)
        dF = torch.empty_like(F32)
        dq = torch.empty_like(q32)
        N.check(L.svt_calib_loss_backward(_p(data.x), _p(data.theta), _p(data.w), data.n,
                                          data.n_sectors, _p(data.index), _p(F32), _p(q32),
                                          _p(g), _p(dF), _p(dq), _p(data.workspace),
                                          data.workspace.numel(), _stream(None)),
                "svt_calib_loss_backward")
        return dF, dq, None


class CalibLossFit(torch.autograd.Function):
    """The loss (differentiable in F and q, as CalibLoss) together with the
    fitted parameters y = F[s] x + q[s] of every track (sector order; not
    differentiated) from one pass over the tracks: for a calibration step
    that also monitors the fits."""

    @staticmethod
    def forward(ctx, F, q, data: CalibData):
        L = N.load()
        F32, q32 = _f32(F), _f32(q)
        loss = torch.empty(1, dtype=torch.float32, device=F.device)
        y = torch.empty((max(data.n, 1), 6), dtype=torch.float32, device=F.device)
        dF = torch.empty_like(F32)
        dq = torch.empty_like(q32)
        N.check(L.svt_calib_loss_grad(_p(data.x), _p(data.theta), _p(data.w), data.n,
                                      data.n_sectors, _p(data.index), _p(F32), _p(q32), _p(loss),
                                      _p(dF), _p(dq), _p(y), _p(data.workspace),
                                      data.workspace.numel(), _stream(None)),
                "svt_calib_loss_grad")
        ctx.data = data
        ctx.save_for_backward(dF, dq)
        y = y[: data.n]
        ctx.mark_non_differentiable(y)
        return loss[0], y

    @staticmethod
    def backward(ctx, gL, gy):
        return CalibLoss.backward(ctx, gL)


def calib_loss_and_fit(F, q, data: CalibData):
    """(L, y) from one pass: L differentiable in F and q, y the fitted parameters."""
    return CalibLossFit.apply(F, q, data)


def fit_fp32(F, q, data: CalibData):
    return FitFP32.apply(F, q, data)


def calib_loss(F, q, data: CalibData, fused: bool = True):
    return (CalibLoss if fused else CalibLossUnfused).apply(F, q, data)
