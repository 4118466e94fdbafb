"""torch.autograd binding of the differentiable timing pass.

``SmoothedTiming.apply(xy, ctx, w_tns, w_wns)`` sets the cell positions
(``sta_set_positions``), runs the timing pass (``sta_update_timing``) and the
hand-written adjoint (``sta_backward``), and returns the smoothed objective
J = w_tns * TNS_g + w_wns * WNS_g as a 0-d tensor; its backward returns
dJ/d(xy).  Every number comes from the CUDA library; this file only moves
tensors.  The context must be created from a placed design with
gamma_ns > 0.
"""
from __future__ import annotations

import torch

from . import sta


class SmoothedTiming(torch.autograd.Function):
    @staticmethod
    def forward(fctx, xy: torch.Tensor, ctx: "sta.Context", w_tns: float = 1.0, w_wns: float = 1.0):
        assert xy.is_cuda and xy.dtype == torch.float32 and xy.is_contiguous()
        ctx.set_positions(xy)
        ctx.update_timing()
        grad = torch.empty((ctx.C, 2), dtype=torch.float64, device=xy.device)
        J, _, _ = ctx.backward(w_tns, w_wns, grad_out=grad)
        fctx.save_for_backward(grad)
        return J.to(torch.float64)

    @staticmethod
    def backward(fctx, gout):
        (grad,) = fctx.saved_tensors
        return (gout * grad).to(torch.float32).reshape(-1), None, None, None


def smoothed_objective(xy: torch.Tensor, ctx: "sta.Context", w_tns: float = 1.0, w_wns: float = 1.0):
    return SmoothedTiming.apply(xy, ctx, w_tns, w_wns)
