"""torch.autograd.Function around fstat_grad.

``FStatBin.apply(theta, ctx_obj)`` returns 2F at the frequency offset
theta[:, 2] for the templates (alpha, delta, fdot) = theta[:, (0, 1, 3)];
its backward multiplies the incoming gradient by d(2F)/d(alpha, delta, f,
fdot) that the library's adjoint kernel computed in the same call.  Only
argument marshalling happens here: the template records are assembled on
the device from ``theta`` and a base record tensor.
"""
from __future__ import annotations

import numpy as np
import torch

from . import TEMPLATE_DTYPE, fstat_grad, pack_templates


class BinSearch:
    """Fixed inputs of a gradient search: plan, data, gaps and the integer
    fields of the templates (spans, gap offsets)."""

    def __init__(self, plan, x_h, templates_np, gaps=None):
        self.plan = plan
        self.x_h = x_h
        self.gaps = gaps
        base = pack_templates(templates_np, device=x_h.device)
        self.base = base.view(torch.int64).view(len(templates_np), TEMPLATE_DTYPE.itemsize // 8)

    def records(self, theta: torch.Tensor) -> torch.Tensor:
        rec = self.base.clone()
        f = rec.view(torch.float64)
        f[:, 0] = theta[:, 0]
        f[:, 1] = theta[:, 1]
        f[:, 2] = theta[:, 3]
        return rec.view(torch.uint8).reshape(-1)


class FStatBin(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta: torch.Tensor, search: BinSearch):
        th = theta.detach().to(torch.float64).contiguous()
        two_f, grad = fstat_grad(search.plan, search.x_h, search.records(th), th[:, 2], search.gaps)
        ctx.save_for_backward(grad)
        return two_f

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g[:, None] * grad, None


def theta_of(templates_np, df) -> np.ndarray:
    """(alpha, delta, df, fdot) rows from template records and offsets."""
    return np.stack([templates_np["alpha"], templates_np["delta"], np.asarray(df, np.float64),
                     templates_np["fdot"]], axis=1)
