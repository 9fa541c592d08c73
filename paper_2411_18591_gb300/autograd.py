"""torch.autograd wrappers over the C ABI: propagations that take part in a PyTorch graph.

The gradients follow PyTorch's convention for complex tensors, which for a real loss is
g = dL/dRe + i dL/dIm, the same convention as the library's backward calls: the gradient of a
field through a propagation is the adjoint propagation of the output gradient (§4), and the
gradient of a phase mask phi in M = exp(i phi) is sum_b Im(g_y conj(M x_b)) with g_y the
adjoint-propagated output gradient. Every step runs in libtop's kernels.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import binding as B


class _Propagate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, field, phase, dy, dx, lam, z, pad, method):
        pre = B.Modulation(phase=phase) if phase is not None else None
        out = B.top_propagate(field.contiguous(), dy, dx, lam, z, pad, method, pre=pre)
        ctx.save_for_backward(field if phase is not None else None, phase)
        ctx.args = (dy, dx, lam, z, pad, method)
        ctx.shape = field.shape
        return out.reshape(field.shape)

    @staticmethod
    def backward(ctx, grad_out):
        field, phase = ctx.saved_tensors
        dy, dx, lam, z, pad, method = ctx.args
        g = grad_out.contiguous().to(torch.complex64)
        want_in = ctx.needs_input_grad[0]
        want_phase = phase is not None and ctx.needs_input_grad[1]
        pre = B.Modulation(phase=phase) if phase is not None else None
        gphase = torch.zeros_like(phase) if want_phase else None
        gin = B.top_propagate_backward(g, dy, dx, lam, z, pad, method, pre=pre,
                                       saved_in=field.contiguous() if want_phase else None,
                                       want_grad_in=want_in, grad_phase=gphase)
        return (gin.reshape(ctx.shape) if want_in else None), gphase, None, None, None, None, None, None


def propagate(field: torch.Tensor, dy: float, dx: float, lam, z, pad: float = 2.0, method="as",
              phase: Optional[torch.Tensor] = None) -> torch.Tensor:
    """P_z(exp(i phase) * field) (Eq. 1, Eq. 4), differentiable with respect to ``field`` and the
    phase mask ``phase`` (float32 [ny, nx], shared by the batch, or [batch, ny, nx])."""
    return _Propagate.apply(field, phase, dy, dx, lam, z, pad, method)
