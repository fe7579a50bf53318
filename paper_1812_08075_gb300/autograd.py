"""torch.autograd wrapper of the SIPG apply: y = A(kappa) x with gradients with respect
to x (the transposed apply) and the per-quadrature-point kappa, both from libdg's
adjoint kernels (dg_apply_adjoint). FP64, scalar problem; x holds one vector [ndofs] or
nrhs vectors [nrhs, ndofs] (nrhs <= the operator's max_rhs) that share one kappa, whose
gradient is then summed over the right-hand sides."""
from __future__ import annotations

import torch

from . import dg


class DGApply(torch.autograd.Function):
    """y = A(kappa) x. Inputs: x [ndofs] or [nrhs, ndofs], kappa_vol [ncell*m^3],
    kappa_face [ncell*6*m^2] (CUDA, float64); op is a ``dg.Operator``."""

    @staticmethod
    def forward(ctx, x, kappa_vol, kappa_face, op):
        x = x.contiguous()
        kappa_vol = kappa_vol.contiguous()
        kappa_face = kappa_face.contiguous()
        op.set_kappa(kappa_vol, kappa_face)
        y = op.apply(x)
        ctx.save_for_backward(x, kappa_vol, kappa_face)
        ctx.op = op
        return y

    @staticmethod
    def backward(ctx, grad_y):
        x, kv, kf = ctx.saved_tensors
        op = ctx.op
        op.set_kappa(kv, kf)
        g = grad_y.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        dx = torch.empty_like(x)
        want_k = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        dkv = torch.empty_like(kv) if want_k else None
        dkf = torch.empty_like(kf) if want_k else None
        dg.dg_apply_adjoint(op.handle, g.data_ptr(), x.data_ptr() if want_k else None, dx.data_ptr(),
                            dkv.data_ptr() if want_k else None, dkf.data_ptr() if want_k else None,
                            torch.cuda.current_stream().cuda_stream, nrhs=nrhs)
        return (dx if ctx.needs_input_grad[0] else None,
                dkv if ctx.needs_input_grad[1] else None,
                dkf if ctx.needs_input_grad[2] else None, None)


def dg_apply(op, x, kappa_vol, kappa_face):
    """Differentiable y = A(kappa) x."""
    return DGApply.apply(x, kappa_vol, kappa_face, op)
