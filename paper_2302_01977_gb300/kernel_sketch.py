"""Differentiable matrix-free kernel sketch S = K(X, X; h) R.

``KernelSketch`` is a ``torch.autograd.Function`` whose forward pass is
``sketch_kernel_apply`` (tiles of the Gaussian kernel matrix computed next to
the SJLT product, never stored) and whose backward pass is
``sketch_kernel_adjoint`` (the hand-written adjoint: dX and dh from dS, tiles of
K recomputed).  Both run in libjlsketch; this module only marshals tensors.

The sketch is the random sample of the matrix-free setting of the paper
(Sec. 1.1) for kernel matrices of points (Sec. 8.1); its gradient in the points
and the width is this project's extension.
"""
from __future__ import annotations

import torch

from . import jlsketch as jl


class KernelSketch(torch.autograd.Function):
    """S = K(X, X; h) R for an SJLT handle ``op`` (a ``jlsketch.Sketch``)."""

    @staticmethod
    def forward(ctx, X, h, op):
        hv = float(h)
        d = jl.sketch_dims(op.h)["d_total"]
        S = torch.empty((X.shape[0], d), dtype=torch.float32, device=X.device)
        jl.sketch_kernel_apply(op.h, X, X, hv, S)
        ctx.save_for_backward(X)
        ctx.hv, ctx.op = hv, op
        ctx.h_like = h if isinstance(h, torch.Tensor) else None
        return S

    @staticmethod
    def backward(ctx, dS):
        (X,) = ctx.saved_tensors
        dS = dS.contiguous()
        dX = torch.empty_like(X)
        dh = torch.empty(1, dtype=torch.float64, device=X.device)
        jl.sketch_kernel_adjoint(ctx.op.h, X, ctx.hv, dS, dX, dh)
        gh = None
        if ctx.h_like is not None:
            gh = dh.reshape(ctx.h_like.shape).to(dtype=ctx.h_like.dtype, device=ctx.h_like.device)
        return dX, gh, None


def kernel_sketch(X, h, op):
    """Differentiable S = K(X, X; h) R (X: contiguous float32 CUDA tensor, n x 3)."""
    return KernelSketch.apply(X, h, op)
