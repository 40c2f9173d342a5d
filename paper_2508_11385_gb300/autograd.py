"""Differentiation of scalar-valued trees through torch.autograd.

``scalar(fn, *tensors)`` evaluates ``fn(*Mats)`` -- a Reduction such as
``accu(square(W % X - Y)) + 1e-3 * accu(square(W))`` -- with one fused
kernel, and its backward pass is one fused adjoint kernel that recomputes the
tree's forward values per element and runs the reverse sweep through the
node types, writing every input's gradient.  Nothing but the inputs is saved
between the passes.  The paper's motivation for gradients is the optimisation
library built on it (Sec. 6: ensmallen and mlpack on top of Bandicoot).
"""
from __future__ import annotations

import torch

from . import expr as E
from . import lib as L


def _grad_like(t: torch.Tensor) -> torch.Tensor:
    return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=t.device)


class _TreeScalar(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fn, *tensors):
        mats = [E.Mat(t.detach()) for t in tensors]
        red = fn(*mats)
        if not isinstance(red, E.Reduction):
            raise TypeError("fn must return a reduction (accu / sum / mean over all elements)")
        r = red.eval()
        ctx.fn = fn
        ctx.save_for_backward(*tensors)
        return r

    @staticmethod
    def backward(ctx, g):
        tensors = ctx.saved_tensors
        mats = [E.Mat(t.detach()) for t in tensors]
        red = ctx.fn(*mats)
        tree, leaves, cmats = E.lower(red.expr)
        # gradient buffers in the leaves' own layouts, in descriptor order
        by_ptr = {}
        grads = []
        for m in leaves:
            gt = _grad_like(m.tensor)
            grads.append(gt)
            by_ptr[m.tensor.data_ptr()] = gt
        gm = [E.Mat(gt).cmat() for gt in grads]
        dev = tensors[0].device
        acc = E._ACC[leaves[0].dtype]
        up = g.detach().to(dtype=acc).reshape(()).contiguous()
        with torch.cuda.device(dev):
            L.coot_eval_adjoint(E.context(dev), tree, cmats, L.reduce(red.kind, red.dim, red.norm_type),
                                up.data_ptr(), gm, E._stream_ptr())
        out = [None]
        for t in tensors:
            gt = by_ptr.get(t.data_ptr())
            out.append(gt if (gt is not None and t.requires_grad) else None)
        return tuple(out)


def scalar(fn, *tensors):
    """L = fn(*Mats) as a differentiable 0-d tensor (fused forward, fused
    adjoint backward)."""
    return _TreeScalar.apply(fn, *tensors)


def loss_l2_schur(W, X, Y, lam=1e-3):
    """L = accu(square(W % X - Y)) + lam * accu(square(W)) (the differentiation
    workload), fused into one accu by linearity."""
    return scalar(lambda w, x, y: E.accu(E.square(w % x - y)) + lam * E.accu(E.square(w)), W, X, Y)
