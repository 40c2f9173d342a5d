"""Differentiation of scalar-valued trees through torch.autograd.

``Loss(fn, *examples)`` lowers ``fn(*Mats)`` -- a Reduction such as
``accu(square(W % X - Y)) + 1e-3 * accu(square(W))`` -- once; calling it on
tensors of the same shapes evaluates the loss with one fused kernel and, on
backward, runs one fused adjoint kernel that recomputes the tree's forward
values per element and sweeps back through the node types, writing every
input's gradient.  Nothing but the inputs is saved between the passes.  The
paper's motivation for gradients is the optimisation library built on top of
it (Sec. 7: ensmallen and mlpack being adapted to Bandicoot).
"""
from __future__ import annotations

import threading

import torch

from . import expr as E
from . import lib as L


def _grad_like(t: torch.Tensor) -> torch.Tensor:
    return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=t.device)


def _cmat(t: torch.Tensor):
    n_rows, n_cols = t.shape
    ld = t.stride(1) if n_cols > 1 else max(n_rows, 1)
    return L.mat(t.data_ptr(), L.DTYPE_CODE[E._DTYPE[t.dtype]], n_rows, n_cols, ld)


class Loss:
    """A scalar loss lowered once for inputs of fixed shapes and layouts."""

    def __init__(self, fn, *examples):
        mats = [E.Mat(t.detach()) for t in examples]
        red = fn(*mats)
        if not isinstance(red, E.Reduction):
            raise TypeError("fn must return a reduction (accu / sum / mean over all elements)")
        self.tree, leaves, _ = E.lower(red.expr)
        ptrs = [t.data_ptr() for t in examples]
        self.leaf_pos = [ptrs.index(m.tensor.data_ptr()) for m in leaves]
        self.red = L.reduce(red.kind, red.dim, red.norm_type)
        self.acc = E._ACC[leaves[0].dtype]
        self.signature = tuple((tuple(t.shape), tuple(t.stride()), t.dtype) for t in examples)
        self.n_inputs = len(examples)

    def __call__(self, *tensors):
        return _LossFn.apply(self, *tensors)

    # the two C-ABI calls, usable without autograd
    def forward(self, *tensors, out=None):
        dev = tensors[0].device
        r = torch.empty((), dtype=self.acc, device=dev) if out is None else out
        cm = [_cmat(tensors[p].detach()) for p in self.leaf_pos]
        L.coot_eval(E.context(dev), self.tree, cm, None, self.red, r.data_ptr(), E._stream_ptr())
        return r

    def backward(self, upstream, *tensors, grads=None):
        dev = tensors[0].device
        if grads is None:
            grads = [_grad_like(t) for t in tensors]
        cm = [_cmat(tensors[p].detach()) for p in self.leaf_pos]
        gm = [(_cmat(grads[p]) if grads[p] is not None else L.mat(None, cm[i].dtype, cm[i].n_rows, cm[i].n_cols))
              for i, p in enumerate(self.leaf_pos)]
        up = upstream.detach().to(dtype=self.acc).reshape(()).contiguous()
        L.coot_eval_adjoint(E.context(dev), self.tree, cm, self.red, up.data_ptr(), gm, E._stream_ptr())
        return grads


class _LossFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, loss, *tensors):
        ctx.loss = loss
        ctx.save_for_backward(*tensors)
        return loss.forward(*tensors)

    @staticmethod
    def backward(ctx, g):
        tensors = ctx.saved_tensors
        need = ctx.needs_input_grad[1:]
        grads = [_grad_like(t) if need[i] else None for i, t in enumerate(tensors)]
        ctx.loss.backward(g, *tensors, grads=grads)
        return (None, *grads)


def scalar(fn, *tensors):
    """L = fn(*Mats) as a differentiable 0-d tensor (fused forward, fused
    adjoint backward); lowers fn on every call -- keep a Loss to reuse it."""
    return Loss(fn, *tensors)(*tensors)


_cache = {}
_cache_lock = threading.Lock()


def loss_l2_schur(W, X, Y, lam=1e-3):
    """L = accu(square(W % X - Y)) + lam * accu(square(W)) (the
    differentiation workload), fused into one accu by linearity."""
    key = (lam,) + tuple((tuple(t.shape), tuple(t.stride()), t.dtype, t.device) for t in (W, X, Y))
    with _cache_lock:
        f = _cache.get(key)
        if f is None:
            f = Loss(lambda w, x, y: E.accu(E.square(w % x - y)) + lam * E.accu(E.square(w)), W, X, Y)
            _cache[key] = f
    return f(W, X, Y)
