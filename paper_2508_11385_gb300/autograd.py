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

import ctypes
import threading

import torch

from . import expr as E
from . import lib as L


def _grad_like(t: torch.Tensor) -> torch.Tensor:
    # empty_like keeps the strides of a dense tensor (a column-major leaf gets
    # a column-major gradient); anything else gets them spelled out
    if t.is_contiguous() or (t.dim() == 2 and t.t().is_contiguous()):
        return torch.empty_like(t)
    return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=t.device)


# the current stream's raw handle of a device: torch's direct query where it
# has one (no Stream object is built), else the public API
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream_of(dev: torch.device) -> int:
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    if _raw_stream is not None:
        return _raw_stream(idx)
    return torch.cuda.current_stream(dev).cuda_stream


def _cmat(t: torch.Tensor):
    n_rows, n_cols = t.shape
    ld = t.stride(1) if n_cols > 1 else max(n_rows, 1)
    return L.mat(t.data_ptr(), L.DTYPE_CODE[E._DTYPE[t.dtype]], n_rows, n_cols, ld)


class Loss:
    """A scalar loss lowered once for inputs of fixed shapes and layouts.

    The C-ABI arguments of both calls (the leaves' coot_mat arrays, the
    gradients' arrays) are built once per set of device pointers and kept,
    so a repeated step with the same tensors costs two launches and little
    host work."""

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
        self._tree_ref = ctypes.byref(self.tree)
        self._leaf_arrays = {}  # device pointers of the inputs -> coot_mat array of the leaves
        self._grad_arrays = {}  # (input pointers, gradient pointers) -> coot_mat array of the gradients
        self._ctx = {}

    def __call__(self, *tensors):
        return _LossFn.apply(self, *tensors)

    def _context(self, dev):
        h = self._ctx.get(dev)
        if h is None:
            h = self._ctx[dev] = E.context(dev)
        return h

    def _leaves(self, tensors):
        key = tuple((t.data_ptr(), t.shape, t.stride(), t.dtype) for t in tensors)
        arr = self._leaf_arrays.get(key)
        if arr is None:
            if len(self._leaf_arrays) > 64:
                self._leaf_arrays.clear()
            arr = (L.coot_mat * len(self.leaf_pos))(*[_cmat(tensors[p].detach()) for p in self.leaf_pos])
            self._leaf_arrays[key] = arr
        return key, arr

    # the two C-ABI calls, usable without autograd
    def forward(self, *tensors, out=None):
        dev = tensors[0].device
        r = torch.empty((), dtype=self.acc, device=dev) if out is None else out
        _, arr = self._leaves(tensors)
        L._check(L._lib.coot_eval(self._context(dev), self._tree_ref, arr, len(self.leaf_pos), None, self.red,
                                  r.data_ptr(), _stream_of(dev)))
        return r

    def backward(self, upstream, *tensors, grads=None):
        dev = tensors[0].device
        if grads is None:
            grads = [_grad_like(t) for t in tensors]
        key, arr = self._leaves(tensors)
        gkey = (key, tuple(g.data_ptr() if g is not None else 0 for g in grads))
        garr = self._grad_arrays.get(gkey)
        if garr is None:
            if len(self._grad_arrays) > 64:
                self._grad_arrays.clear()
            gm = [(_cmat(grads[p]) if grads[p] is not None else L.mat(None, arr[i].dtype, arr[i].n_rows,
                                                                         arr[i].n_cols))
                  for i, p in enumerate(self.leaf_pos)]
            garr = (L.coot_mat * len(gm))(*gm)
            self._grad_arrays[gkey] = garr
        up = upstream.detach()
        if up.dtype != self.acc or up.dim() != 0 or not up.is_contiguous():
            up = up.to(dtype=self.acc).reshape(()).contiguous()
        L._check(L._lib.coot_eval_adjoint(self._context(dev), self._tree_ref, arr, len(self.leaf_pos), self.red,
                                          up.data_ptr(), garr, _stream_of(dev)))
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
    key = (lam, W.shape, W.stride(), X.stride(), Y.stride(), W.dtype, W.device)
    f = _cache.get(key)
    if f is None or (X.shape, Y.shape, X.dtype, Y.dtype) != (W.shape, W.shape, W.dtype, W.dtype):
        with _cache_lock:
            f = Loss(lambda w, x, y: E.accu(E.square(w % x - y)) + lam * E.accu(E.square(w)), W, X, Y)
            if (X.shape, Y.shape, X.dtype, Y.dtype) == (W.shape, W.shape, W.dtype, W.dtype):
                _cache[key] = f
    return f(W, X, Y)
