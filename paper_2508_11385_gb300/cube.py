"""Armadillo's Cube<eT> (Sec. 2): n_rows x n_cols x n_slices, slice after
slice, each slice a column-major matrix.

Element-wise cube expressions are matrix expressions over a re-view of the
same memory, so they run through the same fused kernels:

* the slices side by side, an n_rows x (n_cols * n_slices) matrix, for
  element-wise results, full reductions, reductions along dim 0 (per column
  of every slice) and, with one segment per slice, along dim 1 (per row of
  every slice);
* every slice as one column, an (n_rows * n_cols) x n_slices matrix, for
  reductions and scans along dim 2 (across slices, per element).

``each_slice(fn, *cubes)`` evaluates a matrix expression on every slice as a
batch: one persistent kernel over all slices (the batched family).

    Q = coot.Cube(torch.randn(64, 48, 100, device="cuda").permute(...))
    R = coot.Cube(...)
    Y = (Q % R + 1).eval()                      # a cube
    s = coot.sum(coot.exp(Q), 2).eval()          # 64 x 48 x 1
    t = coot.each_slice(lambda A, B: coot.accu(A % B), Q, R)   # one value per slice
"""
from __future__ import annotations

import numbers

import torch

from . import expr as E
from . import lib as L

__all__ = ["Cube", "cube_empty", "each_slice"]


def cube_empty(n_rows, n_cols, n_slices, dtype=torch.float32, device="cuda"):
    """An uninitialised cube tensor in Armadillo's layout (strides 1, n_rows,
    n_rows * n_cols)."""
    return torch.empty((n_slices, n_cols, n_rows), dtype=dtype, device=device).permute(2, 1, 0)


def _packed(t: torch.Tensor):
    r, c, s = t.shape
    return t.stride(0) == 1 or r <= 1, t.stride(1) == r or c <= 1, t.stride(2) == r * c or s <= 1


class _CubeNode:
    """An element-wise cube expression: op over children (cubes, nodes or
    scalars), lowered to a matrix expression per view."""

    def __init__(self, op, children=(), k=0.0):
        self.op, self.children, self.k = op, tuple(children), float(k)
        shapes = {c.shape3 for c in self.children if isinstance(c, (Cube, _CubeNode))}
        if len(shapes) != 1:
            raise ValueError("cube operands differ in shape: %s" % sorted(shapes))
        self.shape3 = shapes.pop()

    def to_expr(self, mode):
        kids = [c.to_expr(mode) if isinstance(c, (Cube, _CubeNode)) else c for c in self.children]
        if self.op in (L.N_PLUS, L.N_MINUS, L.N_SCHUR, L.N_DIV):
            a, b = kids
            return {L.N_PLUS: lambda: a + b, L.N_MINUS: lambda: a - b, L.N_SCHUR: lambda: a % b,
                    L.N_DIV: lambda: a / b}[self.op]()
        if self.op == "scalar":
            return self._fn(kids[0])
        return E.Expr(self.op, (kids[0],), k=self.k)

    # the same operators as a matrix expression
    def _bin(self, op, o, rev=False):
        if isinstance(o, numbers.Real):
            k = float(o)
            fn = {(L.N_PLUS, False): lambda e: e + k, (L.N_PLUS, True): lambda e: k + e,
                  (L.N_MINUS, False): lambda e: e - k, (L.N_MINUS, True): lambda e: k - e,
                  (L.N_SCAL_TIMES, False): lambda e: e * k, (L.N_SCAL_TIMES, True): lambda e: k * e,
                  (L.N_DIV, False): lambda e: e / k, (L.N_DIV, True): lambda e: k / e}[(op, rev)]
            n = _CubeNode("scalar", (self,))
            n._fn = fn
            return n
        if not isinstance(o, (Cube, _CubeNode)):
            raise TypeError("a cube combines with a cube or a scalar")
        return _CubeNode(op, (o, self) if rev else (self, o))

    def __add__(self, o):
        return self._bin(L.N_PLUS, o)

    def __radd__(self, o):
        return self._bin(L.N_PLUS, o, True)

    def __sub__(self, o):
        return self._bin(L.N_MINUS, o)

    def __rsub__(self, o):
        return self._bin(L.N_MINUS, o, True)

    def __mul__(self, o):
        if not isinstance(o, numbers.Real):
            raise TypeError("cube * cube is not element-wise; use % for the Schur product")
        return self._bin(L.N_SCAL_TIMES, o)

    def __rmul__(self, o):
        return self.__mul__(o)

    def __truediv__(self, o):
        return self._bin(L.N_DIV, o)

    def __rtruediv__(self, o):
        return self._bin(L.N_DIV, o, True)

    def __mod__(self, o):
        return self._bin(L.N_SCHUR, o)

    def __rmod__(self, o):
        return self._bin(L.N_SCHUR, o, True)

    def __neg__(self):
        return _CubeNode(L.N_NEG, (self,))

    # hooks used by the library's functions (exp, accu, sum, ...)
    def _cube_unary(self, op):
        return _CubeNode(op, (self,))

    def _cube_reduce(self, kind, dim, norm_type=0):
        return CubeReduction(kind, self, dim, norm_type)

    def eval(self, out=None, fused=True, stream=None):
        """Evaluate into a cube tensor (allocated in Armadillo's layout when
        out is None)."""
        r, c, s = self.shape3
        e = self.to_expr("cols")
        if out is None:
            out = cube_empty(r, c, s, _leaves_dtype(e), _device(self))
        E.evaluate(e, out=Cube(out).view("cols"), fused=fused, stream=stream)
        return out


def _device(node):
    for c in node.children:
        if isinstance(c, Cube):
            return c.tensor.device
        if isinstance(c, _CubeNode):
            return _device(c)
    raise ValueError("no cube operand")


class Cube(_CubeNode):
    """A cube in device memory, wrapping a 3-D torch tensor (n_rows, n_cols,
    n_slices) with strides (1, n_rows, n_rows * n_cols), e.g.
    ``cube_empty(r, c, s)`` or ``t.permute(2, 1, 0)`` of a contiguous
    (s, c, r) tensor."""

    def __init__(self, t: torch.Tensor):
        if t.dim() != 3:
            raise ValueError("Cube wraps a 3-D tensor")
        if not all(_packed(t)):
            raise ValueError("cube tensor must have strides (1, n_rows, n_rows*n_cols); use cube_empty or "
                             "t.permute(2, 1, 0).contiguous().permute(2, 1, 0)")
        if t.dtype not in E._DTYPE:
            raise TypeError("unsupported dtype %s" % t.dtype)
        self.tensor = t
        self.shape3 = tuple(int(x) for x in t.shape)
        self.op, self.children, self.k = L.N_LEAF, (), 0.0

    @property
    def n_rows(self):
        return self.shape3[0]

    @property
    def n_cols(self):
        return self.shape3[1]

    @property
    def n_slices(self):
        return self.shape3[2]

    def slice(self, s):
        """Slice s as a matrix (a view)."""
        return E.Mat(self.tensor[:, :, s])

    def view(self, mode):
        """The same memory as a matrix: "cols" -- n_rows x (n_cols*n_slices);
        "elems" -- (n_rows*n_cols) x n_slices."""
        r, c, s = self.shape3
        if mode == "cols":
            return torch.as_strided(self.tensor, (r, c * s), (1, max(r, 1)))
        return torch.as_strided(self.tensor, (r * c, s), (1, max(r * c, 1)))

    def to_expr(self, mode):
        return E.Mat(self.view(mode))

    def eval(self, out=None, fused=True, stream=None):
        return self.tensor if out is None else super().eval(out, fused, stream)


def _leaves_dtype(e):
    _, leaves, _ = E.lower(e)
    return leaves[0].tensor.dtype


class CubeReduction:
    """A reduction of a cube expression along dim 0, 1 or 2 (-1: all
    elements); cumsum returns a cube."""

    def __init__(self, kind, node, dim, norm_type=0):
        if dim not in (-1, 0, 1, 2):
            raise ValueError("a cube reduces along dim 0, 1 or 2 (-1: all elements)")
        if kind == L.R_CUMSUM and dim == -1:
            dim = 0
        self.kind, self.node, self.dim, self.norm_type = kind, node, dim, norm_type

    def eval(self, fused=True, stream=None):
        r, c, s = self.node.shape3
        kind, dim = self.kind, self.dim
        if kind == L.R_CUMSUM:
            e = self.node.to_expr("elems" if dim == 2 else "cols")
            out = cube_empty(r, c, s, _leaves_dtype(e), _device_of(self.node))
            red = E.Reduction(kind, e, 1 if dim == 2 else dim, 0, n_seg=s if dim == 1 else 0)
            E.evaluate(e, reduction=red, materialise=Cube(out).view("elems" if dim == 2 else "cols"),
                       fused=fused, stream=stream)
            return out
        if dim == -1:
            _, v = E.evaluate(self.node.to_expr("cols"), reduction=E.Reduction(kind, self.node.to_expr("cols"), -1,
                                                                                 self.norm_type),
                              fused=fused, stream=stream)
            return v
        if dim == 0:
            e = self.node.to_expr("cols")
            _, v = E.evaluate(e, reduction=E.Reduction(kind, e, 0, self.norm_type), fused=fused, stream=stream)
            return v.reshape(s, c).t().unsqueeze(0)                      # (1, c, s)
        if dim == 1:
            e = self.node.to_expr("cols")
            _, v = E.evaluate(e, reduction=E.Reduction(kind, e, 1, self.norm_type, n_seg=s), fused=fused,
                              stream=stream)
            return v.unsqueeze(1)                                         # (r, 1, s)
        e = self.node.to_expr("elems")
        _, v = E.evaluate(e, reduction=E.Reduction(kind, e, 1, self.norm_type), fused=fused, stream=stream)
        return v.reshape(c, r).t().unsqueeze(2)                           # (r, c, 1)


def _device_of(node):
    return node.tensor.device if isinstance(node, Cube) else _device(node)


def each_slice(fn, *cubes, stream=None):
    """Armadillo's Q.each_slice(): fn maps the slices' matrices to a matrix
    expression or to a full reduction (accu / sum / mean over all elements);
    it is evaluated for every slice as one batch.  Returns a cube of the
    per-slice results, or a vector of one reduction value per slice."""
    if not cubes:
        raise ValueError("each_slice needs at least one cube")
    n = cubes[0].n_slices
    if any(c.n_slices != n for c in cubes):
        raise ValueError("cubes differ in the number of slices")
    res = fn(*[c.slice(0) for c in cubes])
    red = res if isinstance(res, E.Reduction) else None
    e = red.expr if red is not None else E._as_expr(res)
    tree, leaves, _ = E.lower(e)
    base = [c.tensor.data_ptr() for c in cubes]
    # leaf l of slice 0 is some cube's slice 0: map it to that cube
    which = [base.index(m.tensor.data_ptr()) for m in leaves]
    dev = cubes[0].tensor.device
    probs = (L.coot_mat * (n * len(leaves)))()
    for q in range(n):
        for li, ci in enumerate(which):
            probs[q * len(leaves) + li] = E.Mat(cubes[ci].tensor[:, :, q]).cmat()
    with torch.cuda.device(dev):
        ctx = E.context(dev)
        s = E._stream_ptr(stream)
        if red is None:
            r, c = e.shape
            out = cube_empty(r, c, n, leaves[0].tensor.dtype, dev)
            outs = (L.coot_mat * n)(*[E.Mat(out[:, :, q]).cmat() for q in range(n)])
            L.coot_eval_batched(ctx, tree, n, len(leaves), probs, outs, L.reduce(), None, s)
            return out
        acc = E._ACC[leaves[0].dtype]
        v = torch.empty(n, dtype=acc, device=dev)
        L.coot_eval_batched(ctx, tree, n, len(leaves), probs, None,
                            L.reduce(red.kind, red.dim, red.norm_type), v.data_ptr(), s)
        return v
