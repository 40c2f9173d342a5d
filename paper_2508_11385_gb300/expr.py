"""Armadillo-style expressions over column-major device matrices.

Mirrors the user API the paper describes (Sec. 2-3): functions and operators
do not compute anything, they return expression objects; evaluation happens
when the expression is assigned (``evaluate`` / ``Mat.eval``) or reduced
(``accu``, ``sum``, ``mean``, ``dot``, ``norm``, ``var``, ``stddev``, ``min``,
``max``, ``index_min``, ``index_max``, ``prod``), and then the whole
tree is handed to the library as one descriptor so it can run as one fused
kernel.

    import paper_2508_11385_gb300 as coot
    A, B, C = (coot.Mat(t) for t in (a, b, c))      # column-major torch tensors
    Y = coot.evaluate(0.5 * A + B % coot.exp(C))     # materialise Y
    s = coot.accu(coot.square(0.5 * A + B % coot.exp(C))).eval()

``%`` is the element-wise (Schur) product as in Armadillo; ``*`` is defined
only between a scalar and a matrix (matrix multiplication is not element-wise
and is not part of this library).
"""
from __future__ import annotations

import builtins
import numbers
import os
import threading

import torch

from . import lib as L

_DTYPE = {torch.float32: "f32", torch.float64: "f64", torch.bfloat16: "bf16", torch.float16: "f16",
          torch.int32: "i32"}
_TORCH = {v: k for k, v in _DTYPE.items()}
_ACC = {"f32": torch.float32, "bf16": torch.float32, "f16": torch.float32, "f64": torch.float64,
        "i32": torch.int64}


# ---------------------------------------------------------------------------
# contexts (one per device, created on first use)
# ---------------------------------------------------------------------------
_ctx_lock = threading.Lock()
_ctxs = {}


def context(device=None):
    """The library context of a CUDA device (kernel caches, workspace)."""
    if device is None:
        device = torch.cuda.current_device()
    if isinstance(device, torch.device):
        device = device.index if device.index is not None else torch.cuda.current_device()
    with _ctx_lock:
        h = _ctxs.get(device)
        if h is None:
            flags = 0
            if os.environ.get("COOT_TUNE", "") in ("1", "on"):
                flags |= L.CTX_TUNE
            h = L.coot_ctx_create(device, flags)
            _ctxs[device] = h
        return h


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# ---------------------------------------------------------------------------
# expression nodes
# ---------------------------------------------------------------------------
MATMUL = "matmul"  # the matrix product: evaluated by the GEMM kernel with the rest fused onto it


class Expr:
    """A node of an expression tree (eOp / eGlue / Op in the paper's terms)."""

    __array_priority__ = 1000

    def __init__(self, op, children=(), k=0.0, view=None):
        self.op = op
        self.children = tuple(children)
        self.k = float(k)
        self.view = view  # (r0, c0, nr, nc) for N_SUBMAT
        self._shape = None

    # ---- shape ---------------------------------------------------------
    @property
    def shape(self):
        if self._shape is None:
            op = self.op
            if op == L.N_SUBMAT:
                self._shape = (self.view[2], self.view[3])
            elif op == L.N_EACH_COL:
                self._shape = (self.children[0].n_rows, self.view)
            elif op == L.N_EACH_ROW:
                self._shape = (self.view, self.children[0].n_cols)
            elif op == L.N_DIAG:
                r, c = self.children[0].shape
                k = self.view
                self._shape = (builtins.max(0, builtins.min(r, c - k) if k >= 0 else builtins.min(r + k, c)), 1)
            elif op == L.N_TRANS:
                r, c = self.children[0].shape
                self._shape = (c, r)
            elif op == MATMUL:
                self._shape = (self.children[0].n_rows, self.children[1].n_cols)
            elif L.N_PLUS <= op <= L.N_DIV:
                sa, sb = self.children[0].shape, self.children[1].shape
                if sa != sb:
                    raise ValueError("incompatible matrix dimensions: %dx%d and %dx%d" % (sa + sb))
                self._shape = sa
            else:
                self._shape = self.children[0].shape
        return self._shape

    @property
    def n_rows(self):
        return self.shape[0]

    @property
    def n_cols(self):
        return self.shape[1]

    @property
    def n_elem(self):
        return self.shape[0] * self.shape[1]

    # ---- operators -----------------------------------------------------
    def __add__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_PLUS, (self,), k=o)
        return Expr(L.N_PLUS, (self, _as_expr(o)))

    def __radd__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_PLUS, (self,), k=o)
        return Expr(L.N_PLUS, (_as_expr(o), self))

    def __sub__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_MINUS_POST, (self,), k=o)
        return Expr(L.N_MINUS, (self, _as_expr(o)))

    def __rsub__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_MINUS_PRE, (self,), k=o)
        return Expr(L.N_MINUS, (_as_expr(o), self))

    def __mul__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_TIMES, (self,), k=o)
        # matrix * matrix is the matrix product (% is the element-wise one)
        o = _as_expr(o)
        if self.n_cols != o.n_rows:
            raise ValueError("matrix product: %dx%d times %dx%d" % (*self.shape, *o.shape))
        return Expr(MATMUL, (self, o))

    def __rmul__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_TIMES, (self,), k=o)
        return _as_expr(o).__mul__(self)

    def __truediv__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_DIV_POST, (self,), k=o)
        return Expr(L.N_DIV, (self, _as_expr(o)))

    def __rtruediv__(self, o):
        if isinstance(o, numbers.Real):
            return Expr(L.N_SCAL_DIV_PRE, (self,), k=o)
        return Expr(L.N_DIV, (_as_expr(o), self))

    def __mod__(self, o):
        return Expr(L.N_SCHUR, (self, _as_expr(o)))

    def __rmod__(self, o):
        return Expr(L.N_SCHUR, (_as_expr(o), self))

    def __neg__(self):
        return Expr(L.N_NEG, (self,))

    def t(self):
        return trans(self)

    def diag(self, k=0):
        """Armadillo's X.diag(k): the k-th diagonal (k > 0 above the main
        one, k < 0 below) as a column vector.  Of a matrix (or a submatrix
        view) it is also a view that ``evaluate(..., out=...)`` and the
        in-place operators can write."""
        r, c = self.shape
        if (k >= 0 and k >= c and c > 0) or (k < 0 and -k >= r and r > 0):
            raise IndexError("diag: diagonal %d outside a %dx%d matrix" % (k, r, c))
        return Expr(L.N_DIAG, (self,), view=int(k))

    def each_col(self):
        """Armadillo's X.each_col(): ``X.each_col() + v`` adds the column
        vector v to every column (also - % / and the reversed forms)."""
        return _Each(self, L.N_EACH_COL)

    def each_row(self):
        """Armadillo's X.each_row(): the same with a row vector per row."""
        return _Each(self, L.N_EACH_ROW)

    # ---- in-place updates of a view (a Mat, a submatrix or a diagonal) ------
    def _assign(self, value):
        evaluate(value, out=self)
        return self

    def __iadd__(self, o):
        return self._assign(self + o)

    def __isub__(self, o):
        return self._assign(self - o)

    def __imul__(self, o):
        return self._assign(self * o)

    def __imod__(self, o):
        return self._assign(self % o)

    def __itruediv__(self, o):
        return self._assign(self / o)

    def eval(self, out=None, fused=True, stream=None):
        return evaluate(self, out=out, fused=fused, stream=stream)


class _Each:
    """X.each_col() / X.each_row(): the other operand of an arithmetic
    operator is a column (row) vector repeated over X's columns (rows)."""

    def __init__(self, x, op):
        self.x, self.op = x, op

    def _rep(self, v):
        v = _as_expr(v)
        if self.op == L.N_EACH_COL:
            if v.n_rows != self.x.n_rows:
                raise ValueError("each_col: needs a %dx1 column vector, got %dx%d" % (self.x.n_rows, *v.shape))
            return broadcast_col(v, self.x.n_cols)
        if v.n_cols != self.x.n_cols:
            raise ValueError("each_row: needs a 1x%d row vector, got %dx%d" % (self.x.n_cols, *v.shape))
        return broadcast_row(v, self.x.n_rows)

    def __add__(self, v):
        return self.x + self._rep(v)

    def __radd__(self, v):
        return self._rep(v) + self.x

    def __sub__(self, v):
        return self.x - self._rep(v)

    def __rsub__(self, v):
        return self._rep(v) - self.x

    def __mod__(self, v):
        return self.x % self._rep(v)

    def __rmod__(self, v):
        return self._rep(v) % self.x

    def __truediv__(self, v):
        return self.x / self._rep(v)

    def __rtruediv__(self, v):
        return self._rep(v) / self.x


class Mat(Expr):
    """A column-major matrix in device memory, wrapping a torch tensor.

    The tensor is 2-D with element (i,j) at data[i*rs + j*ld] (rs =
    t.stride(0), ld = t.stride(1)): column-major when rs == 1, e.g.
    ``torch.empty(n_cols, n_rows).t()``; rs > 1 reads rows rs elements apart
    (a diagonal, every k-th row), one element at a time.  A 1-D tensor is a
    column vector with row stride t.stride(0) (``Z.diagonal()`` works)."""

    def __init__(self, t: torch.Tensor):
        super().__init__(L.N_LEAF)
        rs = 1
        if t.dim() == 1:
            t2 = t.unsqueeze(1)
            n_rows, n_cols, ld = t.shape[0], 1, builtins.max(t.shape[0], 1)
            rs = t.stride(0) if t.shape[0] > 1 else 1
        elif t.dim() == 2:
            t2 = t
            n_rows, n_cols = t.shape
            ld = t.stride(1) if n_cols > 1 else builtins.max(n_rows, 1)
            if n_rows > 1 and t.stride(0) != 1:
                if n_cols > 1 and t.stride(1) == 1:
                    raise ValueError("tensor is row-major (stride(1) == 1): wrap t.t() and use trans(), or "
                                     "t.t().contiguous().t()")
                rs = t.stride(0)
            if n_cols > 1 and ld < (n_rows - 1) * rs + 1 and n_rows > 0:
                raise ValueError("column stride smaller than the rows it spans")
        else:
            raise ValueError("Mat wraps 1-D or 2-D tensors")
        if t.dtype not in _DTYPE:
            raise TypeError("unsupported dtype %s" % t.dtype)
        if t.device.type != "cuda":
            raise ValueError("Mat wraps CUDA tensors (device memory); got %s" % t.device)
        if rs < 1:
            raise ValueError("row stride must be positive")
        self.tensor = t2
        self.dtype = _DTYPE[t.dtype]
        self.ld = int(ld)
        self.rs = int(rs)
        self._shape = (int(n_rows), int(n_cols))

    def submat(self, first_row, first_col, last_row, last_col):
        """Armadillo's X.submat(first_row, first_col, last_row, last_col):
        inclusive last indices."""
        nr, nc = last_row - first_row + 1, last_col - first_col + 1
        if first_row < 0 or first_col < 0 or nr < 0 or nc < 0 or last_row >= self.n_rows or last_col >= self.n_cols:
            raise IndexError("submat: indices out of bounds")
        return Expr(L.N_SUBMAT, (self,), view=(first_row, first_col, nr, nc))

    def cmat(self):
        return L.mat(self.tensor.data_ptr(), L.DTYPE_CODE[self.dtype], self.n_rows, self.n_cols, self.ld,
                     self.rs if self.rs > 1 else 0)


def broadcast_col(v, n_cols):
    """The column vector v repeated as n_cols columns (the operand that
    ``X.each_col() op v`` pairs with X); never materialised."""
    v = _as_expr(v)
    if v.n_cols != 1:
        raise ValueError("broadcast_col: needs a column vector, got %dx%d" % v.shape)
    return Expr(L.N_EACH_COL, (v,), view=int(n_cols))


def broadcast_row(r, n_rows):
    """The row vector r repeated as n_rows rows (``X.each_row() op r``)."""
    r = _as_expr(r)
    if r.n_rows != 1:
        raise ValueError("broadcast_row: needs a row vector, got %dx%d" % r.shape)
    return Expr(L.N_EACH_ROW, (r,), view=int(n_rows))


def _as_expr(x):
    if isinstance(x, Expr):
        return x
    if isinstance(x, torch.Tensor):
        return Mat(x)
    raise TypeError("expected a matrix expression, got %r" % type(x))


# element-wise functions (eOp)
def trans(x):
    return Expr(L.N_TRANS, (_as_expr(x),))


def exp(x):
    if hasattr(x, "_cube_unary"):
        return x._cube_unary(L.N_EXP)
    return Expr(L.N_EXP, (_as_expr(x),))


def log(x):
    if hasattr(x, "_cube_unary"):
        return x._cube_unary(L.N_LOG)
    return Expr(L.N_LOG, (_as_expr(x),))


def abs(x):  # noqa: A001 -- Armadillo's name
    if hasattr(x, "_cube_unary"):
        return x._cube_unary(L.N_ABS)
    return Expr(L.N_ABS, (_as_expr(x),))


def square(x):
    if hasattr(x, "_cube_unary"):
        return x._cube_unary(L.N_SQUARE)
    return Expr(L.N_SQUARE, (_as_expr(x),))


def sqrt(x):
    if hasattr(x, "_cube_unary"):
        return x._cube_unary(L.N_SQRT)
    return Expr(L.N_SQRT, (_as_expr(x),))


# ---------------------------------------------------------------------------
# lowering to the C descriptor
# ---------------------------------------------------------------------------
def lower(expr: Expr, product=None, done=None):
    """(coot_tree, [leaf Mat], [coot_mat]) of an expression; shared
    sub-expressions stay shared (the node list is a DAG).  `product`: a
    matrix-product node that becomes leaf 0 (a GEMM epilogue; the leaf lists
    then start with None).  `done`: {id(product node): Mat} of products
    already evaluated into temporaries, read as leaves."""
    nodes, memo, leaves, leaf_idx = [], {}, [], {}
    done = done or {}
    if product is not None:
        leaves.append(None)

    def visit(e):
        key = id(e)
        if key in memo:
            return memo[key]
        if id(e) in done:
            e = done[id(e)]
        if e is product:
            nodes.append(L.node(L.N_LEAF, leaf=0))
        elif e.op == MATMUL:
            raise NotImplementedError("one matrix product per expression")
        elif e.op == L.N_LEAF:
            lk = (e.tensor.data_ptr(), e.shape, e.ld, e.rs, e.dtype)
            if lk not in leaf_idx:
                leaf_idx[lk] = len(leaves)
                leaves.append(e)
            nodes.append(L.node(L.N_LEAF, leaf=leaf_idx[lk]))
        elif e.op == L.N_SUBMAT:
            a = visit(e.children[0])
            r0, c0, nr, nc = e.view
            nodes.append(L.node(L.N_SUBMAT, a=a, r0=r0, c0=c0, nr=nr, nc=nc))
        elif L.N_PLUS <= e.op <= L.N_DIV:
            a = visit(e.children[0])
            b = visit(e.children[1])
            nodes.append(L.node(e.op, a=a, b=b))
        elif e.op == L.N_EACH_COL:
            nodes.append(L.node(e.op, a=visit(e.children[0]), nc=e.view))
        elif e.op == L.N_EACH_ROW:
            nodes.append(L.node(e.op, a=visit(e.children[0]), nr=e.view))
        elif e.op == L.N_DIAG:
            nodes.append(L.node(e.op, a=visit(e.children[0]), r0=e.view))
        else:
            a = visit(e.children[0])
            nodes.append(L.node(e.op, a=a, k=e.k))
        memo[key] = len(nodes) - 1
        return memo[key]

    visit(expr)
    if len(nodes) > L.MAX_NODES:
        raise ValueError("expression has %d nodes; at most %d" % (len(nodes), L.MAX_NODES))
    dtypes = {m.dtype for m in leaves if m is not None}
    if len(dtypes) > 1:
        raise TypeError("all matrices of an expression must share one dtype (got %s)" % sorted(dtypes))
    return L.make_tree(nodes), leaves, [m.cmat() if m is not None else None for m in leaves]


def _products(e, found, seen):
    """The matrix products of e that are not inside another product's operand."""
    if id(e) in seen:
        return
    seen.add(id(e))
    if e.op == MATMUL:
        found.append(e)
        return
    for c in e.children:
        if isinstance(c, Expr):
            _products(c, found, seen)


def _gemm_operand(e, stream):
    """(Mat, transposed) of a product operand.  An operand that is an
    expression rather than a matrix (or its transpose) is evaluated first
    into a temporary of the storage type, as Armadillo evaluates it into a
    temporary matrix; the fused element-wise kernel (or, for a product, the
    GEMM) computes it."""
    t = False
    while e.op == L.N_TRANS:
        e, t = e.children[0], not t
    if not isinstance(e, Mat):
        e = Mat(evaluate(e, stream=stream))
    return e, t


def _evaluate_gemm(expr, mm, out, stream, done=None):
    """expr with one matrix product mm: the GEMM kernel computes op(A) op(B)
    and evaluates the rest of expr on it before storing (Sec. 3: trans(X)*Y
    as one GEMM call with a transposed operand).  `done`: other products of
    expr, already evaluated into temporaries."""
    (A, ta), (B, tb) = _gemm_operand(mm.children[0], stream), _gemm_operand(mm.children[1], stream)
    nr, nc = expr.shape
    dev = A.tensor.device
    if out is None:
        out = _empty_colmajor(nr, nc, A.dtype, dev)
    if expr is mm:
        tree, extra = None, []
    else:
        tree, leaves, cm = lower(expr, product=mm, done=done)
        extra = cm[1:]
        if any(m.dtype != A.dtype for m in leaves[1:]):
            raise TypeError("all matrices of an expression must share one dtype")
    with torch.cuda.device(dev):
        L.coot_gemm_eval(context(dev), A.cmat(), ta, B.cmat(), tb, tree, extra, _out_cmat(out), _stream_ptr(stream))
    return out


def _empty_colmajor(n_rows, n_cols, dtype, device):
    return torch.empty((n_cols, n_rows), dtype=_TORCH[dtype], device=device).t()


class Reduction:
    """A reduction of an expression; evaluated by ``eval()`` (fused with the
    expression), or combined linearly first: ``accu(a) + k * accu(b)`` is
    evaluated as ``accu(a + k * b)`` in one pass."""

    def __init__(self, kind, expr, dim=-1, norm_type=0, n_seg=0):
        self.kind, self.expr, self.dim, self.norm_type = kind, expr, dim, norm_type
        self.n_seg = n_seg  # dim 1: equal column segments reduced separately (a Cube's slices)

    def _linear(self):
        return self.kind in (L.R_ACCU, L.R_SUM) and self.dim == -1

    def __add__(self, o):
        if isinstance(o, Reduction) and self._linear() and o._linear() and self.expr.shape == o.expr.shape:
            return Reduction(L.R_ACCU, self.expr + o.expr)
        return NotImplemented

    def __sub__(self, o):
        if isinstance(o, Reduction) and self._linear() and o._linear() and self.expr.shape == o.expr.shape:
            return Reduction(L.R_ACCU, self.expr - o.expr)
        return NotImplemented

    def __mul__(self, k):
        if isinstance(k, numbers.Real) and self._linear():
            return Reduction(L.R_ACCU, k * self.expr)
        return NotImplemented

    __rmul__ = __mul__

    def eval(self, out=None, fused=True, stream=None):
        _, r = evaluate(self.expr, reduction=self, fused=fused, stream=stream, materialise=out)
        return r

    def __float__(self):
        return float(self.eval().item())


def accu(x):
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_ACCU, -1, 0)
    return Reduction(L.R_ACCU, _as_expr(x))


def sum(x, dim=None):  # noqa: A001 -- Armadillo's name
    """Armadillo sum: along dim 0 (per column) for a matrix by default, all
    elements for a vector; dim=-1 sums everything."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_SUM, 0 if dim is None else dim, 0)
    x = _as_expr(x)
    if dim is None:
        dim = -1 if (x.n_rows == 1 or x.n_cols == 1) else 0
    return Reduction(L.R_SUM, x, dim)


def mean(x, dim=None):
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_MEAN, 0 if dim is None else dim, 0)
    x = _as_expr(x)
    if dim is None:
        dim = -1 if (x.n_rows == 1 or x.n_cols == 1) else 0
    return Reduction(L.R_MEAN, x, dim)


def dot(a, b):
    return Reduction(L.R_DOT, Expr(L.N_SCHUR, (_as_expr(a), _as_expr(b))))


def norm(x, p=2):
    x = _as_expr(x)
    if p == "fro":
        return Reduction(L.R_NORM_FRO, x)
    if p != 2:
        raise ValueError("norm: p = 2 (vectors) or 'fro'")
    if x.n_rows != 1 and x.n_cols != 1:
        raise ValueError("norm(X) of a matrix is the spectral norm, which this library does not compute; "
                         "use norm(X, 'fro')")
    return Reduction(L.R_NORM2, x)


def _along(x, dim):
    x = _as_expr(x)
    if dim is None:
        dim = -1 if (x.n_rows == 1 or x.n_cols == 1) else 0
    if dim not in (-1, 0, 1):
        raise ValueError("dim must be -1 (all elements), 0 (per column) or 1 (per row)")
    return x, dim


def var(x, norm_type=0, dim=-1):
    """Two-pass variance (norm_type 0: N-1, 1: N) over all elements (dim -1,
    the default), per column (dim 0) or per row (dim 1)."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_VAR, dim, norm_type)
    x, dim = _along(x, dim)
    return Reduction(L.R_VAR, x, dim, norm_type)


def stddev(x, norm_type=0, dim=-1):
    """Square root of ``var`` with the same arguments."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_STDDEV, dim, norm_type)
    x, dim = _along(x, dim)
    return Reduction(L.R_STDDEV, x, dim, norm_type)


def min(x, dim=None):  # noqa: A001 -- Armadillo's name
    """Smallest element (NaN skipped): per column for a matrix by default, all
    elements for a vector; dim -1 over everything, 0 per column, 1 per row."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_MIN, 0 if dim is None else dim, 0)
    x, dim = _along(x, dim)
    return Reduction(L.R_MIN, x, dim)


def max(x, dim=None):  # noqa: A001 -- Armadillo's name
    """Largest element, as ``min``."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_MAX, 0 if dim is None else dim, 0)
    x, dim = _along(x, dim)
    return Reduction(L.R_MAX, x, dim)


def index_min(x, dim=None):
    """Position (int64) of the first smallest element: the column-major linear
    index for dim -1, the row index per column (dim 0), the column index per
    row (dim 1); -1 where there is none.  Defaults as ``min``."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_INDEX_MIN, 0 if dim is None else dim, 0)
    x, dim = _along(x, dim)
    return Reduction(L.R_INDEX_MIN, x, dim)


def index_max(x, dim=None):
    """Position of the first largest element, as ``index_min``."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_INDEX_MAX, 0 if dim is None else dim, 0)
    x, dim = _along(x, dim)
    return Reduction(L.R_INDEX_MAX, x, dim)


def cumsum(x, dim=None):
    """Prefix sums with the expression's shape: down each column (dim 0, the
    default for a matrix), along each row (dim 1); along the vector for a
    vector.  ``cumsum(e).eval()`` returns the matrix."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_CUMSUM, 0 if dim is None else dim, 0)
    x = _as_expr(x)
    if dim is None:
        dim = 1 if x.n_rows == 1 else 0
    if dim not in (0, 1):
        raise ValueError("dim must be 0 (down each column) or 1 (along each row)")
    return Reduction(L.R_CUMSUM, x, dim)


def prod(x, dim=None):
    """Product of the elements, defaults as ``min``; no intermediate
    overflow or underflow, the result is rounded to the accumulation type."""
    if hasattr(x, "_cube_reduce"):
        return x._cube_reduce(L.R_PROD, 0 if dim is None else dim, 0)
    x, dim = _along(x, dim)
    return Reduction(L.R_PROD, x, dim)


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------
_ESIZE = {"f32": 4, "f64": 8, "bf16": 2, "f16": 2, "i32": 4}


def _view_of(e):
    """(data pointer, dtype, n_rows, n_cols, ld, rs) of a writable view: a
    Mat, a submatrix of one, or a diagonal of either."""
    if isinstance(e, Mat):
        return e.tensor.data_ptr(), e.dtype, e.n_rows, e.n_cols, e.ld, e.rs
    if e.op == L.N_SUBMAT:
        ptr, dt, _, _, ld, rs = _view_of(e.children[0])
        r0, c0, nr, nc = e.view
        return ptr + (r0 * rs + c0 * ld) * _ESIZE[dt], dt, nr, nc, ld, rs
    if e.op == L.N_DIAG:
        ptr, dt, _, _, ld, rs = _view_of(e.children[0])
        k = e.view
        kr, kc = (-k, 0) if k < 0 else (0, k)
        n = e.n_rows
        return ptr + (kr * rs + kc * ld) * _ESIZE[dt], dt, n, 1, builtins.max(n, 1), rs + ld
    raise TypeError("out must be a tensor, a Mat, a submatrix view or a diagonal view")


def _out_cmat(out):
    if isinstance(out, torch.Tensor):
        return Mat(out).cmat()
    ptr, dt, nr, nc, ld, rs = _view_of(out)
    return L.mat(ptr, L.DTYPE_CODE[dt], nr, nc, ld, rs if rs > 1 else 0)


def evaluate(expr, out=None, reduction=None, red_out=None, fused=True, stream=None, materialise=None):
    """Evaluate ``expr`` (delayed evaluation on assignment).

    * ``out``: a tensor (column-major, or rows rs apart) or a view -- a Mat,
      ``X.submat(...)``, ``X.diag(k)`` -- to receive Y (allocated when None
      and no reduction is requested, or when ``materialise`` is True);
    * ``reduction``: a Reduction (or None) fused onto the same pass; its
      result is returned as a tensor of the accumulation dtype (0-d for a
      scalar, column-major 1 x n_cols / n_rows x 1 for dim 0 / 1).
    Returns Y (a tensor) when there is no reduction, else (Y or None, result).
    """
    expr = _as_expr(expr)
    mms = []
    _products(expr, mms, set())
    if mms:
        return _evaluate_with_products(expr, mms, out, reduction, red_out, fused, stream, materialise)
    tree, leaves, cmats = lower(expr)
    dt = leaves[0].dtype
    dev = leaves[0].tensor.device
    nr, nc = expr.shape
    if reduction is not None and reduction.kind == L.R_CUMSUM:
        # the scan is written where Y would be: out (allocated when None)
        if isinstance(materialise, torch.Tensor):
            out = materialise
        if out is None:
            out = _empty_colmajor(nr, nc, dt, dev)
        red = L.reduce(reduction.kind, reduction.dim, reduction.norm_type, reduction.n_seg)
        with torch.cuda.device(dev):
            ctx = context(dev)
            fn = L.coot_eval if fused else L.coot_eval_unfused
            fn(ctx, tree, cmats, _out_cmat(out), red, None, _stream_ptr(stream))
        return None, out
    want_y = out is not None or reduction is None or materialise is True
    if isinstance(materialise, torch.Tensor):
        out = materialise
    if want_y and out is None:
        out = _empty_colmajor(nr, nc, dt, dev)
    out_m = _out_cmat(out) if out is not None else None
    red = L.reduce()
    rt = None
    if reduction is not None:
        red = L.reduce(reduction.kind, reduction.dim, reduction.norm_type, reduction.n_seg)
        if red_out is None:
            acc = torch.int64 if reduction.kind in (L.R_INDEX_MIN, L.R_INDEX_MAX) else _ACC[dt]
            if reduction.dim == 0:
                rt = torch.empty((1, nc), dtype=acc, device=dev)  # a row vector: contiguous either way
            elif reduction.dim == 1 and reduction.n_seg > 1:
                rt = torch.empty((reduction.n_seg, nr), dtype=acc, device=dev).t()  # segment s in column s
            elif reduction.dim == 1:
                rt = torch.empty((nr, 1), dtype=acc, device=dev)
            else:
                rt = torch.empty((), dtype=acc, device=dev)
        else:
            rt = red_out
    with torch.cuda.device(dev):
        ctx = context(dev)
        s = _stream_ptr(stream)
        fn = L.coot_eval if fused else L.coot_eval_unfused
        fn(ctx, tree, cmats, out_m, red, rt.data_ptr() if rt is not None else None, s)
    if reduction is None:
        return out
    return out, rt


def _evaluate_with_products(expr, mms, out, reduction, red_out, fused, stream, materialise):
    """An expression with matrix products.  The first product carries the
    rest of the expression as its fused epilogue; every other product is
    evaluated first into a temporary of the storage type (Armadillo's
    temporaries).  A reduction of such an expression runs over its evaluated
    result: the GEMM with its epilogue, then the fused reduction."""
    done = {id(mm): Mat(evaluate(mm, stream=stream)) for mm in mms[1:]}
    if reduction is None:
        return _evaluate_gemm(expr, mms[0], out if out is not None else
                              (materialise if isinstance(materialise, torch.Tensor) else None), stream, done)
    if reduction.expr is not expr:
        raise NotImplementedError("a reduction of a matrix product reduces the expression being evaluated")
    if reduction.kind == L.R_CUMSUM:
        y = Mat(_evaluate_gemm(expr, mms[0], None, stream, done))
        return evaluate(y, reduction=Reduction(L.R_CUMSUM, y, reduction.dim, 0, reduction.n_seg), out=out,
                        fused=fused, stream=stream, materialise=materialise)
    keep = out if out is not None else (materialise if isinstance(materialise, torch.Tensor) else None)
    yt = _evaluate_gemm(expr, mms[0], keep, stream, done)
    y = Mat(yt)
    _, r = evaluate(y, reduction=Reduction(reduction.kind, y, reduction.dim, reduction.norm_type, reduction.n_seg),
                    red_out=red_out, fused=fused, stream=stream)
    want_y = out is not None or materialise is True or isinstance(materialise, torch.Tensor)
    return (yt if want_y else None), r


def warmup(expr, reduction=None, out=None):
    """JIT-compile (and tune, when enabled) the kernel of an evaluation."""
    expr = _as_expr(expr)
    tree, leaves, cmats = lower(expr)
    red = L.reduce() if reduction is None else L.reduce(reduction.kind, reduction.dim, reduction.norm_type,
                                                        reduction.n_seg)
    dev = leaves[0].tensor.device
    if out is None and reduction is not None and reduction.kind == L.R_CUMSUM:
        out = _empty_colmajor(expr.n_rows, expr.n_cols, leaves[0].dtype, dev)  # a scan needs its output
    out_m = _out_cmat(out) if out is not None else None
    with torch.cuda.device(dev):
        L.coot_warmup(context(dev), tree, cmats, out_m, red)


def signature(expr, reduction=None, out=None) -> str:
    expr = _as_expr(expr)
    tree, leaves, cmats = lower(expr)
    red = L.reduce() if reduction is None else L.reduce(reduction.kind, reduction.dim, reduction.norm_type,
                                                        reduction.n_seg)
    out_m = _out_cmat(out) if out is not None else None
    return L.coot_signature(tree, cmats, out_m, red)


def last_launch(device=None) -> dict:
    return L.coot_last_launch(context(device))


def check_device_flag(device=None, stream=None) -> int:
    return L.coot_check_device_flag(context(device), _stream_ptr(stream))


__all__ = ["Mat", "Expr", "Reduction", "trans", "exp", "log", "abs", "square", "sqrt", "accu", "sum", "mean",
           "dot", "norm", "var", "evaluate", "warmup", "signature", "context", "last_launch", "check_device_flag",
           "lower"]
