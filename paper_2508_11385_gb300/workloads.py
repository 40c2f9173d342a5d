"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws random matrices
(column-major, as the library and the oracle both read them) so that the GPU
path and the CPU oracle are fed the very same stored values.

Recipe (every draw is FP64 from a ``torch.Generator`` seeded per workload,
leaves drawn in order A, B, C, ..., then rounded to nearest-even into the
storage dtype):

* ``plain_small``   -- seed 0: A, B, C FP32 1024x1024, uniform[-1, 1].
* ``large_trees``   -- seed 1: A..F n x n, normal(0, 1) for FP32/FP64;
                       INT32 uniform integers in [-1000, 1000].
* ``precision``     -- seed 3: vectors of 2^28 elements,
                       x = s * exp(2 z), z ~ normal(0, 1), s = +-1
                       equiprobable (lognormal(0, 2) with random signs);
                       y an independent draw for dot.  Values that are not
                       finite after rounding (FP16 overflow) are redrawn.
* ``batching``      -- seed 4: rows and cols each floor(exp(U(ln 4, ln 513)))
                       (log-uniform in [4, 512]); A, B r x c and C c x r,
                       normal(0, 1) FP32.
* ``graph_chain``   -- seed 5: A, B, C FP32 2048x2048 normal(0, 1).
* ``differentiation`` -- seed 6: W, X normal(0, 1), Y uniform[-1, 1], FP32.

The paper's own benchmarks (Sec. 5) fill vectors and matrices from a uniform
random generator and time sum / axpy over N = 1e5 .. 1e8 elements; these
recipes keep that structure at GB300 sizes.
"""
from __future__ import annotations

import math

import torch

TORCH_DTYPE = {
    "f32": torch.float32,
    "f64": torch.float64,
    "bf16": torch.bfloat16,
    "f16": torch.float16,
    "i32": torch.int32,
}

SEEDS = {"plain_small": 0, "large_trees": 1, "precision": 3, "batching": 4,
         "graph_chain": 5, "differentiation": 6}


def generator(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def colmajor_empty(n_rows: int, n_cols: int, dtype: str, device="cpu") -> torch.Tensor:
    """An uninitialised n_rows x n_cols column-major tensor (strides (1, n_rows))."""
    return torch.empty((n_cols, n_rows), dtype=TORCH_DTYPE[dtype], device=device).t()


def _as_colmajor(t_cols_rows: torch.Tensor) -> torch.Tensor:
    # a (n_cols, n_rows) row-major buffer read as its transpose is column-major
    return t_cols_rows.t()


def uniform(n_rows, n_cols, lo, hi, dtype, gen, device="cpu"):
    x = torch.rand((n_cols, n_rows), generator=gen, dtype=torch.float64, device=device)
    x = x.mul_(hi - lo).add_(lo)
    return _as_colmajor(x.to(TORCH_DTYPE[dtype]))


def normal(n_rows, n_cols, dtype, gen, device="cpu", std=1.0):
    x = torch.randn((n_cols, n_rows), generator=gen, dtype=torch.float64, device=device)
    if std != 1.0:
        x.mul_(std)
    return _as_colmajor(x.to(TORCH_DTYPE[dtype]))


def int_uniform(n_rows, n_cols, lo, hi, gen, device="cpu"):
    x = torch.randint(lo, hi + 1, (n_cols, n_rows), generator=gen, dtype=torch.int64, device=device)
    return _as_colmajor(x.to(torch.int32))


def signed_lognormal(n, dtype, gen, device="cpu", sigma=2.0):
    """n-element column vector: s * exp(sigma * z); non-finite values after
    rounding to ``dtype`` are redrawn (FP16 overflow above 65504)."""
    def draw(m):
        z = torch.randn(m, generator=gen, dtype=torch.float64, device=device)
        s = torch.randint(0, 2, (m,), generator=gen, device=device, dtype=torch.int8)
        x = torch.exp(z.mul_(sigma))
        x = torch.where(s == 0, -x, x)
        return x.to(TORCH_DTYPE[dtype])

    x = draw(n)
    for _ in range(64):
        bad = ~torch.isfinite(x.to(torch.float32)) if dtype in ("bf16", "f16") else ~torch.isfinite(x)
        nb = int(bad.sum())
        if nb == 0:
            break
        x[bad] = draw(nb)
    return x.reshape(n, 1)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def plain_small(n=1024, device="cpu"):
    g = generator(SEEDS["plain_small"], device)
    return [uniform(n, n, -1.0, 1.0, "f32", g, device) for _ in range(3)]


def large_trees(dtype="f32", n=8192, n_leaves=6, device="cpu", m=None):
    """A..F of n x m (m defaults to n)."""
    m = n if m is None else m
    g = generator(SEEDS["large_trees"], device)
    if dtype == "i32":
        return [int_uniform(n, m, -1000, 1000, g, device) for _ in range(n_leaves)]
    return [normal(n, m, dtype, g, device) for _ in range(n_leaves)]


def precision(dtype="f32", n=1 << 28, device="cpu"):
    """x, y: two n x 1 signed-lognormal vectors."""
    g = generator(SEEDS["precision"], device)
    return signed_lognormal(n, dtype, g, device), signed_lognormal(n, dtype, g, device)


def batching_shapes(n_problems=50000, lo=4, hi=512, seed=None):
    """(rows, cols) int64 tensors, each floor(exp(U(ln lo, ln(hi+1)))) clipped to [lo, hi]."""
    g = generator(SEEDS["batching"] if seed is None else seed)
    u = torch.rand((2, n_problems), generator=g, dtype=torch.float64)
    v = torch.floor(torch.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).clamp_(lo, hi)
    return v[0].to(torch.int64), v[1].to(torch.int64)


def batching(n_problems=50000, device="cpu", lo=4, hi=512):
    """Returns (rows, cols, A_list, B_list, C_list), each problem's A, B r x c
    and C c x r, carved out of three contiguous pools (column-major)."""
    rows, cols = batching_shapes(n_problems, lo, hi)
    g = generator(SEEDS["batching"] + 1000, device)
    sizes = (rows * cols).tolist()
    total = int(sum(sizes))
    pools = [torch.randn(total, generator=g, dtype=torch.float64, device=device).to(torch.float32)
             for _ in range(3)]
    A, B, C = [], [], []
    off = 0
    for r, c, s in zip(rows.tolist(), cols.tolist(), sizes):
        A.append(pools[0][off:off + s].view(c, r).t())
        B.append(pools[1][off:off + s].view(c, r).t())
        C.append(pools[2][off:off + s].view(r, c).t())
        off += s
    return rows, cols, A, B, C, pools


def graph_chain(n=2048, device="cpu"):
    g = generator(SEEDS["graph_chain"], device)
    return [normal(n, n, "f32", g, device) for _ in range(3)]


def differentiation(n=4096, device="cpu"):
    g = generator(SEEDS["differentiation"], device)
    W = normal(n, n, "f32", g, device)
    X = normal(n, n, "f32", g, device)
    Y = uniform(n, n, -1.0, 1.0, "f32", g, device)
    return W, X, Y


def to_numpy_colmajor(t: torch.Tensor):
    """Host NumPy array with the same column-major layout (BF16/FP16 as uint16
    bit patterns)."""
    t = t.detach().cpu()
    if t.dtype in (torch.bfloat16, torch.float16):
        t = t.view(torch.int16)
        return t.numpy().view("uint16")
    return t.numpy()
