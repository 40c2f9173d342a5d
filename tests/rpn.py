"""Test helpers for RPN tree programs (the oracle's program format).

* ``random_tree``     -- seeded random element-wise trees over leaves A..F;
* ``eval_exact``      -- exact rational evaluation (``fractions.Fraction``) of
                         the +, -, %, / and scalar forms, used to pin the oracle;
* ``eval_emulated``   -- evaluation with every node rounded to a target float
                         type (NumPy float32/float64 arithmetic, exp/log via the
                         correctly rounded double result), used to check that the
                         oracle's error bound covers a real rounded evaluation.

Nothing here is imported by the library or the oracle.
"""
from __future__ import annotations

import math
import random
from fractions import Fraction

import numpy as np

BIN = ["+", "-", "%", "/"]
SCAL = ["k*", "x+k", "x-k", "k-x", "x/k", "k/x"]
UN_ARITH = ["neg", "abs", "square"]
UN_TRANSC = ["exp", "log", "sqrt"]


def random_tree(rng: random.Random, n_leaves=3, depth=3, ops_bin=BIN, ops_scal=SCAL,
                ops_un=UN_ARITH, scalars=(0.5, 2.0, 3.0, -1.5, 0.25)):
    """Random RPN program (no reduction) of at most ``depth`` op levels."""
    def gen(d):
        if d == 0 or rng.random() < 0.2:
            return [chr(ord("A") + rng.randrange(n_leaves))]
        kind = rng.random()
        if kind < 0.5 and ops_bin:
            op = rng.choice(ops_bin)
            return gen(d - 1) + gen(d - 1) + [op]
        if kind < 0.75 and ops_scal:
            op = rng.choice(ops_scal)
            k = "#%r" % rng.choice(scalars)
            x = gen(d - 1)
            if op == "k*":
                return [k] + x + ["*"]
            if op == "x+k":
                return x + [k, "+"]
            if op == "x-k":
                return x + [k, "-"]
            if op == "k-x":
                return [k] + x + ["-"]
            if op == "x/k":
                return x + [k, "/"]
            return [k] + x + ["/"]
        if ops_un:
            return gen(d - 1) + [rng.choice(ops_un)]
        return gen(d - 1)

    return " ".join(gen(depth))


def _tokens(program):
    return program.split()


def eval_exact(program: str, leaves):
    """Exact evaluation over 2-D float arrays; returns a nested list of
    Fractions (None where a division by zero occurred).  Supports + - % /,
    the scalar forms, neg, abs, square, trans, submat and accu/sum/mean/dot."""
    st = []
    for tok in _tokens(program):
        if len(tok) == 1 and "A" <= tok <= "H":
            a = leaves[ord(tok) - ord("A")]
            st.append([[Fraction(float(a[i, j])) for j in range(a.shape[1])] for i in range(a.shape[0])])
        elif tok.startswith("#"):
            st.append(Fraction(float(tok[1:])))
        elif tok in ("+", "-", "%", "/", "*"):
            y = st.pop()
            x = st.pop()
            st.append(_exact_bin(tok, x, y))
        elif tok in ("neg", "abs", "square"):
            x = st.pop()
            f = {"neg": lambda v: -v, "abs": abs, "square": lambda v: v * v}[tok]
            st.append([[None if v is None else f(v) for v in row] for row in x])
        elif tok == "trans":
            x = st.pop()
            st.append([list(r) for r in zip(*x)])
        elif tok.startswith("submat:"):
            r0, c0, nr, nc = map(int, tok.split(":")[1:])
            x = st.pop()
            st.append([row[c0:c0 + nc] for row in x[r0:r0 + nr]])
        elif tok == "accu":
            x = st.pop()
            st.append(sum(v for row in x for v in row))
        elif tok in ("sum:0", "mean:0"):
            x = st.pop()
            s = [sum(x[i][j] for i in range(len(x))) for j in range(len(x[0]))]
            if tok == "mean:0":
                s = [v / len(x) for v in s]
            st.append([s])
        elif tok in ("sum:1", "mean:1"):
            x = st.pop()
            s = [sum(row) for row in x]
            if tok == "mean:1":
                s = [v / len(x[0]) for v in s]
            st.append([[v] for v in s])
        elif tok == "mean":
            x = st.pop()
            n = sum(len(r) for r in x)
            st.append(sum(v for row in x for v in row) / n)
        elif tok == "dot":
            y = st.pop()
            x = st.pop()
            st.append(sum(a * b for ra, rb in zip(x, y) for a, b in zip(ra, rb)))
        else:
            raise ValueError(tok)
    assert len(st) == 1
    return st[0]


def _exact_bin(op, x, y):
    xs = not isinstance(x, list)
    ys = not isinstance(y, list)
    m = y if xs else x

    def f(a, b):
        if a is None or b is None:
            return None
        if op == "+":
            return a + b
        if op == "-":
            return a - b
        if op in ("%", "*"):
            return a * b
        if b == 0:
            return None
        return a / b

    return [[f(x if xs else x[i][j], y if ys else y[i][j]) for j in range(len(m[0]))] for i in range(len(m))]


def eval_emulated(program: str, leaves, ftype=np.float32):
    """Evaluate with each node rounded to ``ftype`` (an emulated device).
    Scalars are converted to ``ftype`` first, as the device does."""
    st = []
    with np.errstate(all="ignore"):
        for tok in _tokens(program):
            if len(tok) == 1 and "A" <= tok <= "H":
                st.append(np.asarray(leaves[ord(tok) - ord("A")], dtype=ftype))
            elif tok.startswith("#"):
                st.append(ftype(float(tok[1:])))
            elif tok in ("+", "-", "%", "/", "*"):
                y = st.pop()
                x = st.pop()
                r = {"+": np.add, "-": np.subtract, "%": np.multiply, "*": np.multiply,
                     "/": np.divide}[tok](x, y)
                st.append(np.asarray(r, dtype=ftype))
            elif tok == "neg":
                st.append(-st.pop())
            elif tok == "abs":
                st.append(np.abs(st.pop()))
            elif tok == "square":
                x = st.pop()
                st.append(np.asarray(x * x, dtype=ftype))
            elif tok == "sqrt":
                st.append(np.sqrt(st.pop()).astype(ftype))
            elif tok in ("exp", "log"):
                x = st.pop()
                f = math.exp if tok == "exp" else math.log
                out = np.empty_like(x)
                for idx, v in np.ndenumerate(x):
                    try:
                        out[idx] = ftype(f(float(v)))
                    except (OverflowError, ValueError):
                        out[idx] = ftype(np.exp(np.float64(v)) if tok == "exp" else np.log(np.float64(v)))
                st.append(out)
            elif tok == "trans":
                st.append(np.ascontiguousarray(st.pop().T))
            elif tok.startswith("each_col:"):
                st.append(np.repeat(st.pop(), int(tok.split(":")[1]), axis=1))
            elif tok.startswith("each_row:"):
                st.append(np.repeat(st.pop(), int(tok.split(":")[1]), axis=0))
            elif tok == "diag" or tok.startswith("diag:"):
                k = int(tok.split(":")[1]) if ":" in tok else 0
                st.append(np.diag(st.pop(), k).reshape(-1, 1).copy())
            else:
                raise ValueError(tok)
    assert len(st) == 1
    return st[0]
