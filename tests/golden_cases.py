"""Reader for the worked cases under ``tests/golden/`` (format: the header of
``tests/golden/fig1_example_program.txt``) and the comparison they state.

Every expected value in those files comes from a closed form or from the
definition of an operation, written by hand; none was produced by the oracle
or by the GPU library.  ``test_golden.py`` holds the oracle to them on the CPU
and ``test_gpu_golden.py`` the CUDA path on the GPU."""
from __future__ import annotations

import glob
import math
import os
from dataclasses import dataclass, field

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# reduction bound of the compute type (FP32 for FP32/BF16/FP16 storage)
REL = {"f32": 1e-6, "bf16": 1e-6, "f16": 1e-6, "f64": 1e-13, "i32": 0.0}
# spacing at 1.0 of the compute type and of the storage type
_EPS_COMPUTE = {"f32": 2.0 ** -23, "bf16": 2.0 ** -23, "f16": 2.0 ** -23, "f64": 2.0 ** -52}
_EPS_STORAGE = {"bf16": 2.0 ** -7, "f16": 2.0 ** -10}


@dataclass
class Leaf:
    name: str
    n_rows: int
    n_cols: int
    values: list


@dataclass
class Case:
    name: str
    source: str
    cite: str = ""
    dtypes: list = field(default_factory=list)
    leaves: list = field(default_factory=list)
    prog: str = ""
    expect: tuple = None  # (n_rows, n_cols, values)
    tol: tuple = ("exact",)
    after: Leaf = None

    def leaf_index(self, name):
        return ord(name) - ord("A")


def _number(tok):
    t = tok.lower()
    if t in ("inf", "+inf"):
        return math.inf
    if t == "-inf":
        return -math.inf
    if t == "nan":
        return math.nan
    try:
        return int(tok)
    except ValueError:
        return float(tok)


def _values(spec, count):
    toks = spec.split()
    if toks and toks[0] == "fill":
        return [_number(toks[1])] * count
    if toks and toks[0] == "seq":
        a, d = _number(toks[1]), _number(toks[2])
        return [a + k * d for k in range(count)]
    vals = [_number(t) for t in toks]
    if len(vals) != count:
        raise ValueError("expected %d values, got %d" % (count, len(vals)))
    return vals


def _shaped(rest):
    head, _, spec = rest.partition(":")
    parts = head.split()
    n_rows, n_cols = int(parts[-2]), int(parts[-1])
    return parts[:-2], n_rows, n_cols, _values(spec, n_rows * n_cols)


def load_file(path):
    cases, cur = [], None
    src = os.path.basename(path)
    with open(path) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "case":
                cur = Case(name=rest.strip(), source=src)
            elif key == "end":
                cases.append(cur)
                cur = None
            elif key == "cite":
                cur.cite = rest.strip()
            elif key == "dtype":
                cur.dtypes = rest.split()
            elif key == "leaf":
                names, r, c, vals = _shaped(rest)
                cur.leaves.append(Leaf(names[0], r, c, vals))
            elif key == "prog":
                cur.prog = rest.strip()
            elif key == "expect":
                _, r, c, vals = _shaped(rest)
                cur.expect = (r, c, vals)
            elif key == "tol":
                t = rest.split()
                cur.tol = (t[0], int(t[1])) if t[0] == "ulp" else (t[0],)
            elif key == "after":
                names, r, c, vals = _shaped(rest)
                cur.after = Leaf(names[0], r, c, vals)
            else:
                raise ValueError("%s: unknown key %r" % (src, key))
    return cases


def load_all():
    out = []
    for path in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt"))):
        out.extend(load_file(path))
    return out


def params():
    """(case, dtype) pairs with readable ids, for pytest.mark.parametrize."""
    import pytest

    return [pytest.param(c, d, id="%s-%s" % (c.name, d)) for c in load_all() for d in c.dtypes]


def host_leaf(leaf: Leaf, dtype: str) -> np.ndarray:
    """The leaf as a column-major host array in the oracle's representation
    (BF16/FP16 as uint16 bit patterns).  Raises if a value is not exactly
    representable in the storage type: the fixtures hold exact inputs only."""
    v = np.array(leaf.values, dtype=np.float64).reshape((leaf.n_rows, leaf.n_cols), order="F")
    if dtype == "i32":
        iv = np.array(leaf.values, dtype=np.int64).reshape((leaf.n_rows, leaf.n_cols), order="F")
        assert np.all((iv >= -2 ** 31) & (iv < 2 ** 31)), leaf.name
        return np.asfortranarray(iv.astype(np.int32))
    if dtype == "f64":
        return np.asfortranarray(v)
    if dtype == "f32":
        a = v.astype(np.float32)
        back = a.astype(np.float64)
    elif dtype == "f16":
        a = v.astype(np.float16)
        back = a.astype(np.float64)
        a = a.view(np.uint16)
    else:  # bf16: the top half of an FP32 value whose low half is zero
        f = v.astype(np.float32)
        bits = f.view(np.uint32)
        assert np.all((bits & 0xFFFF) == 0), "%s: not exact in bf16" % leaf.name
        a = (bits >> 16).astype(np.uint16)
        back = f.astype(np.float64)
    same = (back == v) | (np.isnan(back) & np.isnan(v))
    assert np.all(same), "%s: not exact in %s" % (leaf.name, dtype)
    return np.asfortranarray(a)


def check(got, case: Case, dtype: str, what=""):
    """Compare ``got`` (float64 or int64 array, any shape holding the result
    in column-major order) with the case's expected values and tolerance."""
    r, c, vals = case.expect
    g = np.asarray(got)
    g = g.reshape(-1, order="F") if g.ndim == 2 else g.reshape(-1)
    assert g.size == r * c, "%s: %d values, expected %d x %d" % (what, g.size, r, c)
    kind = case.tol[0]
    for k, e in enumerate(vals):
        x = g[k]
        if dtype == "i32" and isinstance(e, int) and np.issubdtype(g.dtype, np.integer):
            assert int(x) == e, "%s[%d]: %d != %d" % (what, k, int(x), e)
            continue
        x = float(x)
        e = float(e)
        if math.isnan(e) or math.isinf(e):
            ok = (math.isnan(e) and math.isnan(x)) or x == e
            assert ok, "%s[%d]: %r, expected %r" % (what, k, x, e)
            continue
        if kind == "exact":
            tol = 0.0
        elif kind == "rel":
            tol = REL[dtype] * abs(e)
        else:  # ulp N of the compute type, plus half a unit of BF16/FP16 storage
            scale = 2.0 ** math.floor(math.log2(abs(e))) if e != 0 else 0.0
            tol = case.tol[1] * _EPS_COMPUTE[dtype] * scale + 0.5 * _EPS_STORAGE.get(dtype, 0.0) * scale
        assert abs(x - e) <= tol, "%s[%d]: %r, expected %r (tol %.3g)" % (what, k, x, e, tol)


def check_after(got, leaf: Leaf, what=""):
    g = np.asarray(got, dtype=np.float64).reshape(-1, order="F")
    want = np.array(leaf.values, dtype=np.float64)
    assert np.array_equal(g, want), "%s: %s, expected %s" % (what, g.tolist(), want.tolist())
