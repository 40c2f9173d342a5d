"""GPU-vs-oracle comparison helpers for the parity tests.

Tolerances (written here, used by every parity test):
  * INT32 trees: bit-exact (element-wise values and int64 reductions);
  * FP element-wise: |gpu - oracle| <= bound, the oracle's forward error bound
    (2 ulp of the compute type per + - * / node, 4 ulp per exp/log/sqrt node,
    propagated through the tree, plus the rounding to BF16/FP16 storage);
    non-finite oracle values must match exactly (NaN matches NaN);
  * FP reductions: |gpu - oracle| <= REL * |oracle| + bound, REL = 1e-6 for
    FP32 compute (FP32/BF16/FP16 storage) and 1e-13 for FP64; `bound` carries
    the element-wise errors of the tree being reduced (0 for a bare leaf).
"""
import numpy as np
import torch

import coot_rpn
import oracle
import rpn
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import workloads

REL = {"f32": 1e-6, "bf16": 1e-6, "f16": 1e-6, "f64": 1e-13, "i32": 0.0}


def host(tensors):
    return [workloads.to_numpy_colmajor(t) for t in tensors]


def split(program):
    toks = program.split()
    if toks and coot_rpn.is_reduction(toks[-1]):
        return " ".join(toks[:-1]), toks[-1]
    return program, None


def to_f64(t: torch.Tensor):
    t = t.detach()
    if t.dtype in (torch.bfloat16, torch.float16, torch.float32):
        t = t.to(torch.float64)
    return t.cpu().numpy()


def gpu_eval(program, tensors, fused=True, materialise=False):
    e, red = coot_rpn.build(program, tensors)
    if red is None:
        return coot.evaluate(e, fused=fused), None
    Y, r = coot.evaluate(e, reduction=red, fused=fused, materialise=True if materialise else None)
    return Y, r


def compare_matrix(gpu, res, dtype, what=""):
    g = to_f64(gpu)
    if dtype == "i32":
        assert g.shape == res.value.shape, (g.shape, res.value.shape)
        bad = np.argwhere(g.astype(np.int64) != res.value)
        assert bad.size == 0, "%s: INT32 mismatch at %s: gpu %s oracle %s" % (
            what, bad[:3].tolist(), g[tuple(bad[0])], res.value[tuple(bad[0])])
        return 0.0
    v, b = res.value, res.bound
    assert g.shape == v.shape, (g.shape, v.shape)
    fin = np.isfinite(v)
    if not np.all(fin):
        same = (g[~fin] == v[~fin]) | (np.isnan(g[~fin]) & np.isnan(v[~fin]))
        assert np.all(same), "%s: non-finite oracle values differ" % what
    with np.errstate(invalid="ignore"):
        err = np.abs(g - v)
    viol = fin & ~(err <= b)
    if np.any(viol):
        i = tuple(np.argwhere(viol)[0])
        raise AssertionError("%s: |gpu-oracle| %.3g > bound %.3g at %s (gpu %r oracle %r)" % (
            what, err[i], b[i], i, g[i], v[i]))
    return float(np.max(err[fin] / np.maximum(b[fin], 1e-300))) if np.any(fin) else 0.0


def compare_reduction(gpu, res, dtype, what="", rel=None):
    g = to_f64(gpu).reshape(res.value.shape)
    if dtype == "i32":
        assert np.array_equal(g.astype(np.int64), res.value), "%s: INT64 reduction mismatch %s vs %s" % (
            what, g.ravel()[:4], res.value.ravel()[:4])
        return 0.0
    rel = REL[dtype] if rel is None else rel
    v, b = res.value, res.bound
    fin = np.isfinite(v)
    if not np.all(fin):
        same = (g[~fin] == v[~fin]) | (np.isnan(g[~fin]) & np.isnan(v[~fin]))
        assert np.all(same), "%s: non-finite reduction differs: %s vs %s" % (what, g[~fin][:4], v[~fin][:4])
    tol = rel * np.abs(v) + b
    with np.errstate(invalid="ignore"):
        err = np.abs(g - v)
    viol = fin & ~(err <= tol)
    if np.any(viol):
        i = tuple(np.argwhere(viol)[0])
        raise AssertionError("%s: reduction |gpu-oracle| %.3g > tol %.3g (rel err %.3g) at %s: gpu %r oracle %r" % (
            what, err[i], tol[i], err[i] / max(abs(v[i]), 1e-300), i, g[i], v[i]))
    return float(np.max(err[fin] / np.maximum(np.abs(v[fin]), 1e-300))) if np.any(fin) else 0.0


def host_values(h, dtype):
    """Values of a host leaf as float64 (BF16/FP16 arrive as uint16 bits)."""
    if dtype == "bf16":
        return (h.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if dtype == "f16":
        return h.view(np.float16).astype(np.float64)
    return h.astype(np.float64)


def _groups(a, dim):
    """The reduction groups of a matrix: all elements in column-major order
    (dim -1), its columns (dim 0) or its rows (dim 1)."""
    if dim == -1:
        return [a.ravel(order="F")]
    if dim == 0:
        return [a[:, j] for j in range(a.shape[1])]
    return [a[i, :] for i in range(a.shape[0])]


def _first_extreme(vals, want_max):
    """First position of the smallest (largest) non-NaN value, -1 if none."""
    best = -1
    for q, x in enumerate(vals):
        if np.isnan(x):
            continue
        if best < 0 or (x > vals[best] if want_max else x < vals[best]):
            best = q
    return best


def compare_index(gpu, program, hs, dtype, what=""):
    """index_min / index_max: where several positions are correct within the
    oracle's error bounds, the GPU's must be one of them.

    The GPU decides in its compute precision.  A position k is a possible
    first minimum when some set of values inside the bounds makes it one:
    lo[k] < hi[j] for every earlier j and lo[k] <= hi[j] for every later j
    (lo, hi = value -/+ bound; for index_max the same on negated values).  With
    zero bounds (bare leaves, integer trees) that is the exact first position.
    Trees of + - * / sqrt only are also replayed with every node rounded to
    the compute type (rpn.eval_emulated, IEEE round-to-nearest as on the
    device), and then the position must be the replay's exactly."""
    tree, tok = split(program)
    head, _, rest = tok.partition(":")
    dim = int(rest) if rest else -1
    want_max = head == "index_max"
    ry = oracle.evaluate(tree, hs, dtype)
    ro = oracle.evaluate(program, hs, dtype)
    g = gpu.detach().cpu().numpy().astype(np.int64).reshape(ro.value.shape)
    ko = ro.value.astype(np.int64).ravel(order="F")
    kg = g.ravel(order="F")
    sign = -1.0 if want_max else 1.0
    vs = _groups(ry.value * sign, dim)
    bs = _groups(ry.bound, dim) if dtype != "i32" else _groups(np.zeros_like(ry.value, dtype=np.float64), dim)
    assert len(vs) == len(kg), (len(vs), kg.shape)
    for o, (v, b) in enumerate(zip(vs, bs)):
        k = int(kg[o])
        if ko[o] < 0:
            assert k == -1, "%s: output %d: oracle has no element, gpu index %d" % (what, o, k)
            continue
        assert 0 <= k < len(v) and not np.isnan(v[k]), "%s: output %d: gpu index %d invalid" % (what, o, k)
        lo = v - b
        hi = v + b
        ok = ~np.isnan(v)
        early = ok.copy()
        early[k:] = False
        late = ok.copy()
        late[:k + 1] = False
        assert np.all(lo[k] < hi[early]) and np.all(lo[k] <= hi[late]), (
            "%s: output %d: gpu index %d (value %r) cannot be the first extreme; oracle index %d (value %r)" % (
                what, o, k, sign * v[k], ko[o], sign * v[ko[o]]))
    toks = tree.split()
    if dtype != "i32" and not any(t in ("exp", "log") or t.startswith("submat") for t in toks):
        ftype = np.float64 if dtype == "f64" else np.float32
        y = rpn.eval_emulated(tree, [host_values(h, dtype).astype(ftype) for h in hs], ftype).astype(np.float64)
        for o, grp in enumerate(_groups(y, dim)):
            ke = _first_extreme(grp, want_max)
            assert int(kg[o]) == ke, "%s: output %d: gpu index %d, %s replay %d" % (
                what, o, int(kg[o]), ftype.__name__, ke)


def check(program, tensors, dtype, fused=True, materialise=False, out_dtype=None):
    """Evaluate `program` on the GPU and with the oracle; assert parity.
    Returns (Y, r) of the GPU."""
    Y, r = gpu_eval(program, tensors, fused=fused, materialise=materialise)
    torch.cuda.synchronize()
    hs = host(tensors)
    tree, red = split(program)
    if Y is not None:
        ry = oracle.evaluate(tree, hs, dtype, out_dtype)
        compare_matrix(Y, ry, dtype, program)
    if red is not None:
        if red.partition(":")[0] == "cumsum":
            compare_matrix(r, oracle.evaluate(program, hs, dtype, out_dtype), dtype, program)
        elif red.partition(":")[0] in ("index_min", "index_max"):
            compare_index(r, program, hs, dtype, program)
        else:
            rr = oracle.evaluate(program, hs, dtype)
            compare_reduction(r, rr, dtype, program)
    return Y, r


def strided(n_rows, n_cols, dtype, ld_extra=3, offset=0, device="cuda", seed=0, kind="normal"):
    """A column-major n_rows x n_cols view with ld = n_rows + ld_extra,
    starting `offset` elements into its buffer (offset 1 breaks 16-byte
    alignment)."""
    ld = n_rows + ld_extra + offset
    g = workloads.generator(seed, device)
    if dtype == "i32":
        base = workloads.int_uniform(ld, n_cols, -1000, 1000, g, device)
    else:
        base = workloads.normal(ld, n_cols, dtype, g, device)
    return base[offset:offset + n_rows, :]


def rand(n_rows, n_cols, dtype, seed=0, device="cuda", kind="normal", lo=-1.0, hi=1.0):
    g = workloads.generator(seed, device)
    if dtype == "i32":
        return workloads.int_uniform(n_rows, n_cols, -1000, 1000, g, device)
    if kind == "uniform":
        return workloads.uniform(n_rows, n_cols, lo, hi, dtype, g, device)
    if kind == "positive":
        return workloads.uniform(n_rows, n_cols, 0.25, 2.0, dtype, g, device)
    return workloads.normal(n_rows, n_cols, dtype, g, device)
