"""Cubes (n_rows x n_cols x n_slices, Sec. 2) through the fused kernels, vs
the FP64 oracle applied slice by slice (or, along dim 2, to the cube's
elements-by-slices matrix): element-wise trees, full reductions, every
statistic along dims 0, 1 (one segment per slice) and 2, cumsum along every
dim, and each_slice as a batch."""
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import workloads

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (5, 3, 7), (130, 33, 9), (2, 400, 3), (1000, 1, 4)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rand_cube(r, c, s, dtype, seed, kind="normal"):
    g = workloads.generator(seed, "cuda")
    t = coot.cube_empty(r, c, s, {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16,
                                  "i32": torch.int32}[dtype])
    if dtype == "i32":
        t.copy_(torch.randint(-1000, 1000, (r, c, s), generator=g, device="cuda", dtype=torch.int32))
    elif kind == "near_one":
        t.copy_(torch.rand((r, c, s), generator=g, device="cuda", dtype=torch.float64) * 0.04 - 0.02)
    else:
        t.copy_(torch.randn((r, c, s), generator=g, device="cuda", dtype=torch.float64))
    return t


def host_slices(t):
    return [workloads.to_numpy_colmajor(t[:, :, q]) for q in range(t.shape[2])]


def elems_matrix(t):
    r, c, s = t.shape
    return workloads.to_numpy_colmajor(torch.as_strided(t, (r * c, s), (1, r * c)))


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_elementwise_cube_tree(dtype, shape):
    A, B = rand_cube(*shape, dtype, 1), rand_cube(*shape, dtype, 2)
    Q, R = coot.Cube(A), coot.Cube(B)
    Y = (Q % R + 2 * Q).eval()
    torch.cuda.synchronize()
    assert Y.shape == A.shape
    for q, (a, b) in enumerate(zip(host_slices(A), host_slices(B))):
        parity.compare_matrix(Y[:, :, q], oracle.evaluate("A B % #2 A * +", [a, b], dtype), dtype, "slice %d" % q)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("kind", ["sum", "mean", "min", "max", "index_min", "index_max", "prod", "var", "stddev"])
@pytest.mark.parametrize("dim", [0, 1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_cube_statistics_along_dims(dtype, kind, dim, shape):
    if dtype == "i32" and kind in ("mean", "var", "stddev"):
        pytest.skip("not defined for INT32")
    near = kind == "prod"
    A = rand_cube(*shape, dtype, 3, "near_one" if near else "normal")
    B = rand_cube(*shape, dtype, 4, "near_one" if near else "normal")
    Q, R = coot.Cube(A), coot.Cube(B)
    e = coot.exp(Q + R) if (near and dtype != "i32") else Q % R - Q
    tree = "A B + exp" if (near and dtype != "i32") else "A B % A -"
    fn = getattr(coot, kind)
    red = fn(e, dim=dim) if kind not in ("var", "stddev") else fn(e, 0, dim)
    v = red.eval()
    torch.cuda.synchronize()
    r, c, s = shape
    tok = {"sum": "sum", "mean": "mean", "min": "min", "max": "max", "index_min": "index_min",
           "index_max": "index_max", "prod": "prod", "var": "vardim", "stddev": "stddevdim"}[kind]

    def token(d):
        if kind in ("var", "stddev"):
            return "%s:%d:0" % (tok, d)
        return "%s:%d" % (tok, d)

    if dim in (0, 1):
        assert tuple(v.shape) == ((1, c, s) if dim == 0 else (r, 1, s))
        for q, (a, b) in enumerate(zip(host_slices(A), host_slices(B))):
            prog = tree + " " + token(dim)
            g = v[0, :, q] if dim == 0 else v[:, 0, q]
            g = g.reshape(1, -1) if dim == 0 else g.reshape(-1, 1)
            if kind.startswith("index"):
                parity.compare_index(g, prog, [a, b], dtype, "slice %d %s" % (q, prog))
            else:
                parity.compare_reduction(g, oracle.evaluate(prog, [a, b], dtype), dtype, "slice %d %s" % (q, prog))
    else:
        assert tuple(v.shape) == (r, c, 1)
        prog = tree + " " + token(1)
        g = v[:, :, 0].t().reshape(-1, 1)  # element (i, j) at row i + r j
        hs = [elems_matrix(A), elems_matrix(B)]
        if kind.startswith("index"):
            parity.compare_index(g, prog, hs, dtype, "dim 2 " + prog)
        else:
            parity.compare_reduction(g, oracle.evaluate(prog, hs, dtype), dtype, "dim 2 " + prog)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_cube_accu(dtype, shape):
    A = rand_cube(*shape, dtype, 5)
    v = coot.accu(coot.square(coot.Cube(A)) if dtype != "i32" else coot.Cube(A) % coot.Cube(A)).eval()
    torch.cuda.synchronize()
    r, c, s = shape
    cols = workloads.to_numpy_colmajor(torch.as_strided(A, (r, c * s), (1, max(r, 1))))
    parity.compare_reduction(v, oracle.evaluate("A A % accu", [cols], dtype), dtype, "accu")


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("dim", [0, 1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_cube_cumsum(dtype, dim, shape):
    A, B = rand_cube(*shape, dtype, 6), rand_cube(*shape, dtype, 7)
    Y = coot.cumsum(coot.Cube(A) - coot.Cube(B), dim).eval()
    torch.cuda.synchronize()
    assert Y.shape == A.shape
    if dim in (0, 1):
        for q, (a, b) in enumerate(zip(host_slices(A), host_slices(B))):
            parity.compare_matrix(Y[:, :, q], oracle.evaluate("A B - cumsum:%d" % dim, [a, b], dtype), dtype,
                                  "slice %d" % q)
    else:
        r, c, s = shape
        g = torch.as_strided(Y, (r * c, s), (1, r * c))
        parity.compare_matrix(g, oracle.evaluate("A B - cumsum:1", [elems_matrix(A), elems_matrix(B)], dtype), dtype,
                              "dim 2")


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
def test_each_slice_as_a_batch(dtype):
    A, B = rand_cube(40, 30, 25, dtype, 8), rand_cube(40, 30, 25, dtype, 9)
    Q, R = coot.Cube(A), coot.Cube(B)
    Y = coot.each_slice(lambda X, Z: X % Z + X, Q, R)
    v = coot.each_slice(lambda X, Z: coot.accu(X % Z), Q, R)
    torch.cuda.synchronize()
    assert Y.shape == A.shape and v.shape == (25,)
    for q, (a, b) in enumerate(zip(host_slices(A), host_slices(B))):
        parity.compare_matrix(Y[:, :, q], oracle.evaluate("A B % A +", [a, b], dtype), dtype, "slice %d" % q)
        parity.compare_reduction(v[q].reshape(1, 1), oracle.evaluate("A B % accu", [a, b], dtype), dtype,
                                 "accu slice %d" % q)


def test_segmented_row_reduction_through_the_c_abi():
    # n_seg column segments reduced separately, checked against per-segment sums
    from paper_2508_11385_gb300 import lib as L
    A = parity.rand(300, 60, "f32", seed=10)
    r = coot.evaluate(coot.Mat(A), reduction=coot.Reduction(L.R_SUM, coot.Mat(A), 1, 0, n_seg=4))[1]
    torch.cuda.synchronize()
    assert tuple(r.shape) == (300, 4)
    for q in range(4):
        hs = parity.host([A[:, 15 * q:15 * (q + 1)]])
        parity.compare_reduction(r[:, q].reshape(-1, 1), oracle.evaluate("A sum:1", hs, "f32"), "f32", "segment")
    with pytest.raises(L.CootError, match="SHAPE"):
        coot.evaluate(coot.Mat(A), reduction=coot.Reduction(L.R_SUM, coot.Mat(A), 1, 0, n_seg=7))
