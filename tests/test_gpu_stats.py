"""Armadillo statistics fused onto a tree (min, max, index_min, index_max,
prod, stddev, var along a dimension) vs the FP64 oracle, on small and ragged
shapes that span several blocks and tiles, every kernel family (flat, per
column, per row, transposed tiles), every dtype; plus ties, NaN, empty
inputs, integer wrap-around and products whose partial products leave the
floating-point range."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 1), (1000, 1), (129, 65), (4097, 3), (2, 3000)]
EXTREMES = ["min", "max", "min:0", "max:1", "index_min", "index_max", "index_min:0", "index_max:0",
            "index_min:1", "index_max:1"]
SPREAD = ["stddev", "stddev:1", "vardim:0:0", "vardim:1:1", "stddevdim:0:1", "stddevdim:1:0"]
PRODS = ["prod", "prod:0", "prod:1"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _near_one(m, n, dtype, seed):
    """exp of small uniform values: products of thousands stay in range"""
    if dtype == "i32":
        return parity.rand(m, n, dtype, seed=seed)
    return parity.rand(m, n, dtype, seed=seed, kind="uniform", lo=-0.02, hi=0.02)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16", "i32"])
@pytest.mark.parametrize("red", EXTREMES)
@pytest.mark.parametrize("shape", SHAPES)
def test_extremes_over_trees(dtype, red, shape):
    m, n = shape
    A, B, C = (parity.rand(m, n, dtype, seed=s) for s in (1, 2, 3))
    parity.check("A B % C + " + red, [A, B, C], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("red", SPREAD)
@pytest.mark.parametrize("shape", SHAPES)
def test_var_and_stddev_over_trees(dtype, red, shape):
    m, n = shape
    A, B = (parity.rand(m, n, dtype, seed=s) for s in (4, 5))
    parity.check("A #3 + B exp % " + red, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("red", PRODS)
@pytest.mark.parametrize("shape", SHAPES)
def test_prod_over_trees(dtype, red, shape):
    m, n = shape
    A = _near_one(m, n, dtype, 6)
    B = _near_one(m, n, dtype, 7)
    prog = ("A B % " if dtype == "i32" else "A B + exp ") + red
    parity.check(prog, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", ["index_min", "max:0", "index_max:0", "min:1", "index_min:1", "prod:0", "prod:1",
                                 "vardim:0:0", "stddevdim:1:1", "stddev"])
def test_stats_with_transposed_reads(dtype, red):
    if dtype == "i32" and ("var" in red or "stddev" in red):
        pytest.skip("var/stddev are not defined for INT32 trees")
    m, n = 77, 130
    if red.startswith("prod"):
        A = _near_one(n, m, dtype, 1)
        B = _near_one(m, n, dtype, 2)
        prog = ("A trans B % " if dtype == "i32" else "A trans B + exp ") + red
    else:
        A = parity.rand(n, m, dtype, seed=1)
        B = parity.rand(m, n, dtype, seed=2)
        prog = "A trans B % B + " + red
    parity.check(prog, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", ["index_max", "min:0", "index_min:1", "prod:0", "vardim:1:0"])
@pytest.mark.parametrize("offset", [0, 1])
def test_stats_on_strided_and_unaligned_views(dtype, red, offset):
    if dtype == "i32" and "var" in red:
        pytest.skip("var is not defined for INT32 trees")
    A = parity.strided(301, 37, dtype, ld_extra=5, offset=offset, seed=3)
    B = parity.strided(301, 37, dtype, ld_extra=2, offset=offset, seed=4)
    if red.startswith("prod") and dtype != "i32":
        parity.check("A #0.01 * exp B #0.01 * exp % " + red, [A, B], dtype)
    else:
        parity.check("A B - " + red, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_stats_with_materialised_output(dtype):
    A, B = (parity.rand(200, 150, dtype, seed=s) for s in (8, 9))
    for red in ["index_min:0", "max:1", "stddevdim:0:0", "vardim:1:1"]:
        parity.check("A B % A + " + red, [A, B], dtype, materialise=True)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
def test_ties_keep_the_first_position(dtype):
    # every column holds its minimum and maximum three times
    g = np.random.default_rng(11)
    m, n = 531, 47
    a = g.integers(-50, 50, size=(m, n)).astype(np.float64)
    for j in range(n):
        rows = g.choice(m, size=6, replace=False)
        a[rows[:3], j] = -77.0
        a[rows[3:], j] = 91.0
    t = torch.tensor(a, dtype={"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16,
                               "i32": torch.int32}[dtype]).t().contiguous().t().cuda()
    for red in ["index_min", "index_max", "index_min:0", "index_max:0", "index_min:1", "index_max:1", "min:0",
                "max:1"]:
        parity.check("A " + red, [t], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_nan_elements_are_skipped(dtype):
    g = np.random.default_rng(12)
    m, n = 260, 33
    a = g.normal(size=(m, n))
    a[g.random(size=(m, n)) < 0.3] = np.nan
    a[:, 5] = np.nan        # a column with no number
    a[17, :] = np.nan       # a row with no number
    t = torch.tensor(a, dtype=torch.float32 if dtype == "f32" else torch.float64).t().contiguous().t().cuda()
    for red in ["min", "max", "index_min", "index_max", "min:0", "index_max:0", "max:1", "index_min:1"]:
        parity.check("A #2 * " + red, [t], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("shape", [(0, 0), (0, 5), (5, 0)])
def test_empty_statistics(dtype, shape):
    m, n = shape
    tdt = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32}[dtype]
    A = torch.zeros((n, m), dtype=tdt, device="cuda").t()
    reds = ["min", "max", "index_min", "index_max", "prod", "min:0", "index_max:0", "prod:0", "max:1",
            "index_min:1", "prod:1"]
    if dtype != "i32":
        reds += ["stddev", "vardim:0:0", "stddevdim:1:1"]
    for red in reds:
        parity.check("A " + red, [A], dtype)
    # the transposed form takes the same empty paths
    At = torch.zeros((m, n), dtype=tdt, device="cuda").t()
    for red in ["prod:0", "prod:1", "index_max:0", "min:1"]:
        parity.check("A trans " + red, [At], dtype)


def test_int_prod_wraps_modulo_2_64():
    a = torch.tensor([[2 ** 31 - 1], [2 ** 31 - 1], [7], [-3], [65537]], dtype=torch.int32).cuda()
    parity.check("A prod", [a], "i32")
    big = parity.rand(3000, 40, "i32", seed=13)
    parity.check("A #1 + prod:0", [big], "i32")
    parity.check("A #1 + prod:1", [big], "i32")


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_prod_partials_leave_the_range(dtype):
    # alternating 2^(+-e) factors: running products in a plain accumulator
    # overflow or underflow, the exact product is small
    big = 100 if dtype == "f32" else 900
    m = 4098  # as many +big as -big factors, also after the 2^(1/16) ones below
    e = np.where(np.arange(m) % 2 == 0, big, -big).astype(np.float64)
    e[::7] = 0.0625
    a = (2.0 ** e) * np.where(np.arange(m) % 3 == 0, -1.0, 1.0)
    t = torch.tensor(a.reshape(-1, 1), dtype=torch.float32 if dtype == "f32" else torch.float64).cuda()
    parity.check("A prod", [t], dtype)
    parity.check("A #1 * prod:0", [t], dtype)
    # subnormal factors
    tiny = np.full((30, 1), 2.0 ** (-140 if dtype == "f32" else -1060))
    huge = np.full((40, 1), 2.0 ** (105 if dtype == "f32" else 795))  # product exactly 1
    t2 = torch.tensor(np.vstack([tiny, huge]), dtype=t.dtype).cuda()
    parity.check("A prod", [t2], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", ["min", "index_max:0", "prod:1", "stddev", "vardim:0:1"])
def test_unfused_matches_fused(dtype, red):
    if dtype == "i32" and ("var" in red or "stddev" in red):
        pytest.skip("var/stddev are not defined for INT32 trees")
    A = _near_one(120, 90, dtype, 14) if red.startswith("prod") else parity.rand(120, 90, dtype, seed=14)
    B = _near_one(120, 90, dtype, 15) if red.startswith("prod") else parity.rand(120, 90, dtype, seed=15)
    prog = ("A B + exp " if (red.startswith("prod") and dtype != "i32") else "A B % ") + red
    _, rf = parity.gpu_eval(prog, [A, B], fused=True)
    _, ru = parity.gpu_eval(prog, [A, B], fused=False)
    torch.cuda.synchronize()
    hs = parity.host([A, B])
    if red.startswith("index"):
        parity.compare_index(rf, prog, hs, dtype, "fused " + prog)
        parity.compare_index(ru, prog, hs, dtype, "unfused " + prog)
    else:
        rr = oracle.evaluate(prog, hs, dtype)
        parity.compare_reduction(rf, rr, dtype, "fused " + prog)
        parity.compare_reduction(ru, rr, dtype, "unfused " + prog)


def test_python_defaults_follow_armadillo():
    A = coot.Mat(parity.rand(40, 30, "f32", seed=16))
    v = coot.Mat(parity.rand(40, 1, "f32", seed=17))
    assert coot.min(A).eval().shape == (1, 30)          # matrix: per column
    assert coot.index_max(A).eval().dtype == torch.int64
    assert coot.max(v).eval().shape == ()               # vector: all elements
    assert coot.prod(A, 1).eval().shape == (40, 1)
    assert coot.stddev(A).eval().shape == ()            # var/stddev: all elements unless dim given
    assert coot.var(A, 1, 0).eval().shape == (1, 30)


# reductions along dim 1 of trees with transposed reads: the row walk, each
# transposed slot read along the thread's run of columns (16-byte vectors when
# the runs are aligned: leading dimension 300; element by element: 301);
# every run length forced in turn, ragged segments and rows
ROW_TR = ["sum:1", "mean:1", "max:1", "index_min:1", "prod:1", "vardim:1:1", "stddevdim:1:0"]


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("red", ROW_TR)
@pytest.mark.parametrize("shape", [(1003, 300), (1003, 301), (600, 4100), (70, 9001)])
def test_row_walk_with_transposed_reads(dtype, red, shape, monkeypatch):
    # (600, 4100) and (70, 9001): many column segments per row block, whose
    # starts must fall on whole vectors of the transposed reads
    if dtype == "i32" and ("var" in red or "stddev" in red or "mean" in red):
        pytest.skip("not defined for INT32 trees")
    m, n = shape
    if red.startswith("prod"):
        A = _near_one(n, m, dtype, 11)
        B = _near_one(m, n, dtype, 12)
        prog = ("A trans B % " if dtype == "i32" else "A trans B + exp ") + red
    else:
        A = parity.rand(n, m, dtype, seed=11)
        B = parity.rand(m, n, dtype, seed=12)
        prog = "A trans B % B + " + red
    two = "var" in red or "stddev" in red
    for u in (16, 8, 4):
        kname = "coot_row%s_v1u%d" % ("_p1" if two else "", u)
        monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
        parity.check(prog, [A, B], dtype)
        assert coot.last_launch()["kernel"] == kname, coot.last_launch()


def test_transposed_majority_stays_on_tiles():
    # more transposed reads than direct streams: the tile kernels
    A = parity.rand(300, 1003, "f32", seed=13)
    B = parity.rand(300, 1003, "f32", seed=14)
    parity.check("A trans B trans - sum:1", [A, B], "f32")
    assert coot.last_launch()["kernel"].startswith("coot_tile")
