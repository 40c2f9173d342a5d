"""Fused GPU evaluation vs the FP64 oracle, element by element, on small and
ragged sizes that span several blocks/tiles: every op, every leaf layout
(contiguous, strided, unaligned view, transposed), every reduction, every
dtype; plus fused-vs-unfused bitwise equality and the edge cases."""
import random

import numpy as np
import pytest
import torch

import parity
import rpn
import paper_2508_11385_gb300 as coot

pytestmark = pytest.mark.gpu

SHAPES_2 = ["#2 A * B +", "A B % C +", "A trans B +", "A B - exp #1 C abs + /", "A B - square sum:0",
            "A submat:3:5:40:33 accu"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("prog", SHAPES_2)
@pytest.mark.parametrize("shape", [(67, 45), (128, 128), (1023, 3), (5, 4097)])
def test_config2_shapes_small(dtype, prog, shape):
    if dtype == "i32" and "exp" in prog:
        pytest.skip("exp is not defined for INT32 trees")
    m, n = shape
    if "trans" in prog:
        A = parity.rand(n, m, dtype, seed=1)
    else:
        A = parity.rand(m, n, dtype, seed=1)
    if "submat" in prog and (m < 43 or n < 38):
        prog = "A submat:1:2:%d:%d accu" % (m - 1, n - 2)
    B = parity.rand(m, n, dtype, seed=2)
    C = parity.rand(m, n, dtype, seed=3)
    parity.check(prog, [A, B, C], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("prog", SHAPES_2)
def test_fused_equals_unfused_bitwise(dtype, prog):
    if dtype == "i32" and "exp" in prog:
        pytest.skip("exp is not defined for INT32 trees")
    m, n = 300, 77
    A = parity.rand(n, m, dtype, seed=1) if "trans" in prog else parity.rand(m, n, dtype, seed=1)
    B = parity.rand(m, n, dtype, seed=2)
    C = parity.rand(m, n, dtype, seed=3)
    tree, red = parity.split(prog)
    Yf, rf = parity.gpu_eval(prog, [A, B, C], fused=True, materialise=True)
    Yu, ru = parity.gpu_eval(prog, [A, B, C], fused=False, materialise=True)
    torch.cuda.synchronize()
    if Yf is not None and red is None:
        assert torch.equal(Yf.view(-1) if Yf.is_contiguous() else Yf.contiguous().view(-1),
                           Yu.view(-1) if Yu.is_contiguous() else Yu.contiguous().view(-1))
    if red is not None:
        hs = parity.host([A, B, C])
        import oracle
        rr = oracle.evaluate(prog, hs, dtype)
        parity.compare_reduction(ru, rr, dtype, "unfused " + prog)
        parity.compare_reduction(rf, rr, dtype, "fused " + prog)


def test_plain_small_config():
    from paper_2508_11385_gb300 import workloads
    A, B, C = workloads.plain_small(device="cuda")
    parity.check("#0.5 A * B C exp % +", [A, B, C], "f32")
    parity.check("#0.5 A * B C exp % + square accu", [A, B, C], "f32", materialise=True)


@pytest.mark.parametrize("seed", range(24))
@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16"])
def test_random_trees(seed, dtype):
    rng = random.Random(seed)
    m, n = rng.choice([(1, 1), (17, 9), (129, 65), (1000, 7), (33, 257)])
    prog = rpn.random_tree(rng, n_leaves=4, depth=rng.randint(1, 6),
                           ops_un=rpn.UN_ARITH + ["exp", "sqrt", "log"])
    toks = []
    for t in prog.split():  # keep exp/log/sqrt in range
        if t in ("sqrt", "log"):
            toks += ["abs", "#1", "+", t]
        elif t == "exp":
            toks += ["#0.125", "*", t]
        else:
            toks.append(t)
    prog = " ".join(toks)
    leaves = [parity.rand(m, n, dtype, seed=seed * 10 + i, kind="uniform", lo=0.5, hi=2.0) for i in range(4)]
    parity.check(prog, leaves, dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16", "i32"])
@pytest.mark.parametrize("red", ["accu", "sum:0", "sum:1", "mean", "mean:0", "mean:1", "norm:fro", "var", "var:1"])
@pytest.mark.parametrize("shape", [(1, 1), (3, 1), (1000, 1), (129, 65), (4097, 3), (2, 3000)])
def test_reductions_over_trees(dtype, red, shape):
    if dtype == "i32" and red.split(":")[0] in ("mean", "norm", "var"):
        pytest.skip("not defined for INT32 trees")
    m, n = shape
    A = parity.rand(m, n, dtype, seed=5)
    B = parity.rand(m, n, dtype, seed=6)
    parity.check("A B - #2 * A + " + red, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("n", [1, 31, 4097, 100003])
def test_dot_and_norm_vectors(dtype, n):
    a = parity.rand(n, 1, dtype, seed=7)
    b = parity.rand(n, 1, dtype, seed=8)
    parity.check("A B dot", [a, b], dtype)
    if dtype != "i32":
        parity.check("A norm", [a], dtype)
        parity.check("A trans norm", [a], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("red", [None, "accu", "sum:0", "sum:1"])
def test_strided_and_unaligned_views(dtype, red):
    A = parity.strided(70, 33, dtype, ld_extra=5, offset=1, seed=11)   # unaligned, ld = 76
    B = parity.strided(70, 33, dtype, ld_extra=2, offset=0, seed=12)   # aligned base, odd ld
    C = parity.rand(90, 50, dtype, seed=13)
    prog = "A B + C submat:7:3:70:33 %"
    parity.check(prog + ("" if red is None else " " + red), [A, B, C], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "i32"])
@pytest.mark.parametrize("red", [None, "accu", "sum:0", "sum:1", "mean:1"])
def test_transposed_reads(dtype, red):
    A = parity.rand(45, 70, dtype, seed=21)
    B = parity.rand(70, 45, dtype, seed=22)
    C = parity.rand(80, 90, dtype, seed=23)
    prog = "A trans B + C submat:3:4:45:70 trans - A B trans + trans %"
    if dtype == "i32" and red == "mean:1":
        pytest.skip("mean is not defined for INT32 trees")
    parity.check(prog + ("" if red is None else " " + red), [A, B, C], dtype)


def test_empty_and_degenerate():
    for shape in [(0, 5), (5, 0), (0, 0)]:
        A = parity.rand(max(shape[0], 1), max(shape[1], 1), "f32", seed=1)[:shape[0], :shape[1]]
        for red in ["accu", "sum:0", "sum:1", "mean", "var"]:
            parity.check("A #2 * " + red, [A], "f32")
        Y, _ = parity.gpu_eval("A #2 *", [A])
        assert tuple(Y.shape) == shape


def test_int_division_by_zero_sets_flag():
    A = parity.rand(40, 3, "i32", seed=3)
    B = torch.zeros_like(A)
    coot.check_device_flag()  # clear
    parity.check("A B /", [A, B], "i32")
    assert coot.check_device_flag() & 1
    parity.check("A #3 /", [A], "i32")
    assert coot.check_device_flag() == 0


def test_in_place_axpy_aliasing():
    a = parity.rand(1000, 37, "f32", seed=1)
    b = parity.rand(1000, 37, "f32", seed=2)
    b0 = b.clone()
    A, B = coot.Mat(a), coot.Mat(b)
    coot.evaluate(B + 3 * A, out=b)   # B += 3*A (Fig. 1 of the paper)
    torch.cuda.synchronize()
    # one FP32 product then one FP32 sum per element, as two separate torch ops
    assert torch.equal(b, b0 + 3.0 * a)


def test_alias_through_transpose_is_rejected():
    a = parity.rand(64, 64, "f32", seed=1)
    A = coot.Mat(a)
    with pytest.raises(Exception, match="ALIAS"):
        coot.evaluate(A + coot.trans(A), out=a)
