"""Broadcasting (X.each_col() / X.each_row() operands) and diagonal views
(X.diag(k)) fused into the tree, vs the FP64 oracle element by element:
every dtype and kernel family (flat, per column, per row, transposed tiles,
scans), broadcast and diagonal reads of leaves and of expressions,
row-strided leaves, diagonals as outputs (Z.diag() += 100), in-place view
updates, and the unfused path."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 1), (1, 5), (129, 65), (4097, 3), (2, 3000)]
REDS = [None, "accu", "sum:0", "sum:1", "max:1", "index_min:0", "cumsum:0", "cumsum:1"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("red", REDS)
@pytest.mark.parametrize("shape", SHAPES)
def test_each_col_and_each_row(dtype, red, shape):
    m, n = shape
    A = parity.rand(m, n, dtype, seed=1)
    v = parity.rand(m, 1, dtype, seed=2)
    r = parity.rand(1, n, dtype, seed=3)
    prog = "A B each_col:%d %% C each_row:%d +" % (n, m) + ("" if red is None else " " + red)
    parity.check(prog, [A, v, r], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", [None, "accu", "sum:0", "index_max:1", "cumsum:1"])
def test_broadcast_with_transposed_reads(dtype, red):
    m, n = 77, 130
    A = parity.rand(n, m, dtype, seed=4)   # read as trans(A): m x n
    v = parity.rand(m, 1, dtype, seed=5)
    r = parity.rand(n, 1, dtype, seed=6)   # trans(r) is the 1 x n row
    prog = "A trans B each_col:%d - C trans each_row:%d %%" % (n, m) + ("" if red is None else " " + red)
    parity.check(prog, [A, v, r], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("k", [0, 2, -3])
@pytest.mark.parametrize("red", [None, "accu", "max", "cumsum"])
def test_diagonals_of_leaves_and_expressions(dtype, k, red):
    A, B = (parity.rand(300, 211, dtype, seed=s) for s in (7, 8))
    tail = "" if red is None else " " + red
    parity.check("A diag:%d%s" % (k, tail), [A, B], dtype)
    parity.check("A B %% #2 + diag:%d%s" % (k, tail), [A, B], dtype)
    parity.check("A trans B trans - diag:%d%s" % (k, tail), [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
def test_diagonal_broadcast(dtype):
    # diag(A) repeated over the columns of B: a general read with cs = 0
    A = parity.rand(64, 40, dtype, seed=9)
    Z = parity.rand(64, 64, dtype, seed=10)
    parity.check("A B diag each_col:40 +", [A, Z], dtype)
    parity.check("A B diag each_col:40 + sum:1", [A, Z], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_row_strided_leaves(dtype):
    # every third row of a matrix, and a diagonal passed as a 1-D strided tensor
    big = parity.rand(900, 50, dtype, seed=11)
    A = big[::3]                                 # 300 x 50, rows 3 apart
    assert A.stride(0) == 3
    B = parity.rand(300, 50, dtype, seed=12)
    parity.check("A B +", [A, B], dtype)
    parity.check("A B % sum:1", [A, B], dtype)
    Z = parity.rand(200, 200, dtype, seed=13)
    d = Z.diagonal()                             # 1-D, stride ld + 1
    w = parity.rand(200, 1, dtype, seed=14)
    parity.check("A B -", [d, w.view(-1)], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("k", [0, 5, -7])
def test_diagonal_as_the_output(dtype, k):
    # Z.diag(k) += 100 (Fig. 1 of the paper): only the diagonal changes
    Z = parity.rand(150, 120, dtype, seed=15)
    before = Z.clone()
    want = oracle.evaluate("A diag:%d #100 +" % k, parity.host([Z]), dtype)
    d = coot.Mat(Z).diag(k)
    d += 100
    torch.cuda.synchronize()
    got = Z.diagonal(k)
    parity.compare_matrix(got.reshape(-1, 1), want, dtype, "Z.diag(%d) += 100" % k)
    mask = torch.ones_like(Z, dtype=torch.bool)
    mask.diagonal(k).fill_(False)
    assert torch.equal(Z[mask], before[mask])


def test_diagonal_output_of_a_tree_and_an_alias_that_must_fail():
    Z = parity.rand(100, 100, "f32", seed=16)
    A = parity.rand(100, 1, "f32", seed=17)
    want = oracle.evaluate("A B diag %", parity.host([A, Z]), "f32")
    coot.evaluate(coot.Mat(A) % coot.Mat(Z).diag(), out=coot.Mat(Z).diag())  # same elements in place
    torch.cuda.synchronize()
    parity.compare_matrix(Z.diagonal().reshape(-1, 1), want, "f32", "diag(Z) = A % diag(Z)")
    # reading the diagonal shifted by one while writing it races: rejected
    Zm = coot.Mat(Z)
    with pytest.raises(coot.lib.CootError, match="ALIAS"):
        coot.evaluate(Zm.submat(0, 1, 98, 99).diag() + 1, out=Zm.submat(0, 0, 98, 98).diag())


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_in_place_submatrix_and_matrix_updates(dtype):
    A = parity.rand(90, 70, dtype, seed=18)
    B = parity.rand(90, 70, dtype, seed=19)
    want = oracle.evaluate("A B +", parity.host([A, B]), dtype)
    M = coot.Mat(A)
    M += coot.Mat(B)
    torch.cuda.synchronize()
    parity.compare_matrix(A, want, dtype, "A += B")
    C = parity.rand(90, 70, dtype, seed=20)
    before = C.clone()
    v = coot.Mat(C).submat(10, 5, 39, 24)
    v -= 3
    torch.cuda.synchronize()
    assert torch.equal(C[10:40, 5:25], before[10:40, 5:25] - 3)
    C[10:40, 5:25] = before[10:40, 5:25]
    assert torch.equal(C, before)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("prog", ["A B each_col:70 % C each_row:90 +", "A diag #1 + accu",
                                  "A B each_col:70 - sum:1"])
def test_unfused_views_match_the_oracle(dtype, prog):
    A = parity.rand(90, 70, dtype, seed=21)
    v = parity.rand(90, 1, dtype, seed=22)
    r = parity.rand(1, 70, dtype, seed=23)
    parity.check(prog, [A, v, r], dtype, fused=False)


def test_views_are_rejected_where_unsupported():
    # the adjoint needs every leaf read whole: a broadcast read is not
    from paper_2508_11385_gb300 import autograd
    A = parity.rand(64, 32, "f32", seed=24)
    v = parity.rand(64, 1, "f32", seed=25)
    loss = autograd.Loss(lambda a, b: coot.accu(a.each_col() + b), A, v)
    up = torch.ones((), dtype=torch.float32, device="cuda")
    with pytest.raises(coot.lib.CootError, match="UNSUPPORTED"):
        loss.backward(up, A, v)


def test_diagonal_output_with_autotuning(monkeypatch):
    # Z.diag() += 1 in an autotuning context: the tuner's scratch output is
    # plain column-major, whatever the strides of the call's output
    from paper_2508_11385_gb300 import expr as E
    from paper_2508_11385_gb300 import lib as L

    dev = torch.cuda.current_device()
    ctx = L.coot_ctx_create(dev, L.CTX_TUNE | L.CTX_NO_DISK_CACHE)
    monkeypatch.setitem(E._ctxs, dev, ctx)
    try:
        Z = parity.rand(3000, 2900, "f32", seed=16)
        before = Z.clone()
        want = oracle.evaluate("A diag:3 #1 +", parity.host([Z]), "f32")
        d = coot.Mat(Z).diag(3)
        d += 1
        torch.cuda.synchronize()
        parity.compare_matrix(Z.diagonal(3).reshape(-1, 1), want, "f32", "Z.diag(3) += 1, tuned")
        mask = torch.ones_like(Z, dtype=torch.bool)
        mask.diagonal(3).fill_(False)
        assert torch.equal(Z[mask], before[mask])
    finally:
        torch.cuda.synchronize()
        monkeypatch.undo()
        L.coot_ctx_destroy(ctx)
