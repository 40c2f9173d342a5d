"""The matrix product with the tree fused onto it (trans(X)*Y and the other
operand layouts), BF16/FP16 on the tensor cores with FP32 accumulation, vs
the FP64 oracle: element by element within the bound k u sum|a b| plus the
epilogue's node bounds and the rounding to the storage type.  Ragged shapes
across several 128 x 128 tiles and 32-deep K steps, unaligned operands (the
element-by-element copy path), epilogues with extra leaves and scalars, and
the edge cases."""
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (16, 8, 16), (100, 70, 33), (128, 128, 32), (257, 129, 300), (1000, 40, 8), (64, 64, 1000)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def operand(rows, cols, dtype, seed, offset=0):
    if offset:
        return parity.strided(rows, cols, dtype, ld_extra=3, offset=offset, seed=seed)
    return parity.rand(rows, cols, dtype, seed=seed)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("ta,tb", [(True, False), (False, False), (True, True), (False, True)])
@pytest.mark.parametrize("shape", SHAPES)
def test_product_every_layout(dtype, ta, tb, shape):
    m, n, k = shape
    A = operand(k, m, dtype, 1) if ta else operand(m, k, dtype, 1)
    B = operand(n, k, dtype, 2) if tb else operand(k, n, dtype, 2)
    X, Y = coot.Mat(A), coot.Mat(B)
    e = (coot.trans(X) if ta else X) * (coot.trans(Y) if tb else Y)
    out = coot.evaluate(e)
    torch.cuda.synchronize()
    prog = "A" + (" trans" if ta else "") + " B" + (" trans" if tb else "") + " mm"
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B]), dtype), dtype, prog)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("epi", ["P #2 * C +", "P exp", "P C % D - abs sqrt", "#1 P -"])
@pytest.mark.parametrize("shape", [(100, 70, 33), (257, 129, 300)])
def test_fused_epilogues(dtype, epi, shape):
    m, n, k = shape
    A = operand(k, m, dtype, 3)        # trans(X) * Y: the paper's form
    B = operand(k, n, dtype, 4)
    C = operand(m, n, dtype, 5)
    D = operand(m, n, dtype, 6)
    if "exp" in epi or "sqrt" in epi:
        A = A * 0.05
        B = B * 0.05
    X, Y, Cm, Dm = coot.Mat(A), coot.Mat(B), coot.Mat(C), coot.Mat(D)
    P = coot.trans(X) * Y
    e = {"P #2 * C +": lambda: 2 * P + Cm, "P exp": lambda: coot.exp(P),
         "P C % D - abs sqrt": lambda: coot.sqrt(coot.abs(P % Cm - Dm)), "#1 P -": lambda: 1 - P}[epi]()
    out = coot.evaluate(e)
    torch.cuda.synchronize()
    prog = epi.replace("P", "A trans B mm")
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B, C, D]), dtype), dtype, prog)
    assert coot.last_launch()["kernel"] == "coot_gemm"


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("ta,tb", [(True, False), (False, True)])
def test_unaligned_operands(dtype, ta, tb):
    m, n, k = 130, 75, 61
    A = operand(k, m, dtype, 7, offset=1) if ta else operand(m, k, dtype, 7, offset=1)
    B = operand(n, k, dtype, 8, offset=1) if tb else operand(k, n, dtype, 8, offset=1)
    X, Y = coot.Mat(A), coot.Mat(B)
    out = coot.evaluate((coot.trans(X) if ta else X) * (coot.trans(Y) if tb else Y) + 1.0)
    torch.cuda.synchronize()
    prog = "A" + (" trans" if ta else "") + " B" + (" trans" if tb else "") + " mm #1 +"
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B]), dtype), dtype, prog)


def test_edge_cases_and_errors():
    A = parity.rand(50, 40, "bf16", seed=9)
    B = parity.rand(50, 30, "bf16", seed=10)
    X, Y = coot.Mat(A), coot.Mat(B)
    # K = 0: the product is all zeros
    Z0 = torch.zeros((0, 40), dtype=torch.bfloat16, device="cuda")
    Z1 = torch.zeros((0, 30), dtype=torch.bfloat16, device="cuda")
    out = coot.evaluate(coot.trans(coot.Mat(Z0)) * coot.Mat(Z1) + 3.0)
    torch.cuda.synchronize()
    assert torch.equal(out.float(), torch.full((40, 30), 3.0, device="cuda"))
    with pytest.raises(ValueError):
        X * Y                                    # 50x40 times 50x30
    with pytest.raises(L.CootError, match="UNSUPPORTED"):
        F = parity.rand(50, 40, "f32", seed=11)
        G = parity.rand(50, 30, "f32", seed=12)
        coot.evaluate(coot.trans(coot.Mat(F)) * coot.Mat(G))
    with pytest.raises(L.CootError, match="ALIAS"):
        coot.evaluate(coot.trans(X) * Y, out=A[:40, :30])   # out overlaps an operand
