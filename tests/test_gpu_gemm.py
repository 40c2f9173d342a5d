"""The matrix product with the tree fused onto it (trans(X)*Y and the other
operand layouts), BF16/FP16 on the tensor cores with FP32 accumulation and
FP32/FP64 on the CUDA cores, vs
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
        F = parity.rand(50, 40, "i32", seed=11)
        G = parity.rand(50, 30, "i32", seed=12)
        coot.evaluate(coot.trans(coot.Mat(F)) * coot.Mat(G))
    with pytest.raises(L.CootError, match="ALIAS"):
        coot.evaluate(coot.trans(X) * Y, out=A[:40, :30])   # out overlaps an operand


# the tcgen05 kernel: trans(X) * Y with 16-byte aligned operands and column
# strides (k a multiple of 8 here); ragged m, n and k come in as TMA zeros
TC_SHAPES = [(128, 256, 64), (256, 512, 96), (128, 768, 1024), (1024, 256, 160), (130, 260, 72), (1, 1, 8),
             (300, 20, 8), (1000, 40, 8), (64, 64, 1000)]


def _no_tc_context(dev):
    """A second context whose GEMMs always take the mma.sync kernel."""
    return L.coot_ctx_create(torch.device(dev).index or 0, L.CTX_NO_TCGEN05)


def _tc_expected(m, n, k, ta, tb):
    # contiguous operands: TMA needs the column strides to be multiples of 8 elements
    lda = k if ta else m
    ldb = n if tb else k
    return "coot_gemm_tc" if lda % 8 == 0 and ldb % 8 == 0 else "coot_gemm"


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("ta,tb", [(True, False), (False, False), (True, True), (False, True)])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_tcgen05_product(dtype, ta, tb, shape):
    # K-major (trans(X), Y) and MN-major (X, trans(Y)) operands
    m, n, k = shape
    A = operand(k, m, dtype, 21) if ta else operand(m, k, dtype, 21)
    B = operand(n, k, dtype, 22) if tb else operand(k, n, dtype, 22)
    X, Y = coot.Mat(A), coot.Mat(B)
    out = coot.evaluate((coot.trans(X) if ta else X) * (coot.trans(Y) if tb else Y))
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == _tc_expected(m, n, k, ta, tb)
    assert coot.check_device_flag() == 0
    prog = "A" + (" trans" if ta else "") + " B" + (" trans" if tb else "") + " mm"
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B]), dtype), dtype, prog)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("epi", ["P #2 * C +", "P C % D - abs sqrt", "#1 P -"])
@pytest.mark.parametrize("shape", [(256, 512, 320), (200, 300, 136)])
def test_tcgen05_fused_epilogues(dtype, epi, shape):
    m, n, k = shape
    A = operand(k, m, dtype, 23) * 0.1
    B = operand(k, n, dtype, 24) * 0.1
    C = operand(m, n, dtype, 25)
    D = operand(m, n, dtype, 26)
    X, Y, Cm, Dm = coot.Mat(A), coot.Mat(B), coot.Mat(C), coot.Mat(D)
    P = coot.trans(X) * Y
    e = {"P #2 * C +": lambda: 2 * P + Cm, "P C % D - abs sqrt": lambda: coot.sqrt(coot.abs(P % Cm - Dm)),
         "#1 P -": lambda: 1 - P}[epi]()
    out = coot.evaluate(e)
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_tc"
    prog = epi.replace("P", "A trans B mm")
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B, C, D]), dtype), dtype, prog)


def test_tcgen05_and_mma_sync_agree_within_the_bound():
    # the same call through both kernels, each within the oracle's bound
    m, n, k = 384, 512, 512
    A = operand(k, m, "bf16", 27)
    B = operand(k, n, "bf16", 28)
    X, Y = coot.Mat(A), coot.Mat(B)
    tc = coot.evaluate(coot.trans(X) * Y)
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_tc"
    ctx = _no_tc_context("cuda")
    try:
        ms = torch.empty((n, m), dtype=torch.bfloat16, device="cuda").t()
        L.coot_gemm_eval(ctx, X.cmat(), 1, Y.cmat(), 0, None, [], coot.Mat(ms).cmat(),
                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert L.coot_last_launch(ctx)["kernel"] == "coot_gemm"
    finally:
        L.coot_ctx_destroy(ctx)
    ref = oracle.evaluate("A trans B mm", parity.host([A, B]), "bf16")
    parity.compare_matrix(tc, ref, "bf16", "tcgen05")
    parity.compare_matrix(ms, ref, "bf16", "mma.sync")


def test_tcgen05_output_view_and_many_tiles():
    # a strided output view and a grid of many tile groups (ragged last group)
    m, n, k = 2176, 768, 256
    A = operand(k, m, "bf16", 31)
    B = operand(k, n, "bf16", 32)
    big = torch.zeros((n + 5, m + 9), dtype=torch.bfloat16, device="cuda").t()
    out = big[3:3 + m, 2:2 + n]
    coot.evaluate(coot.trans(coot.Mat(A)) * coot.Mat(B) + 0.5, out=out)
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_tc"
    parity.compare_matrix(out, oracle.evaluate("A trans B mm #0.5 +", parity.host([A, B]), "bf16"), "bf16", "view")
    assert float(big[:3].abs().sum()) == 0.0 and float(big[3 + m:].abs().sum()) == 0.0
    assert float(big[:, :2].abs().sum()) == 0.0 and float(big[:, 2 + n:].abs().sum()) == 0.0


@pytest.mark.parametrize("case", ["k=61 (column stride not a multiple of 8)", "unaligned base",
                                  "X*Y with m=130 (column stride of X)"])
def test_tcgen05_declines(case):
    m, n, k = 128, 256, 64
    if case.startswith("k=61"):
        A, B, ta = operand(61, m, "bf16", 33), operand(61, n, "bf16", 34), True
    elif case == "unaligned base":
        A, B, ta = operand(k, m, "bf16", 33, offset=1), operand(k, n, "bf16", 34), True
    else:
        A, B, ta = operand(130, k, "bf16", 33), operand(k, n, "bf16", 34), False
    X, Y = coot.Mat(A), coot.Mat(B)
    out = coot.evaluate((coot.trans(X) if ta else X) * Y)
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm", case
    prog = "A" + (" trans" if ta else "") + " B mm"
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B]), "bf16"), "bf16", case)


def test_tcgen05_persistent_many_tiles_sampled():
    # 32 x 17 = 544 output tiles on at most one CTA per SM: every CTA walks
    # several tiles through both accumulator buffers.  Sampled rows and
    # columns of the result against the oracle on the matching operand columns.
    m, n, k = 4096, 4352 - 40, 200
    A = operand(k, m, "bf16", 35)
    B = operand(k, n, "bf16", 36)
    C = operand(m, n, "bf16", 37)
    out = coot.evaluate(coot.trans(coot.Mat(A)) * coot.Mat(B) - coot.Mat(C))
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_tc"
    g = torch.Generator().manual_seed(38)
    rows = torch.cat([torch.randperm(m, generator=g)[:120], torch.tensor([0, 127, 128, m - 1])]).tolist()
    cols = torch.cat([torch.randperm(n, generator=g)[:120], torch.tensor([0, 255, 256, n - 1])]).tolist()
    ri, ci = torch.tensor(rows, device="cuda"), torch.tensor(cols, device="cuda")
    As, Bs = A[:, ri].contiguous(), B[:, ci].contiguous()
    Cs = C[ri][:, ci].t().contiguous().t()
    got = out[ri][:, ci]
    ref = oracle.evaluate("A trans B mm C -", parity.host([As, Bs, Cs]), "bf16")
    parity.compare_matrix(got, ref, "bf16", "sampled")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, True)])
def test_tcgen05_mn_major_operands_with_fused_epilogue(dtype, ta, tb):
    # MN-major operands (X, trans(Y)) on the tcgen05 kernel with the tree's
    # other leaves and a scalar fused into the epilogue
    m, n, k = 256, 384, 200
    A = (operand(k, m, dtype, 41) if ta else operand(m, k, dtype, 41)) * 0.1
    B = (operand(n, k, dtype, 42) if tb else operand(k, n, dtype, 42)) * 0.1
    C = operand(m, n, dtype, 43)
    X, Y, Cm = coot.Mat(A), coot.Mat(B), coot.Mat(C)
    P = (coot.trans(X) if ta else X) * (coot.trans(Y) if tb else Y)
    out = coot.evaluate(2 * P + Cm)
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_tc"
    prog = "A" + (" trans" if ta else "") + " B" + (" trans" if tb else "") + " mm #2 * C +"
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B, C]), dtype), dtype, prog)


def test_tcgen05_gemm_in_a_graph_replays_bitwise():
    # a warmed GEMM call captured with the library's graph API: the TMA
    # descriptors travel in the kernel arguments, so the replay is exact
    m, n, k = 384, 512, 256
    A = operand(k, m, "bf16", 44)
    B = operand(k, n, "bf16", 45)
    X, Y = coot.Mat(A), coot.Mat(B)
    out = torch.empty((n, m), dtype=torch.bfloat16, device="cuda").t()
    ctx = coot.context()
    s = torch.cuda.Stream()
    call = lambda: L.coot_gemm_eval(ctx, X.cmat(), 1, Y.cmat(), 0, None, [], coot.Mat(out).cmat(), s.cuda_stream)
    call()
    torch.cuda.synchronize()
    assert L.coot_last_launch(ctx)["kernel"] == "coot_gemm_tc"
    eager = out.clone()
    out.zero_()
    torch.cuda.synchronize()
    L.coot_graph_begin(ctx, s.cuda_stream)
    call()
    g = L.coot_graph_end(ctx, s.cuda_stream)
    out.zero_()
    torch.cuda.synchronize()
    L.coot_graph_launch(g, s.cuda_stream)
    torch.cuda.synchronize()
    L.coot_graph_destroy(g)
    assert torch.equal(out, eager)
    assert coot.check_device_flag() == 0
    parity.compare_matrix(out, oracle.evaluate("A trans B mm", parity.host([A, B]), "bf16"), "bf16", "graph")


# Expressions around the fused product.  Armadillo evaluates an operand
# expression, a second product, or the product under a reduction into a
# temporary of the element type first; here the temporaries come from the
# same kernels, so each case equals its decomposition bit for bit, and the
# decomposition's pieces are checked against the oracle.

def test_operand_expressions_are_evaluated_first():
    m, n, k = 192, 256, 160
    A = operand(m, k, "bf16", 51) * 0.1
    B = operand(k, n, "bf16", 52)
    X, Y = coot.Mat(A), coot.Mat(B)
    out = coot.evaluate(coot.exp(X) * coot.trans(2 * coot.trans(Y) + 1))
    T1 = coot.evaluate(coot.exp(X))
    T2 = coot.evaluate(2 * coot.trans(Y) + 1)
    ref = coot.evaluate(coot.Mat(T1) * coot.trans(coot.Mat(T2)))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    parity.compare_matrix(T1, oracle.evaluate("A exp", parity.host([A]), "bf16"), "bf16", "exp(X)")
    parity.compare_matrix(ref, oracle.evaluate("A B trans mm", parity.host([T1, T2]), "bf16"), "bf16", "product")


def test_two_products_and_a_chained_product():
    m, n, k = 128, 192, 96
    A, B = operand(m, k, "bf16", 53), operand(k, n, "bf16", 54)
    C, D = operand(m, k, "bf16", 55), operand(k, n, "bf16", 56)
    E = operand(n, 64, "bf16", 57)
    Am, Bm, Cm, Dm, Em = (coot.Mat(t) for t in (A, B, C, D, E))
    two = coot.evaluate(Am * Bm + 0.5 * (Cm * Dm))
    Tcd = coot.evaluate(Cm * Dm)
    ref2 = coot.evaluate(Am * Bm + 0.5 * coot.Mat(Tcd))
    chained = coot.evaluate((Am * Bm) * Em)
    Tab = coot.evaluate(Am * Bm)
    ref3 = coot.evaluate(coot.Mat(Tab) * Em)
    torch.cuda.synchronize()
    assert torch.equal(two, ref2)
    assert torch.equal(chained, ref3)
    parity.compare_matrix(ref2, oracle.evaluate("A B mm #0.5 C * +", parity.host([A, B, Tcd]), "bf16"), "bf16",
                          "A*B + 0.5*T")
    parity.compare_matrix(ref3, oracle.evaluate("A B mm", parity.host([Tab, E]), "bf16"), "bf16", "T*E")


@pytest.mark.parametrize("kind", ["accu", "sum0", "sum1", "max", "cumsum0"])
def test_reductions_of_a_product(kind):
    m, n, k = 160, 224, 128
    A = operand(k, m, "bf16", 58)
    B = operand(k, n, "bf16", 59)
    C = operand(m, n, "bf16", 60)
    P = coot.trans(coot.Mat(A)) * coot.Mat(B) + coot.Mat(C)
    red = {"accu": lambda e: coot.accu(e), "sum0": lambda e: coot.sum(e, 0), "sum1": lambda e: coot.sum(e, 1),
           "max": lambda e: coot.max(e, 0), "cumsum0": lambda e: coot.cumsum(e, 0)}[kind]
    got = red(P).eval()
    Y = coot.evaluate(P)
    ref = red(coot.Mat(Y)).eval()
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    tok = {"accu": "accu", "sum0": "sum:0", "sum1": "sum:1", "max": "max:0", "cumsum0": "cumsum:0"}[kind]
    hy = parity.host([Y])
    if kind == "cumsum0":
        parity.compare_matrix(ref, oracle.evaluate("A " + tok, hy, "bf16"), "bf16", tok)
    else:
        parity.compare_reduction(ref, oracle.evaluate("A " + tok, hy, "bf16"), "bf16", tok)


# FP32 / FP64 operands: the CUDA-core kernel, accumulation in the storage type
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("ta,tb", [(True, False), (False, False), (True, True), (False, True)])
@pytest.mark.parametrize("shape", SHAPES)
def test_simt_product_every_layout(dtype, ta, tb, shape):
    m, n, k = shape
    A = operand(k, m, dtype, 61) if ta else operand(m, k, dtype, 61)
    B = operand(n, k, dtype, 62) if tb else operand(k, n, dtype, 62)
    X, Y = coot.Mat(A), coot.Mat(B)
    out = coot.evaluate((coot.trans(X) if ta else X) * (coot.trans(Y) if tb else Y))
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_simt"
    prog = "A" + (" trans" if ta else "") + " B" + (" trans" if tb else "") + " mm"
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B]), dtype), dtype, prog)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("epi", ["P #2 * C +", "P C % D - abs sqrt", "P exp"])
def test_simt_fused_epilogues(dtype, epi):
    m, n, k = 257, 130, 75
    A = operand(k, m, dtype, 63, offset=1) * 0.1   # unaligned, strided
    B = operand(k, n, dtype, 64) * 0.1
    C = operand(m, n, dtype, 65)
    D = operand(m, n, dtype, 66)
    X, Y, Cm, Dm = coot.Mat(A), coot.Mat(B), coot.Mat(C), coot.Mat(D)
    P = coot.trans(X) * Y
    e = {"P #2 * C +": lambda: 2 * P + Cm, "P C % D - abs sqrt": lambda: coot.sqrt(coot.abs(P % Cm - Dm)),
         "P exp": lambda: coot.exp(P)}[epi]()
    out = coot.evaluate(e)
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_gemm_simt"
    prog = epi.replace("P", "A trans B mm")
    parity.compare_matrix(out, oracle.evaluate(prog, parity.host([A, B, C, D]), dtype), dtype, prog)


def test_simt_large_sampled():
    # many 128 x 128 tiles with ragged edges: sampled rows and columns
    m, n, k = 1100, 700, 333
    A = operand(m, k, "f32", 67)
    B = operand(k, n, "f32", 68)
    out = coot.evaluate(coot.Mat(A) * coot.Mat(B))
    torch.cuda.synchronize()
    g = torch.Generator().manual_seed(69)
    rows = torch.cat([torch.randperm(m, generator=g)[:60], torch.tensor([0, 127, 128, m - 1])]).tolist()
    cols = torch.cat([torch.randperm(n, generator=g)[:60], torch.tensor([0, 127, 128, n - 1])]).tolist()
    ri, ci = torch.tensor(rows, device="cuda"), torch.tensor(cols, device="cuda")
    As, Bs = A[ri].t().contiguous().t(), B[:, ci].contiguous()
    parity.compare_matrix(out[ri][:, ci], oracle.evaluate("A B mm", parity.host([As, Bs]), "f32"), "f32", "sampled")
