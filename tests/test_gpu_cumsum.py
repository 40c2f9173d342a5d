"""cumsum of a tree along dim 0 / dim 1 vs the FP64 oracle, element by
element within the oracle's bound (element bounds plus (k-1) u sum|y| for
output k of a line): every dtype, ragged shapes that span several warps,
steps and blocks, the segmented two-pass path (few long lines), transposed
reads, strided and unaligned views, in-place scans, empty inputs and INT32
wrap-around."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 1), (1, 5), (1000, 1), (1, 1000), (129, 65), (4097, 3), (2, 3000), (3000, 2)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16", "i32"])
@pytest.mark.parametrize("red", ["cumsum", "cumsum:0", "cumsum:1"])
@pytest.mark.parametrize("shape", SHAPES)
def test_cumsum_over_trees(dtype, red, shape):
    m, n = shape
    A, B, C = (parity.rand(m, n, dtype, seed=s) for s in (1, 2, 3))
    parity.check("A B % C + " + red, [A, B, C], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red,shape", [("cumsum:0", (200003, 2)), ("cumsum:0", (50000, 7)),
                                        ("cumsum:1", (3, 70001)), ("cumsum:1", (700, 3000))])
def test_segmented_lines(dtype, red, shape):
    # few long lines: each line is cut into segments, a totals pass first
    m, n = shape
    A, B = (parity.rand(m, n, dtype, seed=s) for s in (4, 5))
    prog = ("A B -" if dtype == "i32" else "A B - #0.5 *") + " " + red
    parity.check(prog, [A, B], dtype)
    info = coot.last_launch()
    assert info["n_launches"] in (1, 2)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", ["cumsum:0", "cumsum:1"])
def test_cumsum_with_transposed_reads(dtype, red):
    A = parity.rand(90, 170, dtype, seed=6)
    B = parity.rand(170, 90, dtype, seed=7)
    parity.check("A trans B + " + red, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", ["cumsum:0", "cumsum:1"])
@pytest.mark.parametrize("offset", [0, 1])
def test_cumsum_on_strided_and_unaligned_views(dtype, red, offset):
    A = parity.strided(301, 37, dtype, ld_extra=5, offset=offset, seed=8)
    B = parity.strided(301, 37, dtype, ld_extra=2, offset=offset, seed=9)
    parity.check("A B % " + red, [A, B], dtype)


@pytest.mark.parametrize("dtype", ["f32", "i32"])
@pytest.mark.parametrize("dim", [0, 1])
def test_cumsum_in_place(dtype, dim):
    A = parity.rand(513, 77, dtype, seed=10)
    hs = parity.host([A])
    want = oracle.evaluate("A cumsum:%d" % dim, hs, dtype)
    # in place: the scan's output is its own input
    M = coot.Mat(A)
    coot.evaluate(M, reduction=coot.cumsum(M, dim), materialise=A)
    torch.cuda.synchronize()
    parity.compare_matrix(A, want, dtype, "in-place cumsum")


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("shape", [(0, 0), (0, 5), (5, 0)])
def test_empty_cumsum(dtype, shape):
    m, n = shape
    tdt = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32}[dtype]
    A = torch.zeros((n, m), dtype=tdt, device="cuda").t()
    for red in ["cumsum:0", "cumsum:1"]:
        Y = coot.cumsum(coot.Mat(A), int(red[-1])).eval()
        assert tuple(Y.shape) == (m, n)


def test_int_cumsum_wraps():
    a = torch.tensor([[2 ** 31 - 1], [5], [-7], [-(2 ** 31)], [-3]], dtype=torch.int32).cuda()
    parity.check("A cumsum", [a], "i32")


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
@pytest.mark.parametrize("red", ["cumsum:0", "cumsum:1"])
def test_unfused_cumsum_matches_the_oracle(dtype, red):
    A, B = (parity.rand(400, 300, dtype, seed=s) for s in (11, 12))
    parity.check("A B - " + red, [A, B], dtype, fused=False)


def test_fp32_cumsum_is_float_float_accurate():
    # exact prefix sums rounded once: integer-valued data keeps every prefix
    # exact below 2^24, also where a running FP32 sum of 0.1 increments
    # would drift -- here the check is against the exactly rounded prefix
    g = torch.Generator(device="cuda").manual_seed(13)
    a = (torch.rand((1 << 18, 1), generator=g, device="cuda") * 2 - 1).float()
    hs = parity.host([a])
    r = oracle.evaluate("A cumsum", hs, "f32")
    y = coot.cumsum(coot.Mat(a)).eval().cpu().double().numpy()
    exact_f32 = r.value.astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(exact_f32).astype(np.float32)).astype(np.float64)
    # float-float: within one ulp of the exactly rounded prefix (a plain
    # FP32 running sum of 2^18 terms drifts by many ulps)
    assert np.all(np.abs(y - exact_f32) <= ulp)
