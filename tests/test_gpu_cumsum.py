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


# ---------------------------------------------------------------------------
# the one-pass row scan (coot_scanp_*): bands of 32 V rows, panels of 8 warps
# x UC columns; every variant forced in turn
# ---------------------------------------------------------------------------
SCANP = [(1, 16, 8), (2, 8, 8)]
TDT = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16, "f16": torch.float16,
       "i32": torch.int32}


def _scanp_names(dtype):
    vmax = 16 // TDT[dtype].itemsize
    return ["coot_scanp_v%du%dw%d" % (v, uc, nw) for v, uc, nw in SCANP if v <= vmax]


def _ld(m):
    return m + 8 + (-m) % 8  # columns 16-byte aligned for every dtype


def _aligned(m, n, dtype, seed, kind="normal"):
    return parity.strided(m, n, dtype, ld_extra=_ld(m) - m, seed=seed, kind=kind)


def _aligned_out(m, n, dtype):
    return torch.zeros((n, _ld(m)), dtype=TDT[dtype], device="cuda").t()[:m, :]


def _scan_into(prog, tensors, out):
    import coot_rpn

    e, red = coot_rpn.build(prog, tensors)
    coot.evaluate(e, reduction=red, materialise=out)
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16", "i32"])
@pytest.mark.parametrize("shape", [(1, 1), (33, 1), (5, 200), (257, 64), (1001, 300), (4100, 129)])
def test_one_pass_row_scan_every_variant(dtype, shape, monkeypatch):
    # ragged bands (rows not a multiple of 32 V), ragged panels (columns not
    # a multiple of 8 UC), partial vectors at the bottom of the last band
    m, n = shape
    A, B, C = (_aligned(m, n, dtype, seed=20 + s) for s in range(3))
    prog = "A B % C + cumsum:1"
    want = oracle.evaluate(prog, parity.host([A, B, C]), dtype)
    for kname in _scanp_names(dtype):
        monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
        out = _aligned_out(m, n, dtype)
        _scan_into(prog, [A, B, C], out)
        info = coot.last_launch()
        assert info["kernel"] == kname and info["n_launches"] == 1, info
        parity.compare_matrix(out, want, dtype, "%s %s %dx%d" % (kname, dtype, m, n))


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_one_pass_row_scan_of_views_transposed_trees_and_in_place(dtype, monkeypatch):
    for kname in _scanp_names(dtype):
        monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
        # unaligned strided views (scalar variant only)
        A = parity.strided(301, 150, dtype, ld_extra=5, offset=1, seed=30)
        B = parity.strided(301, 150, dtype, ld_extra=2, offset=1, seed=31)
        if kname == "coot_scanp_v1u16w8":
            parity.check("A B % cumsum:1", [A, B], dtype)
            assert coot.last_launch()["kernel"] == kname
        # a transposed tree: materialised by the tile kernel, then scanned in place
        P = parity.rand(130, 290, dtype, seed=32)
        Q = parity.rand(290, 130, dtype, seed=33)
        parity.check("A trans B + cumsum:1", [P, Q], dtype)
        # in place: the scan's output is its own input
        X = _aligned(700, 90, dtype, seed=34)
        hs = parity.host([X])
        want = oracle.evaluate("A cumsum:1", hs, dtype)
        M = coot.Mat(X)
        coot.evaluate(M, reduction=coot.cumsum(M, 1), materialise=X)
        torch.cuda.synchronize()
        assert coot.last_launch()["kernel"] == kname
        parity.compare_matrix(X, want, dtype, "in-place " + kname)


def test_one_pass_row_scan_is_the_default_for_tall_matrices():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    m = 32 * sms + 7
    A, B = (parity.rand(m, 40, "f32", seed=s) for s in (40, 41))
    parity.check("A B - cumsum:1", [A, B], "f32")
    info = coot.last_launch()
    assert info["kernel"].startswith("coot_scanp_") and info["n_launches"] == 1, info
    # fewer rows than one band per SM: the segmented scan
    A, B = (parity.rand(300, 4000, "f32", seed=s) for s in (42, 43))
    parity.check("A B - cumsum:1", [A, B], "f32")
    assert not coot.last_launch()["kernel"].startswith("coot_scanp_")


@pytest.mark.parametrize("kname", ["coot_scan_v4u2", "coot_scan_v4u4", "coot_scanp_v1u16w8", "coot_scanp_v2u8w8"])
def test_row_scans_do_not_evaluate_rows_past_the_end(kname, monkeypatch):
    # INT32 division: the padding rows of the last partial vector hold zeros,
    # and evaluating them would raise the division-by-zero flag
    m, n = 1001, 70
    A = _aligned(m, n, "i32", seed=50)
    B = _aligned(m, n, "i32", seed=51)
    B.copy_(B.abs() + 1)
    monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
    coot.check_device_flag()  # clear
    out = _aligned_out(m, n, "i32")
    _scan_into("A B / cumsum:1", [A, B], out)
    assert coot.last_launch()["kernel"] == kname
    assert coot.check_device_flag() == 0
    parity.compare_matrix(out, oracle.evaluate("A B / cumsum:1", parity.host([A, B]), "i32"), "i32", kname)


def test_one_pass_row_scan_is_float_float_accurate(monkeypatch):
    # long rows through the one-pass scan: every prefix within one ulp of the
    # exactly rounded prefix, as for the column scan
    monkeypatch.setenv("COOT_FORCE_KERNEL", "coot_scanp_v1u16w8")
    g = torch.Generator(device="cuda").manual_seed(14)
    a = (torch.rand((1 << 16, 40), generator=g, device="cuda") * 2 - 1).float().t()  # 40 x 65536 column-major
    hs = parity.host([a])
    r = oracle.evaluate("A cumsum:1", hs, "f32")
    y = coot.cumsum(coot.Mat(a), 1).eval()
    torch.cuda.synchronize()
    assert coot.last_launch()["kernel"] == "coot_scanp_v1u16w8"
    y = y.cpu().double().numpy()
    exact_f32 = r.value.astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(exact_f32).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(y - exact_f32) <= ulp)


# ---------------------------------------------------------------------------
# trees with transposed reads scanned in one pass: along dim 1 directly (the
# transposed slots read along each thread's run of columns), along dim 0 over
# the transposed problem (the output written transposed); both when the scan
# lines outnumber 32 x the SMs.  16-byte aligned runs are read and written as
# vectors, others element by element.
# ---------------------------------------------------------------------------
def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16", "i32"])
@pytest.mark.parametrize("dim", [0, 1])
@pytest.mark.parametrize("ragged", [0, 1])
def test_transposed_tree_scanned_in_one_pass(dtype, dim, ragged):
    long_, short = 32 * _sms() + 7, 300 + ragged  # ragged: runs of the output not 16-byte aligned
    m, n = (long_, short) if dim == 1 else (short, long_)
    A = parity.rand(n, m, dtype, seed=60)      # read transposed
    B = parity.rand(m, n, dtype, seed=61)
    C = parity.rand(m, n, dtype, seed=62)
    prog = "A trans B %% C + cumsum:%d" % dim
    parity.check(prog, [A, B, C], dtype)
    info = coot.last_launch()
    assert info["kernel"] == "coot_scanp_v1u16w8" and info["n_launches"] == 1, info


@pytest.mark.parametrize("dtype", ["f32", "i32"])
@pytest.mark.parametrize("dim", [0, 1])
def test_transposed_scan_of_unaligned_and_broadcast_views(dtype, dim):
    long_, short = 32 * _sms() + 3, 97
    m, n = (long_, short) if dim == 1 else (short, long_)
    # transposed reads of views that start one element into their buffer (no
    # vector runs), a column and a row repeated over the tree
    A = parity.strided(n, m, dtype, ld_extra=5, offset=1, seed=63)
    B = parity.strided(m, n, dtype, ld_extra=2, offset=1, seed=64)
    col = parity.rand(m, 1, dtype, seed=65)
    row = parity.rand(1, n, dtype, seed=66)
    prog = "A trans B - C each_col:%d %% D each_row:%d + cumsum:%d" % (n, m, dim)
    parity.check(prog, [A, B, col, row], dtype)
    assert coot.last_launch()["kernel"] == "coot_scanp_v1u16w8"


def test_transposed_scan_falls_back_to_two_steps_for_short_lines():
    # fewer scan lines than 32 x the SMs: materialised, then scanned
    A = parity.rand(500, 200, "f32", seed=67)
    B = parity.rand(200, 500, "f32", seed=68)
    parity.check("A trans B + cumsum:1", [A, B], "f32")
    assert coot.last_launch()["n_launches"] >= 2


@pytest.fixture
def tuned(monkeypatch):
    # the module's context swapped for an autotuning one (the benchmark's
    # configuration): every kernel variant runs on the tuner's scratch output
    from paper_2508_11385_gb300 import expr as E
    from paper_2508_11385_gb300 import lib as L

    dev = torch.cuda.current_device()
    ctx = L.coot_ctx_create(dev, L.CTX_TUNE | L.CTX_NO_DISK_CACHE)
    monkeypatch.setitem(E._ctxs, dev, ctx)
    yield ctx
    torch.cuda.synchronize()
    monkeypatch.undo()
    L.coot_ctx_destroy(ctx)


@pytest.mark.parametrize("prog", ["A trans B %% C + cumsum:%d", "A trans cumsum:%d"])
@pytest.mark.parametrize("dim", [0, 1])
def test_transposed_scans_with_autotuning(tuned, prog, dim):
    # the tuner times every variant on a plain scratch output, whatever the
    # call's output (here transposed, for dim 0)
    long_, short = 32 * _sms() + 40, 600
    m, n = (long_, short) if dim == 1 else (short, long_)
    A = parity.rand(n, m, "f32", seed=70)
    B = parity.rand(m, n, "f32", seed=71)
    C = parity.rand(m, n, "f32", seed=72)
    p = prog % dim
    parity.check(p, [A, B, C] if "B" in p else [A], "f32")


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_transposed_scan_along_dim0_of_views(dtype):
    # the transposed problem of trees with a diagonal broadcast (a general
    # read with column stride 0) and a submatrix view (column stride of its
    # parent), scanned along dim 0
    n = 32 * _sms() + 9
    A = parity.rand(n, 37, dtype, seed=80)        # read transposed: 37 x n
    B = parity.rand(40, n + 6, dtype, seed=81)    # its 37 x n block from (1, 2)
    C = parity.rand(37, 37, dtype, seed=82)       # diag: 37 x 1, repeated over n columns
    parity.check("A trans B submat:1:2:37:%d - C diag each_col:%d + cumsum:0" % (n, n), [A, B, C], dtype)
    assert coot.last_launch()["kernel"] == "coot_scanp_v1u16w8"
