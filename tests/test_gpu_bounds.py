"""The bounds-check build (COOT_CTX_DEBUG_BOUNDS): every leaf read and output
write of the streaming kernel families is checked against the extent of its
matrix.  Correct kernels must give the oracle's results and raise no flag on
ragged, strided, unaligned, broadcast, diagonal and transposed reads, in every
family (flat and 2-D chunk walks, per-column and per-row reductions, tiles,
scans, the adjoint).  The check itself is shown to work by declaring every
extent one element short (COOT_DEBUG_BOUNDS_SHRINK=1): the kernel then skips
the last element of each leaf -- it never reads outside the matrix -- and
raises the flag."""
import pytest
import torch

import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import expr as E
from paper_2508_11385_gb300 import lib as L
from paper_2508_11385_gb300 import workloads
from paper_2508_11385_gb300.autograd import scalar

pytestmark = pytest.mark.gpu


@pytest.fixture()
def bounds_ctx(monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.cuda.current_device()
    ctx = L.coot_ctx_create(dev, L.CTX_DEBUG_BOUNDS | L.CTX_NO_DISK_CACHE)
    monkeypatch.setitem(E._ctxs, dev, ctx)  # the library's calls in this test use it
    yield ctx
    torch.cuda.synchronize()
    monkeypatch.undo()
    L.coot_ctx_destroy(ctx)


def _leaves(dtype, seed):
    g = workloads.generator(seed, "cuda")
    mk = (lambda r, c: workloads.int_uniform(r, c, -1000, 1000, g, "cuda")) if dtype == "i32" else \
        (lambda r, c: workloads.uniform(r, c, 0.5, 2.0, dtype, g, "cuda"))
    A = mk(517 + 5, 203)[2:2 + 517, :]      # unaligned view, ld 522
    B = mk(517, 203)
    Ct = mk(203, 517)                       # read transposed
    col = mk(517, 1)
    row = mk(1, 203)
    sq = mk(518, 518)
    return [A, B, Ct, col, row, sq]


PROGS = ["A B % #2 *", "A B % accu", "A B - square sum:0", "A B + sum:1", "A C trans + max:1",
         "A C trans % sum:0", "A D each_col:203 % E each_row:517 + accu", "F diag:1 D - min",
         "F submat:1:3:517:203 A - index_max", "A B % cumsum:0", "A B % cumsum:1", "A C trans - cumsum:0",
         "A abs B % var", "A B % vardim:1:0"]


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
def test_bounds_build_matches_oracle_without_a_flag(bounds_ctx, dtype):
    leaves = _leaves(dtype, 5)
    s = torch.cuda.current_stream().cuda_stream
    for prog in PROGS:
        if dtype == "i32" and "var" in prog:
            continue
        if dtype == "bf16" and "trans" in prog and "cumsum" in prog:
            # a scan of a tree with transposed reads first materialises the
            # tree in its storage type (one more rounding for 16-bit types),
            # which the oracle's one-rounding bound does not model
            continue
        for materialise in (False, True):
            parity.check(prog, leaves, dtype, materialise=materialise)
            assert L.coot_check_device_flag(bounds_ctx, s) == 0, "%s (%s): device flag raised" % (prog, dtype)


def coot_rpn_build(prog, leaves):
    import coot_rpn

    return coot_rpn.build(prog, leaves)


def test_bounds_build_adjoint(bounds_ctx):
    W, X, Y = workloads.differentiation(n=96, device="cuda")
    Wp, Xp = W.clone().requires_grad_(True), X.clone().requires_grad_(True)
    loss = scalar(lambda w, x, y: coot.accu(coot.square(w % x - y)), Wp, Xp, Y)
    loss.backward()
    torch.cuda.synchronize()
    assert L.coot_check_device_flag(bounds_ctx, torch.cuda.current_stream().cuda_stream) == 0
    gw = 2 * (W * X - Y) * X
    assert torch.allclose(Wp.grad, gw, rtol=1e-5, atol=1e-5)


def test_a_short_extent_is_caught_and_not_read(bounds_ctx, monkeypatch):
    monkeypatch.setenv("COOT_DEBUG_BOUNDS_SHRINK", "1")
    A = parity.rand(300, 7, "f32", seed=3)
    B = parity.rand(300, 7, "f32", seed=4)
    s = torch.cuda.current_stream().cuda_stream
    for prog in ("A B % accu", "A B % #3 *", "A B trans trans + sum:1"):
        e, red = coot_rpn_build(prog, [A, B])
        if red is None:
            coot.evaluate(e)
        else:
            coot.evaluate(e, reduction=red)
        torch.cuda.synchronize()
        f = L.coot_check_device_flag(bounds_ctx, s)
        assert f & L.FLAG_OUT_OF_BOUNDS, "%s: the short extent was not reported" % prog


@pytest.mark.parametrize("dtype", ["f32", "bf16", "i32"])
def test_bounds_build_one_pass_scans(bounds_ctx, dtype, monkeypatch):
    # the one-pass row scan, forced on the mixed leaves (unaligned view,
    # broadcasts), then on trees with transposed reads scanned in one pass
    # along dim 1 (tall) and along dim 0 over the transposed problem (wide)
    s = torch.cuda.current_stream().cuda_stream
    leaves = _leaves(dtype, 6)
    monkeypatch.setenv("COOT_FORCE_KERNEL", "coot_scanp_v1u16w8")
    for prog in ("A B % cumsum:1", "A D each_col:203 % E each_row:517 + cumsum:1"):
        for materialise in (False, True):
            parity.check(prog, leaves, dtype, materialise=materialise)
            assert coot.last_launch()["kernel"] == "coot_scanp_v1u16w8"
            assert L.coot_check_device_flag(bounds_ctx, s) == 0, "%s (%s): device flag raised" % (prog, dtype)
    monkeypatch.delenv("COOT_FORCE_KERNEL")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    g = workloads.generator(7, "cuda")
    mk = (lambda r, c: workloads.int_uniform(r, c, -1000, 1000, g, "cuda")) if dtype == "i32" else \
        (lambda r, c: workloads.uniform(r, c, 0.5, 2.0, dtype, g, "cuda"))
    long_ = 32 * sms + 5
    for m, n, dim in ((long_, 37, 1), (37, long_, 0)):
        At = mk(n + 3, m)[1:1 + n, :]   # read transposed, one element into its buffer
        B = mk(m, n)
        prog = "A trans B - cumsum:%d" % dim
        parity.check(prog, [At, B], dtype)
        assert coot.last_launch()["kernel"] == "coot_scanp_v1u16w8"
        assert L.coot_check_device_flag(bounds_ctx, s) == 0, "%s (%s): device flag raised" % (prog, dtype)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_bounds_build_row_walk_with_transposed_runs(bounds_ctx, dtype):
    # reductions along dim 1 of trees with a transposed read whose runs are
    # 16-byte aligned (read by whole warps through shared memory) and a
    # ragged last warp (read lane by lane)
    s = torch.cuda.current_stream().cuda_stream
    g = workloads.generator(8, "cuda")
    mk = lambda r, c: workloads.uniform(r, c, 0.5, 2.0, dtype, g, "cuda")  # noqa: E731
    m, n = 1003, 304
    At, B = mk(n, m), mk(m, n)
    for prog in ("A trans B % sum:1", "A trans B - max:1", "A trans B + vardim:1:1"):
        parity.check(prog, [At, B], dtype)
        assert coot.last_launch()["kernel"].startswith("coot_row"), coot.last_launch()
        assert L.coot_check_device_flag(bounds_ctx, s) == 0, "%s (%s): device flag raised" % (prog, dtype)
