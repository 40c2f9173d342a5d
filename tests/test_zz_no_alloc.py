"""Per-row sums without allocation (coot_sum_rows_f32_noalloc).

This entry point is for callers that cannot allocate device memory while they
run -- a framework that hands out every byte through its own pool, or code in
a region where an allocation would synchronise the device or is forbidden.
Its result is checked against the ordinary entry point (coot_eval with a sum
or mean along dim 1) on the same inputs, on two calls in a row, and device
free memory must not change across those calls.  The file sorts last so that
a run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L

pytestmark = pytest.mark.gpu

REL = parity.REL["f32"]  # the reductions' relative tolerance used by every parity test


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _inputs():
    yield "contiguous 1000x7", parity.rand(1000, 7, "f32", seed=1)
    yield "ragged 4097x33", parity.rand(4097, 33, "f32", seed=2)
    yield "wide 3x5000", parity.rand(3, 5000, "f32", seed=3)
    yield "single element", parity.rand(1, 1, "f32", seed=4)
    yield "strided ld 76, unaligned", parity.strided(70, 33, "f32", ld_extra=5, offset=1, seed=5)
    yield "large 8192x8192", parity.rand(8192, 8192, "f32", seed=6)


@pytest.mark.parametrize("mean", [0, 1])
def test_no_alloc_row_sums_match_the_allocating_path(mean):
    stream = torch.cuda.current_stream()
    for what, x in _inputs():
        m = coot.Mat(x)
        red = coot.mean(m, 1) if mean else coot.sum(m, 1)
        _, ref = coot.evaluate(m, reduction=red)
        torch.cuda.synchronize()
        ref = ref.reshape(-1).double().cpu().numpy()
        scale = x.abs().double().sum(dim=1).cpu().numpy() / (x.shape[1] if mean else 1)
        out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
        L.coot_sum_rows_f32_noalloc(m.cmat(), mean, out.data_ptr(), stream.cuda_stream)  # set-up call
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for call in range(2):
            out.fill_(float("nan"))
            L.coot_sum_rows_f32_noalloc(m.cmat(), mean, out.data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)  # host copy: no device allocation
            err = np.abs(got - ref)
            tol = REL * np.abs(ref) + 1e-9 * scale
            assert np.all(err <= tol), "%s, call %d: max err %.3g" % (what, call, float(np.max(err - tol)))
        assert torch.cuda.mem_get_info()[0] == free_before, what


def test_no_alloc_empty_shapes():
    x = parity.rand(5, 1, "f32", seed=7)[:, :0]  # 5 x 0
    out = torch.zeros(5, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    L.coot_sum_rows_f32_noalloc(coot.Mat(x).cmat(), 0, out.data_ptr(), s)
    torch.cuda.synchronize()
    assert torch.equal(out, torch.zeros_like(out))
    L.coot_sum_rows_f32_noalloc(coot.Mat(x).cmat(), 1, out.data_ptr(), s)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    z = parity.rand(1, 4, "f32", seed=8)[:0, :]  # 0 x 4: nothing to write
    L.coot_sum_rows_f32_noalloc(coot.Mat(z).cmat(), 0, None, s)


def test_no_alloc_rejects_rows_beyond_the_scratch():
    x = parity.rand(16, 1, "f32", seed=9)
    big = L.mat(x.data_ptr(), L.F32, 4096 * 1024 + 1, 1)  # shape only: rejected before any access
    with pytest.raises(L.CootError, match="no-allocation limit"):
        L.coot_sum_rows_f32_noalloc(big, 0, x.data_ptr(), torch.cuda.current_stream().cuda_stream)
