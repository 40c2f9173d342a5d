"""Per-row sums without allocation (coot_sum_rows_f32_noalloc).

This entry point is for callers that cannot allocate device memory while they
run -- a framework that hands out every byte through its own pool, or code in
a region where an allocation would synchronise the device or is forbidden.
Its result is checked against the FP64 oracle's sum / mean along dim 1 and
against the ordinary entry point (coot_eval with a sum or mean along dim 1)
on the same inputs, on two calls in a row, and device free memory must not
change across those calls.  A second process starts with the scratch array
filled with garbage (as a call that failed part-way could leave it) and must
still get correct sums.  The file sorts last so that a run stopping at the
first failure has run every other test before it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L

pytestmark = pytest.mark.gpu

REL = parity.REL["f32"]  # the reductions' relative tolerance used by every parity test
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _check_against_oracle(got, x, mean, what):
    """got (float64, n_rows) against the oracle's sum:1 / mean:1 of x, within
    the suite's FP32 reduction tolerance (1e-6 relative; a bare leaf has no
    element bound)."""
    r = oracle.evaluate("A mean:1" if mean else "A sum:1", parity.host([x]), "f32")
    parity.compare_reduction(torch.from_numpy(got), r, "f32", what)


@pytest.mark.parametrize("mean", [0, 1])
def test_no_alloc_row_sums_match_the_oracle_and_the_allocating_path(mean):
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
            _check_against_oracle(got, x, mean, "%s, call %d" % (what, call))
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


def test_no_alloc_rejects_row_strided_views():
    x = parity.rand(64, 8, "f32", seed=10)
    out = torch.full((8,), 7.0, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    # rows 2 apart (a row-strided view of x): rejected, nothing written
    m = L.mat(x.data_ptr(), L.F32, 8, 8, ld=64, rs=2)
    with pytest.raises(L.CootError) as e:
        L.coot_sum_rows_f32_noalloc(m, 0, out.data_ptr(), s)
    assert e.value.name == "COOT_ERR_UNSUPPORTED"
    m = L.mat(x.data_ptr(), L.F32, 8, 8, ld=64, rs=-1)
    with pytest.raises(L.CootError) as e:
        L.coot_sum_rows_f32_noalloc(m, 0, out.data_ptr(), s)
    assert e.value.name == "COOT_ERR_INVALID"
    torch.cuda.synchronize()
    assert torch.equal(out, torch.full_like(out, 7.0))


_POISONED = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np, torch
import oracle, parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L
s = torch.cuda.current_stream().cuda_stream
for seed, (r, c) in enumerate([(8192, 4096), (4097, 33), (70, 900)]):
    x = parity.rand(r, c, "f32", seed=20 + seed)
    out = torch.full((r,), float("nan"), dtype=torch.float32, device="cuda")
    for call in range(2):
        L.coot_sum_rows_f32_noalloc(coot.Mat(x).cmat(), 0, out.data_ptr(), s)
        torch.cuda.synchronize()
        res = oracle.evaluate("A sum:1", parity.host([x]), "f32")
        parity.compare_reduction(out.cpu(), res, "f32", "poisoned scratch %dx%d call %d" % (r, c, call))
        out.fill_(float("nan"))
print("poisoned-scratch ok")
"""


def test_no_alloc_correct_after_a_poisoned_scratch():
    """A fresh process whose first call finds every ticket and partial of the
    scratch set to garbage (0xA5 bytes) must still produce the oracle's sums:
    each call clears the tickets it uses before its launch."""
    env = dict(os.environ, COOT_NOALLOC_POISON_SCRATCH="1")
    code = _POISONED.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                       timeout=600)
    out = r.stdout.decode(errors="replace")
    assert r.returncode == 0 and "poisoned-scratch ok" in out, out[-3000:]
