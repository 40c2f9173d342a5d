"""The call cache of coot_eval (a fused call prepared once per tree, layouts,
alignment and reduction): repeated calls with new pointers give the oracle's
results, a change of alignment or layout prepares a new call, and the checks
that depend on the pointers (aliasing, a NULL result buffer) still run on a
prepared call."""
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_repeated_calls_with_new_data_and_alignment():
    prog = "A B % #2 + sum:0"
    for it in range(6):
        off = it % 2  # aligned, then a view one element in (other alignment class)
        A = parity.strided(301, 40, "f32", ld_extra=3, offset=off, seed=10 + it)
        B = parity.strided(301, 40, "f32", ld_extra=3, offset=off, seed=20 + it)
        parity.check(prog, [A, B], "f32")
        parity.check("A B - exp", [A, B], "f32")


def test_aliasing_is_checked_on_a_prepared_call():
    buf = parity.rand(200, 60, "f32", seed=1)
    A = buf[:, :50]
    Y = parity.rand(200, 50, "f32", seed=2)
    ma = coot.Mat(A)
    coot.evaluate(ma + 1.0, out=Y)          # prepares the call (out apart from A)
    coot.evaluate(ma + 1.0, out=A)          # identical read: allowed in place
    with pytest.raises(L.CootError, match="ALIAS"):
        coot.evaluate(ma + 1.0, out=buf[:, 1:51])  # same layout, shifted onto A: rejected


def test_null_result_buffer_on_a_prepared_call():
    A = parity.rand(64, 64, "f32", seed=3)
    tree, _, cm = coot.expr.lower(coot.Mat(A) * 2.0)
    ctx = coot.context()
    r = torch.empty((), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    L.coot_eval(ctx, tree, cm, None, L.reduce(L.R_ACCU), r.data_ptr(), s)
    with pytest.raises(L.CootError, match="red_out is NULL"):
        L.coot_eval(ctx, tree, cm, None, L.reduce(L.R_ACCU), None, s)
    torch.cuda.synchronize()
    parity.compare_reduction(r, oracle.evaluate("A #2 * accu", parity.host([A]), "f32"), "f32", "accu")
