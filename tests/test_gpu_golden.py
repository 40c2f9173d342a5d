"""The CUDA path against the worked cases in tests/golden/ (hand-written
expected values: the paper's example program of Sec. 2, Fig. 1, closed forms
of the statistics, element-wise functions, transposes and views, and the int32
element type), with the tolerance each case states.  The diagonal update of
Fig. 1 also runs in place (Z.diag() += 100) and the whole matrix is checked."""
import numpy as np
import pytest
import torch

import coot_rpn
import golden_cases
import parity
import paper_2508_11385_gb300 as coot

pytestmark = pytest.mark.gpu

_TORCH = {"f32": torch.float32, "f64": torch.float64, "i32": torch.int32, "bf16": torch.bfloat16,
          "f16": torch.float16}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def device_leaf(leaf, dtype):
    """Column-major device tensor holding the leaf's stored values."""
    h = golden_cases.host_leaf(leaf, dtype)
    rows_major = np.ascontiguousarray(h.T)  # (n_cols, n_rows) row-major = column-major (n_rows, n_cols)
    if dtype in ("bf16", "f16"):
        t = torch.from_numpy(rows_major.view(np.int16)).view(_TORCH[dtype])
    else:
        t = torch.from_numpy(rows_major)
    return t.to("cuda").t()


def gpu_program(prog):
    # the oracle spells the matrix product "mm"; the library's operator is *
    return " ".join("*" if tok == "mm" else tok for tok in prog.split())


@pytest.mark.parametrize("case,dtype", golden_cases.params())
def test_gpu_matches_golden(case, dtype):
    tensors = [device_leaf(l, dtype) for l in case.leaves]
    Y, r = parity.gpu_eval(gpu_program(case.prog), tensors)
    torch.cuda.synchronize()
    got = parity.to_f64(r if r is not None else Y)
    golden_cases.check(got, case, dtype, "%s/%s" % (case.name, dtype))


@pytest.mark.parametrize("case,dtype", [p for p in golden_cases.params() if p.values[0].after is not None])
def test_gpu_diagonal_update_in_place(case, dtype):
    tensors = [device_leaf(l, dtype) for l in case.leaves]
    target = tensors[case.leaf_index(case.after.name)]
    expr, red = coot_rpn.build(gpu_program(case.prog), tensors)
    assert red is None
    coot.evaluate(expr, out=coot.Mat(target).diag())
    torch.cuda.synchronize()
    golden_cases.check_after(parity.to_f64(target), case.after, "%s/%s in place" % (case.name, dtype))
