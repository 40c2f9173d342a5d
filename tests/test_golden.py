"""The oracle against the worked cases in tests/golden/: results fixed by the
paper's example program (Sec. 2, Fig. 1), by closed forms of the statistics,
by the definitions of the element-wise functions, transposes and views, and by
the int32 element type's semantics, each value written by hand."""
import pytest

import golden_cases
import oracle


def test_every_file_has_cases_with_citations():
    cases = golden_cases.load_all()
    assert len({c.source for c in cases}) >= 4
    for c in cases:
        assert c.cite.startswith("Sec. "), c.name
        assert c.dtypes and c.prog and c.expect is not None, c.name


@pytest.mark.parametrize("case,dtype", golden_cases.params())
def test_oracle_matches_golden(orc, case, dtype):
    leaves = [golden_cases.host_leaf(l, dtype) for l in case.leaves]
    res = oracle.evaluate(case.prog, leaves, dtype)
    golden_cases.check(res.value, case, dtype, "%s/%s" % (case.name, dtype))


def test_a_planted_mistake_fails():
    # the comparison itself must reject a wrong value, a wrong position and a
    # NaN where a number is expected
    case = [c for c in golden_cases.load_all() if c.name == "fig1_axpy"][0]
    wrong = [float(v) for v in case.expect[2]]
    wrong[3] += 1.0
    with pytest.raises(AssertionError):
        golden_cases.check(wrong, case, "f32")
    exp1 = [c for c in golden_cases.load_all() if c.name == "exp_of_one"][0]
    with pytest.raises(AssertionError):
        golden_cases.check([2.7182818284590452 * (1 + 2e-6)], exp1, "f32")
    with pytest.raises(AssertionError):
        golden_cases.check([float("nan")], exp1, "f32")
