"""Mistakes planted in a copy of the oracle (on the CPU) must fail its pins:
each mutation below is a plausible slip -- swapped operands, a wrong index, a
wrong normalisation, a sign error in the compensation, a dropped term of the
error bound -- and the pin suite run against the mutated build must fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("int minus operands", "case B_MINUS: return wrap32(a - b);", "case B_MINUS: return wrap32(b - a);"),
    ("fp minus operands", "      r = a - b;\n", "      r = b - a;\n"),
    ("trans index", "int64_t s = i + j * r, d = j + i * c;", "int64_t s = i + j * r, d = i + j * r;"),
    ("var normalisation", "double den = (kind == R_VAR0) ? (double)(n - 1) : (double)n;", "double den = (double)n;"),
    ("compensation sign", "c += (s - t) + x[i];", "c += (t - s) + x[i];"),
    ("submat offsets", "int64_t s = (r0 + i) + (c0 + j) * x->r, d = i + j * nr;",
     "int64_t s = (c0 + i) + (r0 + j) * x->r, d = i + j * nr;"),
    ("product bound term", "e = mulb(a, bb) + mulb(b, ba)", "e = mulb(a, bb)"),
    ("exp bound propagation", "bv = (ba == 0.0) ? 0.0 : v * expm1(ba);", "bv = 0.0;"),
    ("mean divisor", "        s = s / (double)len;", "        s = s / (double)nout;"),
    ("gradient of division", "case B_DIV: da = 1.0 / b; db = -a / (b * b);", "case B_DIV: da = 1.0 / b; db = a / (b * b);"),
    ("extreme keeps the last tie", "if (best < 0 || (want_min ? v < bv : v > bv)) {",
     "if (best < 0 || (want_min ? v <= bv : v >= bv)) {"),
    ("product exponent", "          E += k;\n          const double p = ph * m;", "          const double p = ph * m;"),
    ("cumsum default direction", "if (dim < 0) dim = (r == 1) ? 1 : 0;", "if (dim < 0) dim = (r == 1) ? 0 : 1;"),
    ("cumsum summation bound", "bsum + (double)t * u * asum + orc_ulp(v, ORC_F64)", "bsum + orc_ulp(v, ORC_F64)"),
    ("diag offset direction", "const int64_t kr = arg < 0 ? -arg : 0, kc = arg > 0 ? arg : 0;",
     "const int64_t kc = arg < 0 ? -arg : 0, kr = arg > 0 ? arg : 0;"),
    ("each_row shape", "    r = arg;\n    c = x->c;", "    r = x->c;\n    c = arg;"),
    ("matmul operand index", "const double a = x->v[i + t * m], b = y->v[t + j * k];",
     "const double a = x->v[t + i * k], b = y->v[t + j * k];"),
    ("matmul summation bound", "double b = bsum + (double)k * u * asum + orc_ulp(v, ORC_F64);",
     "double b = bsum + orc_ulp(v, ORC_F64);"),
    ("cumsum compensation", "const double e = (sh - (s2 - bp)) + (y - bp);", "const double e = 0.0;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_the_pins(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    work = tmp_path / "repo"
    (work / "oracle").mkdir(parents=True)
    for f in ("oracle.h", "__init__.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), work / "oracle" / f)
    (work / "oracle" / "oracle.c").write_text(src.replace(old, new))
    shutil.copytree(os.path.join(ROOT, "tests"), work / "tests",
                    ignore=shutil.ignore_patterns("__pycache__", "test_oracle_mutations.py", "test_gpu*", "test_abi.py",
                                                  "test_multiproc.py"))
    shutil.copytree(os.path.join(ROOT, "paper_2508_11385_gb300"), work / "paper_2508_11385_gb300",
                    ignore=shutil.ignore_patterns("__pycache__", "_build", "*.so", "csrc"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py"], cwd=work, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "the pins did not catch the planted mistake '%s'" % name
    assert "failed" in r.stdout


# mistakes whose effect on a value the hand-written worked cases in
# tests/golden/ fix (the others change only error bounds, gradients, or
# results of exact integer sums): those cases alone must catch them too
GOLDEN_CATCHES = ["trans index", "var normalisation", "submat offsets", "mean divisor", "extreme keeps the last tie",
                  "product exponent", "cumsum default direction", "diag offset direction", "each_row shape",
                  "matmul operand index"]


@pytest.mark.parametrize("name", GOLDEN_CATCHES)
def test_planted_mistake_fails_the_worked_cases(tmp_path, name):
    old, new = [(o, n) for m, o, n in MUTATIONS if m == name][0]
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    work = tmp_path / "repo"
    (work / "oracle").mkdir(parents=True)
    for f in ("oracle.h", "__init__.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), work / "oracle" / f)
    (work / "oracle" / "oracle.c").write_text(src.replace(old, new))
    (work / "tests").mkdir()
    for f in ("conftest.py", "golden_cases.py", "test_golden.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), work / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), work / "tests" / "golden")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "tests/test_golden.py"],
                       cwd=work, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "the worked cases did not catch the planted mistake '%s'" % name
    assert "failed" in r.stdout

