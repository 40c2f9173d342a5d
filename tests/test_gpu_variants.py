"""Every kernel variant (vector width x unroll) of the chunk walk (`coot_str_*`)
with a full reduction, on trees that cannot be walked as one long column
(submatrix views, broadcasts, diagonals, unaligned strided leaves), each
forced in turn (COOT_FORCE_KERNEL) and checked against the oracle, with and
without the materialised result, on ragged shapes that span several blocks."""
import pytest
import torch

import parity

pytestmark = pytest.mark.gpu

R, C = 1000, 37


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _variants(dtype, two_pass):
    v = 16 // {"f32": 4, "f64": 8, "bf16": 2, "i32": 4}[dtype]
    p = "_p1" if two_pass else ""
    return ["coot_str%s_v%du1" % (p, v), "coot_str%s_v%du2" % (p, v), "coot_str%s_v%du4" % (p, v),
            "coot_str%s_v1u4" % p]


def _leaves(dtype, seed, R=R, C=C, square=True):
    # column stride R + 16: 16-byte aligned columns for every dtype
    big = [parity.rand(R + 16, C + 5, dtype, seed=seed + i, kind="positive") for i in range(2)]
    A = big[0][8:8 + R, 2:2 + C]            # a view with 16-byte aligned columns
    B = big[1][1:1 + R, 4:4 + C]            # unaligned start: scalar variants only
    col = parity.rand(R, 1, dtype, seed=seed + 7, kind="positive")
    row = parity.rand(1, C, dtype, seed=seed + 8, kind="positive")
    sq = parity.rand(R + 1, (R if square else C) + 1, dtype, seed=seed + 9, kind="positive")
    return [A, B, col, row, sq]


TREES = [
    ("A B % {red}", False),
    ("A C each_col:37 % D each_row:1000 + {red}", False),
    ("A C each_col:37 % {red}", False),
    ("A abs sqrt B - {red}", False),
    ("E submat:1:1:1000:37 A + {red}", False),
    ("E diag:1 C - {red}", False),
    ("A B % {red}", True),
    ("A C each_col:37 - {red}", True),
]
REDS = ["accu", "min", "index_max", "prod", "var", "norm:fro"]


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "i32"])
@pytest.mark.parametrize("red", REDS)
def test_every_full_reduction_variant_matches_oracle(dtype, red, monkeypatch):
    if dtype == "i32" and red in ("var", "norm:fro"):
        pytest.skip("not defined for INT32 trees")
    leaves = _leaves(dtype, 11)
    trees = TREES
    if red == "prod" and dtype != "i32":
        # ratios' eighth roots: a product of 37,000 factors that stays in range
        trees = [("A B / sqrt sqrt sqrt {red}", False), ("A C each_col:37 / sqrt sqrt sqrt {red}", True)]
    for tree, materialise in trees:
        prog = tree.format(red=red)
        if dtype == "i32" and ("sqrt" in prog):
            continue
        for kname in _variants(dtype, red == "var"):
            monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
            parity.check(prog, leaves, dtype, materialise=materialise)
    monkeypatch.delenv("COOT_FORCE_KERNEL")


def test_forced_variant_is_the_one_launched(monkeypatch):
    import paper_2508_11385_gb300 as coot

    leaves = _leaves("f32", 3)
    for kname in _variants("f32", False):
        monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
        parity.check("A C each_col:37 % accu", leaves, "f32")
        torch.cuda.synchronize()
        assert coot.last_launch()["kernel"] == kname


# columns long enough that most units of the walk lie inside one column with
# every row inside the tree (the walk's check-free form), and a ragged last
# chunk per column (the checked form)
RL, CL = 20011, 6
TREES_LONG = [
    ("A B % {red}", False),
    ("A C each_col:6 % D each_row:20011 + {red}", False),
    ("A C each_col:6 - {red}", True),
    ("E submat:1:1:20011:6 A + {red}", False),
]


@pytest.mark.parametrize("dtype", ["f32", "bf16", "i32"])
@pytest.mark.parametrize("red", ["accu", "min", "index_max", "var"])
def test_every_variant_on_long_columns(dtype, red, monkeypatch):
    if dtype == "i32" and red == "var":
        pytest.skip("not defined for INT32 trees")
    leaves = _leaves(dtype, 31, RL, CL, square=False)
    for tree, materialise in TREES_LONG:
        prog = tree.format(red=red)
        for kname in _variants(dtype, red == "var"):
            monkeypatch.setenv("COOT_FORCE_KERNEL", kname)
            parity.check(prog, leaves, dtype, materialise=materialise)
    monkeypatch.delenv("COOT_FORCE_KERNEL")
