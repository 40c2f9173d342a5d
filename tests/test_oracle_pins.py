"""Pins of the FP64 CPU oracle against things other than itself.

Closed forms, exact rational brute force (fractions.Fraction), math.fsum
(correctly rounded sums), the platform libm, NumPy's two-pass variance and
spacing, NumPy int32 wrap-around arithmetic, and an emulated FP32 device whose
every node is correctly rounded.  Each check is chosen so that a plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand, a wrong normalisation) fails at least one of them.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

import rpn
from paper_2508_11385_gb300 import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def F(a):
    """column-major host copy"""
    return np.asfortranarray(a)


def bits(a, dtype):
    """storage-format host array for the oracle (BF16/FP16 as uint16 bits)"""
    t = torch.as_tensor(np.asarray(a, dtype=np.float64)).to(workloads.TORCH_DTYPE[dtype])
    if dtype in ("bf16", "f16"):
        return F(t.view(torch.int16).numpy().view(np.uint16))
    return F(t.numpy())


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16", "f16", "i32"])
@pytest.mark.parametrize("m,n", [(1, 1), (3, 7), (64, 33)])
def test_accu_of_ones_is_element_count(orc, dtype, m, n):
    r = orc.evaluate("A accu", [bits(np.ones((m, n)), dtype)], dtype)
    assert r.is_reduction and r.value.shape == (1, 1)
    assert r.value[0, 0] == m * n


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
def test_square_of_a_minus_a_is_zero(orc, dtype):
    rng = np.random.default_rng(1)
    a = rng.integers(-1000, 1000, size=(9, 5)) if dtype == "i32" else rng.normal(size=(9, 5))
    r = orc.evaluate("A A - square", [bits(a, dtype)], dtype)
    assert np.all(r.value == 0)
    if r.bound is not None:
        # exact zero leaves a bound of nothing but the local allowance at 0
        assert np.all(r.bound <= 3 * orc.ulp(0.0, "f32"))


def test_trans_is_index_swap_and_involution(orc):
    m, n = 5, 3
    a = np.array([[i + 100 * j for j in range(n)] for i in range(m)], dtype=np.float64)
    t = orc.evaluate("A trans", [F(a)], "f64").value
    assert t.shape == (n, m)
    for i in range(m):
        for j in range(n):
            assert t[j, i] == a[i, j]
    tt = orc.evaluate("A trans trans", [F(a)], "f64").value
    assert np.array_equal(tt, a)


def test_submat_of_index_encoded_matrix(orc):
    m, n = 11, 9
    a = np.array([[i + 1e4 * j for j in range(n)] for i in range(m)], dtype=np.float64)
    v = orc.evaluate("A submat:2:3:4:5", [F(a)], "f64").value
    assert v.shape == (4, 5)
    for i in range(4):
        for j in range(5):
            assert v[i, j] == (2 + i) + 1e4 * (3 + j)
    r = orc.evaluate("A submat:2:3:4:5 accu", [F(np.ones((m, n)))], "f64")
    assert r.value[0, 0] == 20


def test_submat_with_leading_dimension(orc):
    # the same view read from a matrix stored with ld > n_rows
    big = np.array([[i + 1e4 * j for j in range(8)] for i in range(12)], dtype=np.float64, order="F")
    view = big[:10, :]  # ld = 12
    v = orc.evaluate("A submat:1:2:3:4", [view], "f64").value
    assert v[0, 0] == 1 + 2e4 and v[2, 3] == 3 + 5e4


@pytest.mark.parametrize("n", [2, 3, 10, 1001])
@pytest.mark.parametrize("a0,d", [(3.0, 0.5), (-2.0, 0.25), (0.0, 1.0)])
def test_var_of_arithmetic_sequence(orc, n, a0, d):
    x = (a0 + d * np.arange(n, dtype=np.float64)).reshape(-1, 1)
    v0 = orc.evaluate("A var", [F(x)], "f64").value[0, 0]
    assert v0 == pytest.approx(d * d * n * (n + 1) / 12.0, rel=1e-15)
    v1 = orc.evaluate("A var:1", [F(x)], "f64").value[0, 0]
    assert v1 == pytest.approx(d * d * (n * n - 1) / 12.0, rel=1e-15)


def test_var_single_element_is_zero(orc):
    assert orc.evaluate("A var", [F(np.array([[7.5]]))], "f64").value[0, 0] == 0.0


def test_sum_along_dims_of_ones(orc):
    m, n = 6, 4
    s0 = orc.evaluate("A sum:0", [bits(np.ones((m, n)), "f32")], "f32").value
    s1 = orc.evaluate("A sum:1", [bits(np.ones((m, n)), "f32")], "f32").value
    assert s0.shape == (1, n) and np.all(s0 == m)
    assert s1.shape == (m, 1) and np.all(s1 == n)


def test_sum_along_dims_index_encoded(orc):
    m, n = 5, 3
    a = np.array([[i + 10 * j for j in range(n)] for i in range(m)], dtype=np.float64)
    s0 = orc.evaluate("A sum:0", [F(a)], "f64").value[0]
    s1 = orc.evaluate("A sum:1", [F(a)], "f64").value[:, 0]
    assert list(s0) == [sum(i + 10 * j for i in range(m)) for j in range(n)]
    assert list(s1) == [sum(i + 10 * j for j in range(n)) for i in range(m)]
    m0 = orc.evaluate("A mean:0", [F(a)], "f64").value[0]
    m1 = orc.evaluate("A mean:1", [F(a)], "f64").value[:, 0]
    assert np.allclose(m0, s0 / m, rtol=0, atol=0)
    assert np.allclose(m1, s1 / n, rtol=0, atol=0)


@pytest.mark.parametrize("n", [1, 4, 9, 1000])
def test_norm_of_ones(orc, n):
    r = orc.evaluate("A norm", [bits(np.ones((n, 1)), "f32")], "f32").value[0, 0]
    assert r == math.sqrt(n)
    r = orc.evaluate("A norm:fro", [bits(np.ones((n, 3)), "f32")], "f32").value[0, 0]
    assert r == math.sqrt(3 * n)


def test_dot_with_ones_is_accu(orc):
    rng = np.random.default_rng(5)
    v = rng.normal(size=(257, 1))
    d = orc.evaluate("A B dot", [F(np.ones((257, 1))), F(v)], "f64").value[0, 0]
    a = orc.evaluate("B accu", [F(np.ones((257, 1))), F(v)], "f64").value[0, 0]
    assert d == a


def test_int_sum_one_to_n(orc):
    n = 100000
    x = np.arange(1, n + 1, dtype=np.int32).reshape(-1, 1)
    assert orc.evaluate("A accu", [F(x)], "i32").value[0, 0] == n * (n + 1) // 2


@pytest.mark.parametrize("k", [0.5, -3.25, 7.0])
def test_mean_of_constant(orc, k):
    assert orc.evaluate("A mean", [F(np.full((13, 7), k))], "f64").value[0, 0] == k


def test_empty_reductions(orc):
    e = np.zeros((0, 3))
    assert orc.evaluate("A accu", [F(e)], "f64").value[0, 0] == 0.0
    assert math.isnan(orc.evaluate("A mean", [F(e)], "f64").value[0, 0])
    s0 = orc.evaluate("A sum:0", [F(e)], "f64").value
    assert s0.shape == (1, 3) and np.all(s0 == 0)


# ------------------------------------------------------- exact brute force

def _dyadic(rng, shape, lo=-8, hi=8):
    # small dyadic rationals: exact in every float type used here
    return rng.integers(lo * 16, hi * 16 + 1, size=shape) / 16.0


@pytest.mark.parametrize("seed", range(40))
def test_random_tree_against_exact_rationals(orc, seed):
    rng = random.Random(seed)
    nrng = np.random.default_rng(seed)
    m, n = rng.randint(1, 7), rng.randint(1, 5)
    leaves = [_dyadic(nrng, (m, n)) for _ in range(3)]
    prog = rpn.random_tree(rng, n_leaves=3, depth=rng.randint(1, 4))
    exact = rpn.eval_exact(prog, leaves)
    r = orc.evaluate(prog, [F(x) for x in leaves], "f64")
    for i in range(m):
        for j in range(n):
            e = exact[i][j]
            v = r.value[i, j]
            if e is None:  # a division by zero somewhere in the exact walk
                continue
            ef = float(e)
            if not math.isfinite(v):
                continue
            # the oracle's bound for an FP64 tree covers its own rounding
            assert abs(v - ef) <= r.bound[i, j] + 2 * math.ulp(ef), (prog, i, j, v, ef)


@pytest.mark.parametrize("op", ["+", "-", "%", "/"])
def test_single_binary_op_is_correctly_rounded(orc, op):
    nrng = np.random.default_rng(7)
    a = nrng.normal(size=(6, 4))
    b = nrng.normal(size=(6, 4)) + 3.0
    r = orc.evaluate("A B %s" % op, [F(a), F(b)], "f64").value
    ex = rpn.eval_exact("A B %s" % op, [a, b])
    for i in range(6):
        for j in range(4):
            assert r[i, j] == float(ex[i][j])


@pytest.mark.parametrize("form,expect", [
    ("#2.5 A *", lambda a: 2.5 * a), ("A #2.5 +", lambda a: a + 2.5),
    ("#2.5 A +", lambda a: 2.5 + a), ("A #2.5 -", lambda a: a - 2.5),
    ("#2.5 A -", lambda a: 2.5 - a), ("A #2.5 /", lambda a: a / 2.5),
    ("#2.5 A /", lambda a: 2.5 / a), ("A neg", lambda a: -a),
])
def test_scalar_forms_orientation(orc, form, expect):
    a = F(np.array([[1.0, -3.0], [0.5, 8.0]]))
    r = orc.evaluate(form, [a], "f64").value
    assert np.array_equal(r, expect(np.asarray(a)))


def test_scalar_is_converted_to_element_type(orc):
    a = F(np.ones((2, 2), dtype=np.float32))
    r = orc.evaluate("#0.1 A *", [a], "f32").value
    assert r[0, 0] == float(np.float32(0.1))
    r = orc.evaluate("#0.1 A *", [F(np.ones((2, 2)))], "f64").value
    assert r[0, 0] == 0.1
    r = orc.evaluate("#2.9 A *", [F(np.full((2, 2), 3, dtype=np.int32))], "i32").value
    assert r[0, 0] == 6  # 2.9 -> 2


@pytest.mark.parametrize("red", ["accu", "sum:0", "sum:1", "mean", "mean:0", "mean:1"])
def test_reductions_against_exact_rationals(orc, red):
    nrng = np.random.default_rng(11)
    a = _dyadic(nrng, (7, 5)) * (2.0 ** nrng.integers(-30, 30, size=(7, 5)))
    ex = rpn.eval_exact("A " + red, [a])
    r = orc.evaluate("A " + red, [F(a)], "f64").value
    if not isinstance(ex, list):
        ex = [[ex]]
    for i, row in enumerate(ex):
        for j, e in enumerate(row):
            assert abs(r[i, j] - float(e)) <= 2 * math.ulp(float(e)) + 1e-300


def test_dot_against_exact_rationals(orc):
    nrng = np.random.default_rng(12)
    a = _dyadic(nrng, (40, 1))
    b = _dyadic(nrng, (40, 1))
    ex = rpn.eval_exact("A B dot", [a, b])
    assert orc.evaluate("A B dot", [F(a), F(b)], "f64").value[0, 0] == float(ex)


# ------------------------------------------------------- library pins

def test_neumaier_sum_matches_fsum(orc):
    g = workloads.generator(99)
    x = workloads.signed_lognormal(200000, "f64", g).numpy().ravel()
    s = orc.sum_neumaier(x)
    f = math.fsum(x)
    assert abs(s - f) <= math.ulp(f)
    r = orc.evaluate("A accu", [F(x.reshape(-1, 1))], "f64").value[0, 0]
    assert abs(r - f) <= math.ulp(f)


def test_neumaier_beats_plain_sum_on_cancellation(orc):
    x = np.array([1.0, 1e100, 1.0, -1e100] * 1000)
    assert orc.sum_neumaier(x) == 2000.0


@pytest.mark.parametrize("fn", ["exp", "log", "sqrt"])
def test_transcendentals_match_libm(orc, fn):
    nrng = np.random.default_rng(3)
    a = np.abs(nrng.normal(size=(50, 3))) * 5 + 1e-3
    r = orc.evaluate("A " + fn, [F(a)], "f64").value
    f = getattr(math, fn)
    for idx, v in np.ndenumerate(a):
        assert r[idx] == f(v)
    ref = getattr(np, fn)(a)
    assert np.all(np.abs(r - ref) <= 2 * np.spacing(np.abs(ref)))


@pytest.mark.parametrize("ddof,tok", [(1, "var"), (0, "var:1")])
def test_var_matches_numpy(orc, ddof, tok):
    g = workloads.generator(17)
    x = workloads.signed_lognormal(100001, "f64", g).numpy()
    v = orc.evaluate("A " + tok, [F(x)], "f64").value[0, 0]
    assert v == pytest.approx(np.var(x.ravel(), ddof=ddof), rel=1e-13)


def test_norm_matches_numpy(orc):
    nrng = np.random.default_rng(8)
    x = nrng.normal(size=(1000, 1))
    assert orc.evaluate("A norm", [F(x)], "f64").value[0, 0] == pytest.approx(np.linalg.norm(x), rel=1e-15)
    X = nrng.normal(size=(30, 40))
    assert orc.evaluate("A norm:fro", [F(X)], "f64").value[0, 0] == pytest.approx(
        np.linalg.norm(X, "fro"), rel=1e-15)


@pytest.mark.parametrize("dtype,npt", [("f32", np.float32), ("f64", np.float64), ("f16", np.float16)])
def test_ulp_matches_numpy_spacing(orc, dtype, npt):
    vals = [1.0, 1.5, 2.0, 3.0e-5, 1e-40, 6.1e-5, 60000.0, 123456.789, 1e-300, 0.0, 2.0 ** -126]
    for v in vals:
        x = npt(v)
        if not np.isfinite(x):
            continue
        assert orc.ulp(float(x), dtype) == float(np.spacing(np.abs(x))) or (
            x == 0 and orc.ulp(0.0, dtype) == float(np.spacing(npt(0))))


def test_ulp_bf16(orc):
    # bf16 keeps 8 significant bits: spacing at 1.0 is 2^-7
    assert orc.ulp(1.0, "bf16") == 2.0 ** -7
    assert orc.ulp(3.0, "bf16") == 2.0 ** -6
    assert orc.ulp(0.0, "bf16") == 2.0 ** -133


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_half_storage_decoding_matches_torch(orc, dtype):
    g = workloads.generator(21)
    t = workloads.signed_lognormal(5000, dtype, g)
    host = workloads.to_numpy_colmajor(t)
    r = orc.evaluate("A", [host], dtype).value.ravel()
    assert np.array_equal(r, t.to(torch.float64).numpy().ravel())


# ------------------------------------------------------------ INT32 trees

def test_int32_wraps_like_numpy(orc):
    nrng = np.random.default_rng(4)
    a = nrng.integers(-2 ** 31, 2 ** 31, size=(20, 3), dtype=np.int64).astype(np.int32)
    b = nrng.integers(-2 ** 31, 2 ** 31, size=(20, 3), dtype=np.int64).astype(np.int32)
    with np.errstate(over="ignore"):
        for prog, ref in [("A B +", a + b), ("A B -", a - b), ("A B %", a * b),
                          ("A square", a * a), ("A neg", -a), ("A abs", np.abs(a)),
                          ("#3 A * B +", np.int32(3) * a + b)]:
            assert np.array_equal(orc.evaluate(prog, [F(a), F(b)], "i32").value, ref.astype(np.int64)), prog


def test_int32_abs_and_neg_of_min(orc):
    a = F(np.array([[-2 ** 31, 5]], dtype=np.int32))
    assert orc.evaluate("A abs", [a], "i32").value[0, 0] == -2 ** 31
    assert orc.evaluate("A neg", [a], "i32").value[0, 0] == -2 ** 31


def test_int32_division_truncates_and_flags_zero(orc):
    a = F(np.array([[-7, 7, -2 ** 31, 5]], dtype=np.int32))
    b = F(np.array([[2, -2, -1, 0]], dtype=np.int32))
    r = orc.evaluate("A B /", [a, b], "i32")
    assert list(r.value[0]) == [-3, -3, -2 ** 31, 0]
    assert r.div_by_zero
    r = orc.evaluate("A #2 /", [a], "i32")
    assert not r.div_by_zero and list(r.value[0]) == [-3, 3, -2 ** 30, 2]


def test_int32_reductions_are_exact_int64(orc):
    a = np.full((1000, 3), 2 ** 31 - 1, dtype=np.int32)
    assert orc.evaluate("A accu", [F(a)], "i32").value[0, 0] == 3000 * (2 ** 31 - 1)
    s = orc.evaluate("A A % accu", [F(a)], "i32").value[0, 0]  # products wrap to int32 first
    assert s == 3000 * 1
    d = orc.evaluate("A A dot", [F(a)], "i32").value[0, 0]  # dot multiplies exactly
    exact = 3000 * (2 ** 31 - 1) ** 2  # beyond int64: the int64 sum wraps modulo 2^64
    assert d == ((exact + 2 ** 63) % 2 ** 64) - 2 ** 63
    b = np.full((1000, 3), 46340, dtype=np.int32)
    assert orc.evaluate("A A dot", [F(b)], "i32").value[0, 0] == 3000 * 46340 ** 2
    s0 = orc.evaluate("A sum:0", [F(a)], "i32").value
    assert np.all(s0 == 1000 * (2 ** 31 - 1))


def test_int32_rejects_transcendentals_and_float_stats(orc):
    a = F(np.ones((2, 2), dtype=np.int32))
    for prog in ("A exp", "A log", "A sqrt", "A mean", "A var", "A norm:fro"):
        with pytest.raises(orc.OracleError):
            orc.evaluate(prog, [a], "i32")


# ------------------------------------------------------------ error model

@pytest.mark.parametrize("prog,c_dev,c_orc", [("A B +", 2, 1), ("A B /", 2, 1), ("A exp", 4, 2),
                                             ("A log", 4, 2), ("A sqrt", 4, 1), ("A square", 2, 1)])
def test_single_op_bound_is_the_per_op_allowance(orc, prog, c_dev, c_orc):
    nrng = np.random.default_rng(2)
    a = (np.abs(nrng.normal(size=(9, 4))) + 0.1).astype(np.float32)
    b = (np.abs(nrng.normal(size=(9, 4))) + 0.1).astype(np.float32)
    r = orc.evaluate(prog, [F(a), F(b)], "f32")
    for idx, v in np.ndenumerate(r.value):
        assert r.bound[idx] == c_dev * orc.ulp(v, "f32") + c_orc * orc.ulp(v, "f64")


@pytest.mark.parametrize("seed", range(60))
def test_bound_covers_an_emulated_fp32_device(orc, seed):
    """Evaluate random trees with every node rounded to FP32 (IEEE + - * / sqrt,
    correctly rounded exp/log): the FP64 oracle's bound must cover the error."""
    rng = random.Random(1000 + seed)
    nrng = np.random.default_rng(1000 + seed)
    leaves = [(nrng.uniform(0.2, 2.0, size=(8, 6)) * nrng.choice([-1, 1], size=(8, 6))).astype(np.float32)
              for _ in range(3)]
    prog = rpn.random_tree(rng, n_leaves=3, depth=rng.randint(1, 5),
                           ops_un=rpn.UN_ARITH + ["exp", "sqrt", "log"])
    # keep sqrt/log in their domain: apply them to abs(...) + 1 only
    toks = []
    for t in prog.split():
        if t in ("sqrt", "log"):
            toks += ["abs", "#1.0", "+", t]
        elif t == "exp":
            toks += ["#0.25", "*", t]
        else:
            toks.append(t)
    prog = " ".join(toks)
    dev = rpn.eval_emulated(prog, leaves, np.float32)
    r = orc.evaluate(prog, [F(x) for x in leaves], "f32")
    fin = np.isfinite(r.value)
    err = np.abs(dev.astype(np.float64) - r.value)
    assert np.all(err[fin] <= r.bound[fin]), prog


@pytest.mark.parametrize("prog", ["A B + exp", "A B - #3 * exp", "A B % #0.1 * exp",
                                  "A B + C / #4 * exp", "A B + log", "A #10 - B #10 - / #0.01 * exp"])
def test_bound_propagates_through_amplifying_ops(orc, prog):
    """Arguments of magnitude ~10-20 carry rounding errors that exp (and a
    division by a small difference) amplify well past the per-op allowance of
    the last node: only the propagated child bound covers them."""
    nrng = np.random.default_rng(31)
    leaves = [nrng.uniform(6.0, 11.0, size=(64, 16)).astype(np.float32) for _ in range(3)]
    dev = rpn.eval_emulated(prog, leaves, np.float32)
    r = orc.evaluate(prog, [F(x) for x in leaves], "f32")
    fin = np.isfinite(r.value)
    assert np.array_equal(dev[~fin].astype(np.float64), r.value[~fin])
    err = np.abs(dev.astype(np.float64) - r.value)
    assert np.all(err[fin] <= r.bound[fin]), prog
    # the amplification is real: some errors exceed the last node's own allowance
    if prog in ("A B + exp", "A B - #3 * exp"):
        own = np.array([4 * orc.ulp(v, "f32") for v in r.value.ravel()]).reshape(r.value.shape)
        assert np.any(err > own)


def test_bound_covers_bf16_output_rounding(orc):
    nrng = np.random.default_rng(9)
    a = bits(nrng.normal(size=(16, 4)), "bf16")
    b = bits(nrng.normal(size=(16, 4)), "bf16")
    r = orc.evaluate("A B +", [a, b], "bf16")
    ta = torch.from_numpy(a.view(np.int16).copy()).view(torch.bfloat16).float()
    tb = torch.from_numpy(b.view(np.int16).copy()).view(torch.bfloat16).float()
    dev = (ta + tb).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.all(np.abs(dev - r.value) <= r.bound)


def test_compute_type_overflow_is_inf(orc):
    a = F(np.array([[3.0e38, -3.0e38, 1.0]], dtype=np.float32))
    r = orc.evaluate("#2 A *", [a], "f32")
    assert r.value[0, 0] == np.inf and r.value[0, 1] == -np.inf and r.value[0, 2] == 2.0
    r = orc.evaluate("#2 A *", [F(np.array([[3.0e38]]))], "f64")
    assert r.value[0, 0] == 6.0e38  # FP64 trees keep the FP64 range
    h = bits(np.array([[60000.0, 1.0]]), "f16")
    r = orc.evaluate("#2 A *", [h], "f16")
    assert r.value[0, 0] == np.inf and r.value[0, 1] == 2.0  # FP32 compute, FP16 storage overflow
    ref = (torch.tensor([60000.0, 1.0], dtype=torch.float16).float() * 2).to(torch.float16)
    assert ref[0].item() == float("inf")


# ------------------------------------------------------------ malformed input

@pytest.mark.parametrize("prog", ["A B *", "A B +", "A +", "A accu B", "A Z", "A submat:0:0:9:9",
                                  "A norm", "#1 #2 +"])
def test_malformed_programs_are_rejected(orc, prog):
    with pytest.raises(orc.OracleError):
        orc.evaluate(prog, [F(np.ones((3, 2))), F(np.ones((2, 3)))], "f64")


# ------------------------------------------------------------ gradients

def test_grad_matches_closed_form_of_the_differentiation_loss(orc):
    """L = accu(square(W%X - Y)) + 1e-3 accu(square(W)):
    dL/dW = 2 (W%X - Y) % X + 2e-3 W,  dL/dX = 2 (W%X - Y) % W."""
    nrng = np.random.default_rng(6)
    W, X, Y = (nrng.normal(size=(64, 64)) for _ in range(3))
    prog = "A B % C - square #0.001 A square * + accu"
    loss, (gW, gX, gY), _ = orc.grad(prog, [F(W), F(X), F(Y)], "f64")
    R = W * X - Y
    assert loss == pytest.approx(np.sum(R * R) + 1e-3 * np.sum(W * W), rel=1e-13)
    assert np.allclose(gW, 2 * R * X + 2e-3 * W, rtol=1e-13, atol=1e-13)
    assert np.allclose(gX, 2 * R * W, rtol=1e-13, atol=1e-13)
    assert np.allclose(gY, -2 * R, rtol=1e-13, atol=1e-13)


def test_grad_matches_central_differences_on_a_64x64_slice(orc):
    """Central finite differences in FP64 of the oracle's own forward
    evaluation; L is quadratic in each of W and X, so the central difference
    is exact up to rounding."""
    nrng = np.random.default_rng(60)
    W, X, Y = (nrng.normal(size=(64, 64)) for _ in range(3))
    prog = "A B % C - square #0.001 A square * + accu"
    _, (gW, gX, _), _ = orc.grad(prog, [F(W), F(X), F(Y)], "f64")
    h = 1e-3
    for which, G in ((0, gW), (1, gX)):
        for idx in [(i, j) for i in range(0, 64, 3) for j in range(0, 64, 5)]:
            lv = [W.copy(), X.copy(), Y.copy()]
            lv[which][idx] += h
            up = orc.evaluate(prog, [F(x) for x in lv], "f64").value[0, 0]
            lv[which][idx] -= 2 * h
            dn = orc.evaluate(prog, [F(x) for x in lv], "f64").value[0, 0]
            fd = (up - dn) / (2 * h)
            assert abs(fd - G[idx]) <= 1e-7 * max(1.0, abs(G[idx])), (which, idx, fd, G[idx])


@pytest.mark.parametrize("seed", range(12))
def test_grad_of_random_trees_matches_finite_differences(orc, seed):
    rng = random.Random(500 + seed)
    nrng = np.random.default_rng(500 + seed)
    leaves = [nrng.uniform(0.5, 2.0, size=(5, 4)) for _ in range(3)]
    prog = rpn.random_tree(rng, n_leaves=3, depth=rng.randint(1, 4), ops_un=["neg", "square", "exp", "sqrt", "log"])
    if rng.random() < 0.3:
        prog = prog + " trans"
    prog = prog + (" mean" if seed % 2 else " accu")
    try:
        loss, gs, ags = orc.grad(prog, [F(x) for x in leaves], "f64")
    except orc.OracleError:
        pytest.skip("tree with a scalar root")
    if not np.isfinite(loss):
        pytest.skip("non-finite loss")
    h = 1e-6
    for li in range(3):
        for idx in [(0, 0), (4, 3), (2, 1)]:
            lv = [x.copy() for x in leaves]
            lv[li][idx] += h
            up = orc.evaluate(prog, [F(x) for x in lv], "f64").value[0, 0]
            lv[li][idx] -= 2 * h
            dn = orc.evaluate(prog, [F(x) for x in lv], "f64").value[0, 0]
            fd = (up - dn) / (2 * h)
            assert abs(fd - gs[li][idx]) <= 1e-5 * max(1.0, abs(gs[li][idx]), ags[li][idx]), (prog, li, idx)
            assert ags[li][idx] >= abs(gs[li][idx]) * (1 - 1e-12)


def test_grad_through_trans_and_submat(orc):
    nrng = np.random.default_rng(3)
    A = nrng.normal(size=(6, 9))
    B = nrng.normal(size=(4, 5))
    # accu(trans(A.submat(1,2,5,4)) % B): dL/dA is B^T scattered into the view
    _, (gA, gB), _ = orc.grad("A submat:1:2:5:4 trans B % accu", [F(A), F(B)], "f64")
    expect = np.zeros_like(A)
    expect[1:6, 2:6] = B.T
    assert np.array_equal(gA, expect)
    assert np.array_equal(gB, A[1:6, 2:6].T)


def test_grad_bound_covers_an_emulated_fp32_device(orc):
    """The device's reverse sweep for L = accu(square(W%X - Y)) + lam accu(square(W)),
    rounded to FP32 at every operation in the order the adjoint kernel uses,
    stays within 16 u times the oracle's magnitude sweep (including rows where
    W%X - Y cancels)."""
    nrng = np.random.default_rng(66)
    W, X = (nrng.normal(size=(128, 64)).astype(np.float32) for _ in range(2))
    Y = (W * X).astype(np.float32)  # exact cancellation ...
    Y[::2] = nrng.uniform(-1, 1, size=Y[::2].shape).astype(np.float32)  # ... on every other row
    f = np.float32
    lam = f(1e-3)
    r = (W * X).astype(f) - Y
    gW = (f(2) * r * X).astype(f) + ((lam + lam) * W).astype(f)
    gX = (f(2) * r * W).astype(f)
    prog = "A B % C - square #0.001 A square * + accu"
    _, (oW, oX, _), (aW, aX, _) = orc.grad(prog, [F(W), F(X), F(Y)], "f32")
    u = 2.0 ** -24
    assert np.all(np.abs(gW.astype(np.float64) - oW) <= 16 * u * aW)
    assert np.all(np.abs(gX.astype(np.float64) - oX) <= 16 * u * aX)
    # and the plain |terms| sweep would not have covered the cancelling rows
    plain = np.abs(2 * (W.astype(np.float64) * X - Y) * X) + 2e-3 * np.abs(W)
    assert np.any(np.abs(gW.astype(np.float64) - oW) > 16 * u * plain)


# ------------------------------------------------------------ statistics

@pytest.mark.parametrize("dtype", ["f64", "f32", "i32"])
def test_min_max_and_indices_of_a_permutation(orc, dtype):
    nrng = np.random.default_rng(70)
    m, n = 7, 9
    perm = nrng.permutation(m * n).astype(np.float64) - 20
    a = perm.reshape((m, n), order="F")
    h = bits(a, dtype)
    assert orc.evaluate("A min", [h], dtype).value[0, 0] == a.min()
    assert orc.evaluate("A max", [h], dtype).value[0, 0] == a.max()
    assert orc.evaluate("A index_min", [h], dtype).value[0, 0] == np.argmin(a.ravel(order="F"))
    assert orc.evaluate("A index_max", [h], dtype).value[0, 0] == np.argmax(a.ravel(order="F"))
    assert np.array_equal(orc.evaluate("A min:0", [h], dtype).value[0], a.min(axis=0))
    assert np.array_equal(orc.evaluate("A max:1", [h], dtype).value[:, 0], a.max(axis=1))
    assert np.array_equal(orc.evaluate("A index_min:0", [h], dtype).value[0], np.argmin(a, axis=0))
    assert np.array_equal(orc.evaluate("A index_max:1", [h], dtype).value[:, 0], np.argmax(a, axis=1))


def test_extremes_take_the_first_tie_and_pass_over_nan(orc):
    a = F(np.array([[2.0, np.nan, 1.0, 1.0, np.nan, 3.0, 3.0]]).T)
    assert orc.evaluate("A index_min", [a], "f64").value[0, 0] == 2
    assert orc.evaluate("A index_max", [a], "f64").value[0, 0] == 5
    assert orc.evaluate("A min", [a], "f64").value[0, 0] == 1.0
    nan = F(np.full((3, 1), np.nan))
    assert np.isnan(orc.evaluate("A max", [nan], "f64").value[0, 0])
    assert orc.evaluate("A index_max", [nan], "f64").value[0, 0] == -1
    e = F(np.zeros((0, 2)))
    assert np.array_equal(orc.evaluate("A index_min:0", [e], "f64").value[0], [-1, -1])


def test_prod_of_powers_of_two_is_exact(orc):
    k = np.array([3, -1, 5, 0, -7, 2, 1, -2])
    a = F((2.0 ** k).reshape(4, 2, order="F") * np.array([[1, -1]] * 4))
    assert orc.evaluate("A prod", [a], "f64").value[0, 0] == 2.0 ** k.sum() * 1.0  # 4 sign flips
    assert np.array_equal(orc.evaluate("A prod:0", [a], "f64").value[0], np.prod(a, axis=0))
    assert np.array_equal(orc.evaluate("A prod:1", [a], "f64").value[:, 0], np.prod(a, axis=1))


def test_prod_matches_numpy_and_is_compensated(orc):
    nrng = np.random.default_rng(71)
    x = nrng.uniform(0.9, 1.1, size=(200000, 1))
    p = orc.evaluate("A prod", [F(x)], "f64").value[0, 0]
    exact = math.fsum(np.log(x.ravel()))  # the product is exp(sum log x) to ~1e-16 relative
    assert p == pytest.approx(math.exp(exact), rel=1e-12)
    fr = Fraction(1)
    for v in x.ravel()[:300]:
        fr *= Fraction(float(v))
    assert orc.evaluate("A prod", [F(x[:300])], "f64").value[0, 0] == pytest.approx(float(fr), rel=1e-15)


def test_int_prod_wraps_modulo_2_64(orc):
    a = np.array([[2 ** 31 - 1], [2 ** 31 - 1], [7], [-3]], dtype=np.int32)
    exact = (2 ** 31 - 1) ** 2 * 7 * -3
    assert orc.evaluate("A prod", [F(a)], "i32").value[0, 0] == ((exact + 2 ** 63) % 2 ** 64) - 2 ** 63


@pytest.mark.parametrize("n", [2, 5, 1001])
def test_stddev_of_arithmetic_sequence(orc, n):
    d = 0.75
    x = (1.5 + d * np.arange(n, dtype=np.float64)).reshape(-1, 1)
    assert orc.evaluate("A stddev", [F(x)], "f64").value[0, 0] == pytest.approx(
        math.sqrt(d * d * n * (n + 1) / 12.0), rel=1e-15)
    assert orc.evaluate("A stddev:1", [F(x)], "f64").value[0, 0] == pytest.approx(
        math.sqrt(d * d * (n * n - 1) / 12.0), rel=1e-15)


@pytest.mark.parametrize("dim", [0, 1])
@pytest.mark.parametrize("nt", [0, 1])
def test_var_and_stddev_along_a_dimension_match_numpy(orc, dim, nt):
    nrng = np.random.default_rng(72)
    a = nrng.normal(size=(37, 23)) * 3 + 1
    v = orc.evaluate("A vardim:%d:%d" % (dim, nt), [F(a)], "f64").value.ravel()
    s = orc.evaluate("A stddevdim:%d:%d" % (dim, nt), [F(a)], "f64").value.ravel()
    assert np.allclose(v, np.var(a, axis=dim, ddof=1 - nt), rtol=1e-13, atol=0)
    assert np.allclose(s, np.std(a, axis=dim, ddof=1 - nt), rtol=1e-13, atol=0)


@pytest.mark.parametrize("tok", ["min", "max:0", "prod:1", "stddev", "vardim:0:0"])
def test_statistics_bounds_cover_an_emulated_fp32_device(orc, tok):
    nrng = np.random.default_rng(73)
    A = nrng.uniform(0.8, 1.2, size=(50, 20)).astype(np.float32)
    B = nrng.uniform(0.8, 1.2, size=(50, 20)).astype(np.float32)
    prog = "A B % #0.5 B * + exp"
    y = rpn.eval_emulated(prog, [A, B], np.float32).astype(np.float64)
    r = orc.evaluate(prog + " " + tok, [F(A), F(B)], "f32")
    if tok == "min":
        dev = np.array([[y.min()]])
    elif tok == "max:0":
        dev = y.max(axis=0)[None, :]
    elif tok == "prod:1":
        dev = np.prod(y, axis=1)[:, None]
    elif tok == "stddev":
        dev = np.array([[np.std(y, ddof=1)]])
    else:
        dev = np.var(y, axis=0, ddof=1)[None, :]
    assert np.all(np.abs(dev - r.value) <= 1e-6 * np.abs(r.value) + r.bound)


@pytest.mark.parametrize("dtype,lo,hi", [("f32", -140, 105), ("f64", -1060, 795)])
def test_prod_carries_the_exponent_apart(orc, dtype, lo, hi):
    # 30 subnormal factors 2^lo and 40 factors 2^hi: the exact product is 2^0;
    # every running product in the format's own range underflows first
    ft = np.float32 if dtype == "f32" else np.float64
    a = np.vstack([np.full((30, 1), 2.0 ** lo), np.full((40, 1), 2.0 ** hi)]).astype(ft)
    assert 30 * lo + 40 * hi == 0
    assert orc.evaluate("A prod", [F(a)], dtype).value[0, 0] == 1.0
    assert orc.evaluate("A prod:0", [F(a)], dtype).value[0, 0] == 1.0


def test_prod_follows_ieee_special_values_and_rounds_to_the_result_type(orc):
    f = lambda v: F(np.array(v, dtype=np.float32).reshape(-1, 1))
    assert np.isnan(orc.evaluate("A prod", [f([0.0, np.inf, 2.0])], "f32").value[0, 0])
    assert orc.evaluate("A prod", [f([np.inf, -2.0])], "f32").value[0, 0] == -np.inf
    z = orc.evaluate("A prod", [f([-0.0, 3.0, -5.0])], "f32").value[0, 0]
    assert z == 0.0 and not np.signbit(z)
    assert np.isnan(orc.evaluate("A prod", [f([np.nan, 0.0])], "f32").value[0, 0])
    # 1e30 * 1e30 exceeds FP32: an FP32 tree's product is +inf, FP64 keeps it
    assert orc.evaluate("A prod", [f([1e30, 1e30])], "f32").value[0, 0] == np.inf
    assert orc.evaluate("A prod", [F(np.array([[1e30], [1e30]]))], "f64").value[0, 0] == pytest.approx(1e60)
    # and is rounded once to float: 3 * (1 + 2^-23) * (1 + 2^-23)
    x = np.float32(1 + 2.0 ** -23)
    assert orc.evaluate("A prod", [f([3.0, x, x])], "f32").value[0, 0] == float(np.float32(3.0 * float(x) ** 2))


# ------------------------------------------------------------ cumsum

def test_cumsum_of_ones_counts(orc):
    a = F(np.ones((7, 3)))
    v = orc.evaluate("A cumsum", [a], "f64").value
    assert np.array_equal(v, np.tile(np.arange(1, 8, dtype=np.float64)[:, None], (1, 3)))
    v1 = orc.evaluate("A cumsum:1", [a], "f64").value
    assert np.array_equal(v1, np.tile(np.arange(1, 4, dtype=np.float64)[None, :], (7, 1)))


@pytest.mark.parametrize("dim", [0, 1])
def test_cumsum_of_integers_matches_numpy_exactly(orc, dim):
    g = np.random.default_rng(80)
    a = g.integers(-1000, 1000, size=(33, 17)).astype(np.float64)
    assert np.array_equal(orc.evaluate("A cumsum:%d" % dim, [F(a)], "f64").value, np.cumsum(a, axis=dim))
    b = a.astype(np.int32)
    assert np.array_equal(orc.evaluate("A cumsum:%d" % dim, [F(b)], "i32").value, np.cumsum(b, axis=dim))


def test_cumsum_default_runs_along_a_vector(orc):
    r = F(np.array([[1.0, 2.0, 3.0, 4.0]]))
    assert np.array_equal(orc.evaluate("A cumsum", [r], "f64").value, [[1.0, 3.0, 6.0, 10.0]])
    c = F(np.array([[1.0], [2.0], [3.0]]))
    assert np.array_equal(orc.evaluate("A cumsum", [c], "f64").value, [[1.0], [3.0], [6.0]])


def test_cumsum_prefixes_are_exactly_rounded(orc):
    g = np.random.default_rng(81)
    x = g.normal(size=(500, 1)) * np.exp(g.normal(size=(500, 1)) * 8)  # wide exponent range: cancellations
    v = orc.evaluate("A cumsum", [F(x)], "f64").value[:, 0]
    want = [math.fsum(x[:k + 1, 0]) for k in range(500)]
    assert np.array_equal(v, want)


def test_cumsum_int32_wraps(orc):
    x = np.array([[2 ** 31 - 1], [5], [-7], [-(2 ** 31)], [-3]], dtype=np.int32)
    with np.errstate(over="ignore"):
        want = np.cumsum(x, axis=0, dtype=np.int32)
    assert np.array_equal(orc.evaluate("A cumsum", [F(x)], "i32").value, want)


def test_cumsum_rows_are_cumsum_of_the_transpose(orc):
    g = np.random.default_rng(82)
    a = g.normal(size=(9, 14))
    v1 = orc.evaluate("A cumsum:1", [F(a)], "f64").value
    v0 = orc.evaluate("A trans cumsum:0", [F(a)], "f64").value
    assert np.array_equal(v1, v0.T)


@pytest.mark.parametrize("dim", [0, 1])
def test_cumsum_bound_covers_sequential_fp32(orc, dim):
    # numpy's float32 cumsum adds in order in FP32: the recursive summation
    # the bound (k-1) u sum|y| is written for
    g = np.random.default_rng(83)
    A = g.normal(size=(700, 40)).astype(np.float32)
    B = g.normal(size=(700, 40)).astype(np.float32)
    prog = "A B % A +"
    y = rpn.eval_emulated(prog, [A, B], np.float32)
    dev = np.cumsum(y, axis=dim, dtype=np.float32).astype(np.float64)
    r = orc.evaluate(prog + " cumsum:%d" % dim, [F(A), F(B)], "f32")
    assert np.all(np.abs(dev - r.value) <= r.bound)
    # a bare leaf: no element error, only the summation's
    dev = np.cumsum(A, axis=dim, dtype=np.float32).astype(np.float64)
    r = orc.evaluate("A cumsum:%d" % dim, [F(A)], "f32")
    assert np.all(np.abs(dev - r.value) <= r.bound)
    assert np.any(np.abs(dev - r.value) > 0)  # the order of additions shows


def test_cumsum_overflow_and_special_values(orc):
    f = lambda v: F(np.array(v, dtype=np.float32).reshape(-1, 1))
    # a prefix beyond the FP32 range is inf (prefixes after it are exact
    # values again, which a running sum cannot return: not compared on the GPU)
    v = orc.evaluate("A cumsum", [f([3e38, 3e38, -3e38])], "f32").value[:, 0]
    assert v[0] == np.float32(3e38) and v[1] == np.inf and v[2] == pytest.approx(3e38, rel=1e-7)
    w = orc.evaluate("A cumsum", [f([1.0, np.inf, 2.0, -np.inf, 5.0])], "f32").value[:, 0]
    assert w[0] == 1.0 and w[1] == np.inf and w[2] == np.inf and np.isnan(w[3]) and np.isnan(w[4])


# ------------------------------------------------------------ broadcasting and diagonals

@pytest.mark.parametrize("k", [0, 1, 3, -1, -4])
def test_diag_matches_numpy(orc, k):
    g = np.random.default_rng(90)
    a = g.normal(size=(6, 9))
    assert np.array_equal(orc.evaluate("A diag:%d" % k, [F(a)], "f64").value.ravel(), np.diag(a, k))
    assert np.array_equal(orc.evaluate("A trans diag:%d" % -k, [F(a)], "f64").value.ravel(), np.diag(a, k))


def test_diag_of_an_expression_is_the_expression_of_diagonals(orc):
    g = np.random.default_rng(91)
    a, b = g.normal(size=(7, 7)), g.normal(size=(7, 7))
    v = orc.evaluate("A B % #2 + diag", [F(a), F(b)], "f64").value.ravel()
    assert np.array_equal(v, np.diag(a) * np.diag(b) + 2)
    assert orc.evaluate("A diag accu", [F(np.eye(5) * 3)], "f64").value[0, 0] == 15.0  # trace


def test_each_col_and_each_row_repeat_the_vector(orc):
    g = np.random.default_rng(92)
    a = g.normal(size=(5, 4))
    v = g.normal(size=(5, 1))
    r = g.normal(size=(1, 4))
    assert np.array_equal(orc.evaluate("A B each_col:4 -", [F(a), F(v)], "f64").value, a - v)
    assert np.array_equal(orc.evaluate("A B each_row:5 /", [F(a), F(r)], "f64").value, a / r)
    # column sums of a repeated column are n times it; row sums of a repeated row likewise
    assert np.array_equal(orc.evaluate("B each_col:4 sum:1", [F(a), F(v)], "f64").value, 4 * v)
    assert np.array_equal(orc.evaluate("B each_row:5 sum:0", [F(a), F(r)], "f64").value, 5 * r)
    # each_row of r is each_col of trans(r), transposed
    w = orc.evaluate("B trans each_col:5 trans", [F(a), F(r)], "f64").value
    assert np.array_equal(w, orc.evaluate("B each_row:5", [F(a), F(r)], "f64").value)


def test_broadcast_keeps_bounds_and_int_values(orc):
    g = np.random.default_rng(93)
    v = g.integers(-100, 100, size=(6, 1)).astype(np.int32)
    a = g.integers(-100, 100, size=(6, 3)).astype(np.int32)
    assert np.array_equal(orc.evaluate("A B each_col:3 %", [F(a), F(v)], "i32").value, a * v)
    f = g.normal(size=(6, 1)).astype(np.float32)
    r = orc.evaluate("A exp each_col:3", [F(f)], "f32")
    assert np.all(r.bound[:, 0:1] == r.bound[:, 2:3]) and np.all(r.bound > 0)


# ------------------------------------------------------------ matrix product

def test_matmul_exact_cases(orc):
    g = np.random.default_rng(100)
    a = g.normal(size=(6, 9))
    eye = np.eye(9)
    assert np.array_equal(orc.evaluate("A B mm", [F(a), F(eye)], "f64").value, a)
    perm = np.eye(6)[g.permutation(6)]
    assert np.array_equal(orc.evaluate("B A mm", [F(a), F(perm)], "f64").value, perm @ a)
    # integer-valued operands: every product and sum exact
    x = g.integers(-50, 50, size=(7, 11)).astype(np.float64)
    y = g.integers(-50, 50, size=(11, 4)).astype(np.float64)
    assert np.array_equal(orc.evaluate("A B mm", [F(x), F(y)], "f64").value, x @ y)


def test_matmul_of_a_transpose_and_exact_rounding(orc):
    g = np.random.default_rng(101)
    x = g.normal(size=(40, 13))   # K x M
    y = g.normal(size=(40, 17))   # K x N
    v = orc.evaluate("A trans B mm", [F(x), F(y)], "f64").value
    exact = np.array([[float(sum(Fraction(float(x[t, i])) * Fraction(float(y[t, j])) for t in range(40)))
                       for j in range(17)] for i in range(13)])
    assert np.array_equal(v, exact)


@pytest.mark.parametrize("k", [1, 64, 700])
def test_matmul_bound_covers_fp32_accumulation(orc, k):
    # products of FP32 values rounded to FP32 and accumulated in FP32 stay
    # inside the bound: checked for sequential and pairwise orders
    g = np.random.default_rng(102 + k)
    x = g.normal(size=(8, k)).astype(np.float32)
    y = g.normal(size=(k, 5)).astype(np.float32)
    r = orc.evaluate("A B mm", [F(x), F(y)], "f32")
    p = x.astype(np.float64)[:, :, None] * y.astype(np.float64)[None, :, :]   # exact in double
    seq = np.zeros((8, 5), dtype=np.float32)
    for t in range(k):
        seq = (seq + p[:, t, :].astype(np.float32)).astype(np.float32)
    pw = p.astype(np.float32)
    while pw.shape[1] > 1:
        if pw.shape[1] % 2:
            pw = np.concatenate([pw, np.zeros((8, 1, 5), dtype=np.float32)], axis=1)
        pw = (pw[:, 0::2, :] + pw[:, 1::2, :]).astype(np.float32)
    for dev in (seq.astype(np.float64), pw[:, 0, :].astype(np.float64)):
        assert np.all(np.abs(dev - r.value) <= r.bound)
