"""The oracle's OpenMP build (liborc_omp.so, element-wise loops on all host
cores, used for the multi-core CPU baseline) gives bit-identical values,
bounds and flags to the single-threaded build on every kind of node and
reduction: only loops whose elements are independent run in parallel, and
every reduction is one sequential pass in both builds."""
import numpy as np
import pytest

PROGS = {
    "f32": ["A B - exp #1 C abs + /", "#0.5 A * B C exp % +", "D trans B + square", "A B % C - sqrt abs log",
            "A submat:3:2:31:17 neg", "A B / #2 - #3 /", "A D trans % accu", "A B - square sum:0",
            "A B + sum:1", "A mean:0", "A B % mean:1", "A var", "A var:1", "A norm:fro", "A B dot",
            "A min:0", "A B + index_max:1", "A prod", "A stddevdim:1:1", "A B - cumsum:0", "A cumsum:1",
            "A diag:2", "A submat:0:0:40:1 each_col:29 B submat:0:0:40:29 +", "A trans B mm #2 * neg"],
    "f64": ["A B - exp #1 C abs + /", "D trans B + accu", "A B % C + var", "A sum:1", "A B - cumsum:1"],
    "bf16": ["A B % C + sum:0", "#0.1 A * exp", "A norm:fro"],
    "f16": ["A B - abs sqrt", "A B dot"],
    "i32": ["#2 A * B +", "A B % C - sum:0", "A B / accu", "A D trans - prod:1", "A B + cumsum:0",
            "A neg abs square max"],
}


def _leaves(dtype, rng, r, c):
    if dtype == "i32":
        mk = lambda rr, cc: rng.integers(-1000, 1001, size=(rr, cc)).astype(np.int32)  # noqa: E731
        a, b = mk(r, c), mk(r, c)
        b[3, 4] = 0  # a division by zero: the flag must agree too
        return [np.asfortranarray(a), np.asfortranarray(b), np.asfortranarray(mk(r, c)),
                np.asfortranarray(mk(c, r))]
    f = {"f32": np.float32, "f64": np.float64, "bf16": np.float32, "f16": np.float16}[dtype]

    def mk(rr, cc):
        x = (rng.standard_normal((rr, cc)) * 0.5 + 1.5).astype(f)
        if dtype == "bf16":  # round-to-nearest-even to the top 16 bits
            u = x.view(np.uint32)
            u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
            return np.asfortranarray(u)
        if dtype == "f16":
            return np.asfortranarray(x.view(np.uint16))
        return np.asfortranarray(x)

    return [mk(r, c), mk(r, c), mk(r, c), mk(c, r)]


@pytest.mark.parametrize("dtype", sorted(PROGS))
@pytest.mark.parametrize("shape", [(53, 29), (301, 263)])
def test_openmp_build_is_bit_identical(orc, dtype, shape):
    try:
        orc.threads(parallel=True)
    except orc.OracleError as e:
        pytest.skip(str(e))
    rng = np.random.default_rng(hash((dtype, shape)) % 2**32)
    r, c = shape
    for prog in PROGS[dtype]:
        hs = _leaves(dtype, rng, r, c)  # A, B, C: r x c; D: c x r
        a = orc.evaluate(prog, hs, dtype)
        b = orc.evaluate(prog, hs, dtype, parallel=True)
        assert a.value.dtype == b.value.dtype and a.value.shape == b.value.shape, prog
        assert np.array_equal(a.value, b.value, equal_nan=True), prog
        if a.bound is not None:
            assert np.array_equal(a.bound, b.bound, equal_nan=True), prog
        assert a.div_by_zero == b.div_by_zero, prog


def test_openmp_build_uses_more_than_one_thread_where_there_are_cores(orc):
    try:
        n = orc.threads(parallel=True)
    except orc.OracleError as e:
        pytest.skip(str(e))
    import os

    assert orc.threads() == 1
    assert n >= 1 and (n > 1 or (os.cpu_count() or 1) == 1)
