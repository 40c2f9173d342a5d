"""FP64 CPU oracle for Armadillo-style expression trees -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and the
two share no code: the oracle is plain C (``oracle.c``) built with gcc and
driven here through ``ctypes`` with host NumPy arrays.

Every function follows the plain definition of the operation it evaluates
(Bandicoot paper, Sec. 2-4: Armadillo function semantics, expression trees of
Op/eOp/eGlue nodes evaluated on assignment, column-major storage); see
``oracle.h`` for the program format and the error-bound model.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc.so")
# the same source built with -fopenmp: element-wise loops on all host cores,
# reductions sequential, results bit-identical to liborc.so
_OMP_PATH = os.path.join(_HERE, "liborc_omp.so")
_lock = threading.Lock()
_lib = None
_omp = None

DTYPES = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3, "i32": 4}
_NP_OF = {"f32": np.float32, "f64": np.float64, "bf16": np.uint16, "f16": np.uint16, "i32": np.int32}


def _compile(path, extra) -> None:
    src = os.path.join(_HERE, "oracle.c")
    tmp = path + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-D_POSIX_C_SOURCE=200809L", "-Wall", "-Wno-unknown-pragmas"] + extra + ["-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)


def _fresh(path) -> bool:
    src = os.path.join(_HERE, "oracle.c")
    return os.path.exists(path) and os.path.getmtime(path) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h")))


def build(force: bool = False) -> str:
    """Compile oracle.c into liborc.so with gcc (no FMA contraction, no
    fast-math), and into liborc_omp.so with -fopenmp when the compiler has
    OpenMP (the multi-core CPU baseline; skipped silently otherwise)."""
    if force or not _fresh(_LIB_PATH):
        _compile(_LIB_PATH, [])
    if force or not _fresh(_OMP_PATH):
        try:
            _compile(_OMP_PATH, ["-fopenmp"])
        except (subprocess.CalledProcessError, OSError):
            pass
    return _LIB_PATH


def _bind(lib):
    lib.orc_eval.argtypes = [ctypes.c_char_p, ctypes.POINTER(_Mat), ctypes.c_int32,
                             ctypes.c_int32, ctypes.POINTER(_Res)]
    lib.orc_eval.restype = ctypes.c_int
    lib.orc_free.argtypes = [ctypes.POINTER(_Res)]
    lib.orc_sum_neumaier.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int64]
    lib.orc_sum_neumaier.restype = ctypes.c_double
    lib.orc_ulp.argtypes = [ctypes.c_double, ctypes.c_int32]
    lib.orc_ulp.restype = ctypes.c_double
    lib.orc_threads.restype = ctypes.c_int
    return lib


class _Mat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("ld", ctypes.c_int64)]


class _Res(ctypes.Structure):
    _fields_ = [("is_int", ctypes.c_int32), ("is_reduction", ctypes.c_int32),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("v", ctypes.POINTER(ctypes.c_double)), ("b", ctypes.POINTER(ctypes.c_double)),
                ("iv", ctypes.POINTER(ctypes.c_int64)), ("div_by_zero", ctypes.c_int32),
                ("err", ctypes.c_char * 256)]


def _load(parallel: bool = False):
    """The single-threaded build, or with parallel=True the OpenMP build
    (OracleError when it could not be built)."""
    global _lib, _omp
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
        if parallel and _omp is None:
            if not os.path.exists(_OMP_PATH):
                raise OracleError("liborc_omp.so is not built (no OpenMP in the C compiler)")
            _omp = _bind(ctypes.CDLL(_OMP_PATH))
    return _omp if parallel else _lib


def threads(parallel: bool = False) -> int:
    """Threads the element-wise loops of the chosen build use."""
    return _load(parallel).orc_threads()


class OracleError(RuntimeError):
    pass


class Result:
    """Oracle output: ``value`` (float64 or int64 ndarray, column-major shape
    (n_rows, n_cols)), ``bound`` (float64 forward error bound, or None for
    integer trees), ``is_reduction`` and ``div_by_zero``."""

    def __init__(self, value, bound, is_reduction, div_by_zero):
        self.value = value
        self.bound = bound
        self.is_reduction = is_reduction
        self.div_by_zero = div_by_zero


def _as_mat(a: np.ndarray, dtype: str):
    if a.ndim == 1:
        a = a.reshape(-1, 1, order="F")
    if a.ndim != 2:
        raise ValueError("leaves must be 1-D or 2-D")
    want = np.dtype(_NP_OF[dtype])
    if a.dtype != want:
        raise TypeError("leaf dtype %s does not match %s" % (a.dtype, dtype))
    item = a.itemsize
    n_rows, n_cols = a.shape
    # column-major: unit row stride; ld = column stride (any ld >= n_rows)
    if n_rows > 1 and a.strides[0] != item:
        a = np.asfortranarray(a)
    ld = a.strides[1] // item if n_cols > 1 else max(n_rows, 1)
    if n_cols > 1 and a.strides[1] % item:
        a = np.asfortranarray(a)
        ld = n_rows
    return _Mat(a.ctypes.data, DTYPES[dtype], n_rows, n_cols, max(ld, n_rows)), a


def evaluate(program: str, leaves, dtype: str, out_dtype: str | None = None, parallel: bool = False) -> Result:
    """Evaluate an RPN ``program`` over host ``leaves`` (all of ``dtype``).

    BF16/FP16 leaves are passed as uint16 bit patterns.  parallel=True runs
    the element-wise loops on all host cores (bit-identical results)."""
    lib = _load(parallel)
    mats, keep = [], []
    for a in leaves:
        m, held = _as_mat(np.asarray(a), dtype)
        mats.append(m)
        keep.append(held)
    arr = (_Mat * len(mats))(*mats)
    res = _Res()
    od = -1 if out_dtype is None else DTYPES[out_dtype]
    rc = lib.orc_eval(program.encode(), arr, len(mats), od, ctypes.byref(res))
    if rc != 0:
        raise OracleError(res.err.decode())
    try:
        n = res.n_rows * res.n_cols
        shape = (res.n_rows, res.n_cols)
        if res.is_int:
            value = np.ctypeslib.as_array(res.iv, shape=(max(n, 1),))[:n].copy().reshape(shape, order="F")
            bound = None
        else:
            value = np.ctypeslib.as_array(res.v, shape=(max(n, 1),))[:n].copy().reshape(shape, order="F")
            bound = np.ctypeslib.as_array(res.b, shape=(max(n, 1),))[:n].copy().reshape(shape, order="F")
        return Result(value, bound, bool(res.is_reduction), bool(res.div_by_zero))
    finally:
        lib.orc_free(ctypes.byref(res))


def sum_neumaier(x: np.ndarray) -> float:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib.orc_sum_neumaier(x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), x.size)


def ulp(x: float, dtype: str) -> float:
    return _load().orc_ulp(float(x), DTYPES[dtype])


def grad(program: str, leaves, dtype: str):
    """Reverse-mode FP64 gradient of ``program`` (ending in accu / sum / mean)
    with respect to every leaf.  Returns (loss, [grad_i], [absgrad_i]) with
    column-major float64 arrays of the leaves' shapes; absgrad_i is the same
    sweep over absolute values (the scale of the terms summed per element)."""
    lib = _load()
    if not hasattr(lib, "_grad_ready"):
        lib.orc_grad.argtypes = [ctypes.c_char_p, ctypes.POINTER(_Mat), ctypes.c_int32,
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_char_p]
        lib.orc_grad.restype = ctypes.c_int
        lib._grad_ready = True
    mats, keep = [], []
    for a in leaves:
        m, held = _as_mat(np.asarray(a), dtype)
        mats.append(m)
        keep.append(held)
    arr = (_Mat * len(mats))(*mats)
    gs = [np.zeros((m.n_rows, m.n_cols), dtype=np.float64, order="F") for m in mats]
    ags = [np.zeros((m.n_rows, m.n_cols), dtype=np.float64, order="F") for m in mats]
    DP = ctypes.POINTER(ctypes.c_double)
    gp = (DP * len(gs))(*[g.ctypes.data_as(DP) for g in gs])
    ap = (DP * len(ags))(*[g.ctypes.data_as(DP) for g in ags])
    loss = ctypes.c_double()
    err = ctypes.create_string_buffer(256)
    rc = lib.orc_grad(program.encode(), arr, len(mats), gp, ap, ctypes.byref(loss), err)
    if rc != 0:
        raise OracleError(err.value.decode())
    return loss.value, gs, ags
