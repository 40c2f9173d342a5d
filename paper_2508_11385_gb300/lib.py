"""ctypes binding of the C ABI in include/coot.h (argument marshalling only).

Every function here has the name of the C entry point it calls and raises
``CootError`` when that entry point returns a status other than COOT_OK.
The compiled library ``libcootgb.so`` lives next to this file (built by
``build.py``); importing this module without it raises ImportError -- there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcootgb.so")

# ---- enums (coot.h) ---------------------------------------------------------
COOT_OK = 0
STATUS = {0: "COOT_OK", 1: "COOT_ERR_INVALID", 2: "COOT_ERR_SHAPE", 3: "COOT_ERR_DTYPE", 4: "COOT_ERR_ALIAS",
          5: "COOT_ERR_JIT", 6: "COOT_ERR_OOM", 7: "COOT_ERR_CUDA", 8: "COOT_ERR_DEVICE_FLAG",
          9: "COOT_ERR_TIMEOUT", 10: "COOT_ERR_UNSUPPORTED"}
F32, F64, BF16, F16, I32 = 0, 1, 2, 3, 4
DTYPE_CODE = {"f32": F32, "f64": F64, "bf16": BF16, "f16": F16, "i32": I32}

(N_LEAF, N_SUBMAT, N_TRANS, N_SCAL_TIMES, N_SCAL_PLUS, N_SCAL_MINUS_PRE, N_SCAL_MINUS_POST, N_SCAL_DIV_PRE,
 N_SCAL_DIV_POST, N_PLUS, N_MINUS, N_SCHUR, N_DIV, N_NEG, N_EXP, N_LOG, N_ABS, N_SQUARE, N_SQRT, N_EACH_COL,
 N_EACH_ROW, N_DIAG) = range(22)

(R_NONE, R_ACCU, R_SUM, R_MEAN, R_DOT, R_NORM2, R_NORM_FRO, R_VAR, R_STDDEV, R_MIN, R_MAX, R_INDEX_MIN,
 R_INDEX_MAX, R_PROD, R_CUMSUM) = range(15)

CTX_TUNE, CTX_NO_DISK_CACHE, CTX_LOG, CTX_NO_TCGEN05, CTX_DEBUG_BOUNDS = 1, 2, 4, 8, 16
FLAG_INT_DIV_ZERO = 1
FLAG_WAIT_TIMEOUT = 2
FLAG_OUT_OF_BOUNDS = 4
MAX_NODES, MAX_LEAVES, MAX_SCALARS = 64, 8, 16


class coot_mat(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("rs", ctypes.c_int32),
                ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("ld", ctypes.c_int64)]


class coot_node(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("leaf", ctypes.c_int32),
                ("k", ctypes.c_double), ("r0", ctypes.c_int64), ("c0", ctypes.c_int64),
                ("nr", ctypes.c_int64), ("nc", ctypes.c_int64)]


class coot_tree(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("nodes", ctypes.POINTER(coot_node))]


class coot_reduce(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32), ("norm_type", ctypes.c_int32),
                ("n_seg", ctypes.c_int32)]


class coot_launch_info(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_char * 64), ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("vec", ctypes.c_int32), ("unroll", ctypes.c_int32), ("n_launches", ctypes.c_int32),
                ("algorithmic_bytes", ctypes.c_int64)]


class coot_probe_result(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in ("f32_add", "f32_fma", "f32_div", "f32_exp", "f64_add", "f64_fma",
                                               "f64_div", "f64_exp", "read_gbs", "copy_gbs", "host_read_gbs",
                                               "host_write_gbs")] + [
        ("buffer_bytes", ctypes.c_int64), ("l2_bytes", ctypes.c_int64), ("sms", ctypes.c_int32),
        ("sm_clock_khz", ctypes.c_int32)]


class CootError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__("%s: %s" % (self.name, message))


if not os.path.exists(LIB_PATH):
    raise ImportError("libcootgb.so is not built (run paper_2508_11385_gb300.build.build() or "
                      "__graft_entry__.build()); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_S = ctypes.c_int
_MP = ctypes.POINTER(coot_mat)
_TP = ctypes.POINTER(coot_tree)

_SIGS = {
    "coot_ctx_create": ([ctypes.c_int, ctypes.c_uint, ctypes.POINTER(_P)], _S),
    "coot_ctx_destroy": ([_P], _S),
    "coot_eval": ([_P, _TP, _MP, ctypes.c_int32, _MP, coot_reduce, _P, _P], _S),
    "coot_eval_unfused": ([_P, _TP, _MP, ctypes.c_int32, _MP, coot_reduce, _P, _P], _S),
    "coot_warmup": ([_P, _TP, _MP, ctypes.c_int32, _MP, coot_reduce], _S),
    "coot_eval_adjoint": ([_P, _TP, _MP, ctypes.c_int32, coot_reduce, _P, _MP, _P], _S),
    "coot_gemm_eval": ([_P, _MP, ctypes.c_int32, _MP, ctypes.c_int32, _TP, _MP, ctypes.c_int32, _MP, _P], _S),
    "coot_batch_create": ([_P, _TP, ctypes.c_int64, ctypes.c_int32, _MP, _MP, coot_reduce, ctypes.POINTER(_P)], _S),
    "coot_batch_run": ([_P, _P, _P], _S),
    "coot_batch_destroy": ([_P], _S),
    "coot_eval_batched": ([_P, _TP, ctypes.c_int64, ctypes.c_int32, _MP, _MP, coot_reduce, _P, _P], _S),
    "coot_graph_begin": ([_P, _P], _S),
    "coot_graph_end": ([_P, _P, ctypes.POINTER(_P)], _S),
    "coot_graph_launch": ([_P, _P], _S),
    "coot_graph_destroy": ([_P], _S),
    "coot_signature": ([_TP, _MP, ctypes.c_int32, _MP, coot_reduce, ctypes.c_char_p, ctypes.c_size_t], _S),
    "coot_codegen": ([_TP, _MP, ctypes.c_int32, _MP, coot_reduce, ctypes.c_char_p, ctypes.c_size_t], _S),
    "coot_compile": ([_TP, _MP, ctypes.c_int32, _MP, coot_reduce, ctypes.POINTER(ctypes.c_size_t)], _S),
    "coot_sum_rows_f32_noalloc": ([_MP, ctypes.c_int32, _P, _P], _S),
    "coot_check_device_flag": ([_P, _P, ctypes.POINTER(ctypes.c_uint32)], _S),
    "coot_last_launch": ([_P, ctypes.POINTER(coot_launch_info)], _S),
    "coot_probe_device": ([ctypes.c_int, ctypes.POINTER(coot_probe_result)], _S),
    "coot_last_error": ([], ctypes.c_char_p),
    "coot_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "coot_version": ([ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], None),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


def _check(status):
    if status != COOT_OK:
        raise CootError(status, _lib.coot_last_error().decode(errors="replace"))


def _ptr(x):
    return None if x is None else ctypes.byref(x)


def _arr(mats):
    if mats is None:
        return None
    arr = (coot_mat * len(mats))(*mats)
    return arr


def coot_last_error() -> str:
    return _lib.coot_last_error().decode(errors="replace")


def coot_status_string(s: int) -> str:
    return _lib.coot_status_string(s).decode()


def coot_version():
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _lib.coot_version(ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def coot_ctx_create(device: int = 0, flags: int = 0):
    h = _P()
    _check(_lib.coot_ctx_create(device, flags, ctypes.byref(h)))
    return h


def coot_ctx_destroy(ctx):
    _check(_lib.coot_ctx_destroy(ctx))


def coot_eval(ctx, tree, leaves, out, red, red_out, stream):
    lv = _arr(leaves)
    _check(_lib.coot_eval(ctx, ctypes.byref(tree), lv, len(leaves), _ptr(out), red, red_out, stream))


def coot_eval_unfused(ctx, tree, leaves, out, red, red_out, stream):
    lv = _arr(leaves)
    _check(_lib.coot_eval_unfused(ctx, ctypes.byref(tree), lv, len(leaves), _ptr(out), red, red_out, stream))


def coot_warmup(ctx, tree, leaves, out, red):
    lv = _arr(leaves)
    _check(_lib.coot_warmup(ctx, ctypes.byref(tree), lv, len(leaves), _ptr(out), red))


def coot_eval_adjoint(ctx, tree, leaves, red, upstream, grads, stream):
    lv = _arr(leaves)
    gv = _arr(grads)
    _check(_lib.coot_eval_adjoint(ctx, ctypes.byref(tree), lv, len(leaves), red, upstream, gv, stream))


def coot_gemm_eval(ctx, a, trans_a, b, trans_b, epi, extra, out, stream):
    ev = _arr(extra) if extra else None
    _check(_lib.coot_gemm_eval(ctx, ctypes.byref(a), int(trans_a), ctypes.byref(b), int(trans_b),
                               ctypes.byref(epi) if epi is not None else None, ev, len(extra) if extra else 0,
                               ctypes.byref(out), stream))


def coot_batch_create(ctx, tree, n_problems, n_leaves, problems, outs, red):
    h = _P()
    _check(_lib.coot_batch_create(ctx, ctypes.byref(tree), n_problems, n_leaves, problems, outs, red,
                                  ctypes.byref(h)))
    return h


def coot_batch_run(batch, red_out, stream):
    _check(_lib.coot_batch_run(batch, red_out, stream))


def coot_batch_destroy(batch):
    _check(_lib.coot_batch_destroy(batch))


def coot_eval_batched(ctx, tree, n_problems, n_leaves, problems, outs, red, red_out, stream):
    _check(_lib.coot_eval_batched(ctx, ctypes.byref(tree), n_problems, n_leaves, problems, outs, red, red_out,
                                  stream))


def coot_graph_begin(ctx, stream):
    _check(_lib.coot_graph_begin(ctx, stream))


def coot_graph_end(ctx, stream):
    h = _P()
    _check(_lib.coot_graph_end(ctx, stream, ctypes.byref(h)))
    return h


def coot_graph_launch(graph, stream):
    _check(_lib.coot_graph_launch(graph, stream))


def coot_graph_destroy(graph):
    _check(_lib.coot_graph_destroy(graph))


def coot_signature(tree, leaves, out, red) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    lv = _arr(leaves)
    _check(_lib.coot_signature(ctypes.byref(tree), lv, len(leaves), _ptr(out), red, buf, len(buf)))
    return buf.value.decode()


def coot_codegen(tree, leaves, out, red) -> str:
    buf = ctypes.create_string_buffer(1 << 18)
    lv = _arr(leaves)
    _check(_lib.coot_codegen(ctypes.byref(tree), lv, len(leaves), _ptr(out), red, buf, len(buf)))
    return buf.value.decode()


def coot_compile(tree, leaves, out, red) -> int:
    n = ctypes.c_size_t()
    lv = _arr(leaves)
    _check(_lib.coot_compile(ctypes.byref(tree), lv, len(leaves), _ptr(out), red, ctypes.byref(n)))
    return n.value


def coot_sum_rows_f32_noalloc(x, mean, out_ptr, stream):
    """Per-row sums (or means) of an F32 matrix into out_ptr without any
    allocation (see include/coot.h)."""
    _check(_lib.coot_sum_rows_f32_noalloc(ctypes.byref(x), int(mean), out_ptr, stream))


def coot_check_device_flag(ctx, stream) -> int:
    f = ctypes.c_uint32()
    st = _lib.coot_check_device_flag(ctx, stream, ctypes.byref(f))
    if st not in (COOT_OK, 8):
        _check(st)
    return f.value


def coot_last_launch(ctx) -> dict:
    info = coot_launch_info()
    _check(_lib.coot_last_launch(ctx, ctypes.byref(info)))
    return {"kernel": info.kernel.decode(), "grid": info.grid, "block": info.block, "vec": info.vec,
            "unroll": info.unroll, "n_launches": info.n_launches, "algorithmic_bytes": info.algorithmic_bytes}


def coot_probe_device(device: int = 0) -> dict:
    r = coot_probe_result()
    _check(_lib.coot_probe_device(device, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in coot_probe_result._fields_}


def make_tree(nodes):
    """coot_tree over a list of coot_node (the array is kept alive on the tree)."""
    arr = (coot_node * len(nodes))(*nodes)
    t = coot_tree(len(nodes), 0, ctypes.cast(arr, ctypes.POINTER(coot_node)))
    t._keep = arr
    return t


def node(op, a=-1, b=-1, leaf=0, k=0.0, r0=0, c0=0, nr=0, nc=0):
    return coot_node(op, a, b, leaf, k, r0, c0, nr, nc)


def reduce(kind=R_NONE, dim=-1, norm_type=0, n_seg=0):
    return coot_reduce(kind, dim, norm_type, n_seg)


def mat(ptr, dtype, n_rows, n_cols, ld=None, rs=0):
    if ld is None:
        ld = max(n_rows, 1)
    return coot_mat(ptr, dtype, rs, n_rows, n_cols, ld)
