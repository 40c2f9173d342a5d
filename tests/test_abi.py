"""The C-ABI library on the host (no GPU): it loads, exports every symbol the
header declares, validates descriptors with the documented status codes,
produces stable signatures, and NVRTC-compiles generated kernels for sm_103a."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2508_11385_gb300 import build

    build.build()
    from paper_2508_11385_gb300 import lib

    return lib


BASE = 0x7F0000000000  # device addresses are never dereferenced on the host


def mats(L, n, shape=(64, 32), dtype=0, stride=1 << 24):
    return [L.mat(BASE + i * stride, dtype, *shape) for i in range(n)]


def config1_nodes(L):
    return [L.node(L.N_LEAF, leaf=0), L.node(L.N_SCAL_TIMES, a=0, k=0.5), L.node(L.N_LEAF, leaf=1),
            L.node(L.N_LEAF, leaf=2), L.node(L.N_EXP, a=3), L.node(L.N_SCHUR, a=2, b=4), L.node(L.N_PLUS, a=1, b=5)]


def test_header_symbols_are_exported(L):
    hdr = open(os.path.join(ROOT, "include", "coot.h")).read()
    declared = set(re.findall(r"COOT_API\s+[\w\s\*]*?\b(coot_\w+)\s*\(", hdr))
    assert len(declared) >= 20
    assert declared == set(L.EXPORTED), declared ^ set(L.EXPORTED)
    for name in declared:
        assert hasattr(L._lib, name)


def test_version_and_status_strings(L):
    assert L.coot_version() == (1, 0)
    for code, name in L.STATUS.items():
        assert L.coot_status_string(code) == name


def test_signature_ignores_scalars_and_pointers(L):
    t1 = L.make_tree(config1_nodes(L))
    n2 = config1_nodes(L)
    n2[1] = L.node(L.N_SCAL_TIMES, a=0, k=3.25)
    t2 = L.make_tree(n2)
    s1 = L.coot_signature(t1, mats(L, 3), None, L.reduce(L.R_ACCU))
    s2 = L.coot_signature(t2, mats(L, 3, stride=1 << 26), None, L.reduce(L.R_ACCU))
    assert s1 == s2
    assert "eGlue<eOp<Leaf<0>, eop_scalar_times<0>>" in s1
    s3 = L.coot_signature(t1, mats(L, 3, dtype=L.F64), None, L.reduce(L.R_ACCU))
    assert s3 != s1 and "double" in s3


def test_trans_is_pushed_to_the_leaves(L):
    # trans(A + trans(B)) reads A transposed and B directly
    nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_LEAF, leaf=1), L.node(L.N_TRANS, a=1),
             L.node(L.N_PLUS, a=0, b=2), L.node(L.N_TRANS, a=3)]
    t = L.make_tree(nodes)
    sig = L.coot_signature(t, [L.mat(BASE, 0, 20, 30), L.mat(BASE + 4096, 0, 30, 20)], None, L.reduce(L.R_ACCU))
    assert "|tile|" in sig and "|tr1|" in sig  # slot 0 (A) transposed, slot 1 (B) not
    sig2 = L.coot_signature(L.make_tree(nodes[:2] + [L.node(L.N_TRANS, a=1), L.node(L.N_TRANS, a=2),
                                                     L.node(L.N_PLUS, a=0, b=3)]),
                            [L.mat(BASE, 0, 20, 30), L.mat(BASE + 4096, 0, 20, 30)], None, L.reduce(L.R_ACCU))
    assert "|str|" in sig2  # trans(trans(B)) is B


def test_identical_reads_are_merged(L):
    nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_LEAF, leaf=0), L.node(L.N_SCHUR, a=0, b=1)]
    sig = L.coot_signature(L.make_tree(nodes), mats(L, 1), None, L.reduce(L.R_ACCU))
    assert "|ns1|" in sig and "eGlue<Leaf<0>, Leaf<0>, eglue_schur>" in sig


@pytest.mark.parametrize("case,status", [
    ("shape", "COOT_ERR_SHAPE"), ("op", "COOT_ERR_INVALID"), ("forward_ref", "COOT_ERR_INVALID"),
    ("leaf", "COOT_ERR_INVALID"), ("int_exp", "COOT_ERR_DTYPE"), ("int_mean", "COOT_ERR_DTYPE"),
    ("mixed_dtype", "COOT_ERR_DTYPE"), ("dot_root", "COOT_ERR_INVALID"), ("norm_matrix", "COOT_ERR_SHAPE"),
    ("submat_oob", "COOT_ERR_SHAPE"), ("submat_of_expr", "COOT_ERR_INVALID"), ("out_shape", "COOT_ERR_SHAPE"),
    ("alias_trans", "COOT_ERR_ALIAS"), ("alias_shifted", "COOT_ERR_ALIAS"), ("int_scalar", "COOT_ERR_INVALID"),
    ("empty_tree", "COOT_ERR_INVALID"), ("bad_ld", "COOT_ERR_INVALID"),
])
def test_validation_errors(L, case, status):
    red = L.reduce(L.R_NONE)
    lv = mats(L, 2)
    out = L.mat(BASE + (1 << 30), 0, 64, 32)
    nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_LEAF, leaf=1), L.node(L.N_PLUS, a=0, b=1)]
    if case == "shape":
        lv = [L.mat(BASE, 0, 64, 32), L.mat(BASE + 4096, 0, 32, 64)]
    elif case == "op":
        nodes[2] = L.node(77, a=0, b=1)
    elif case == "forward_ref":
        nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_PLUS, a=0, b=2), L.node(L.N_LEAF, leaf=1)]
    elif case == "leaf":
        nodes[1] = L.node(L.N_LEAF, leaf=5)
    elif case == "int_exp":
        lv = mats(L, 2, dtype=L.I32)
        out = L.mat(BASE + (1 << 30), L.I32, 64, 32)
        nodes = nodes + [L.node(L.N_EXP, a=2)]
    elif case == "int_mean":
        lv = mats(L, 2, dtype=L.I32)
        out = None
        red = L.reduce(L.R_MEAN)
    elif case == "mixed_dtype":
        lv = [L.mat(BASE, 0, 64, 32), L.mat(BASE + 4096, L.F64, 64, 32)]
    elif case == "dot_root":
        red = L.reduce(L.R_DOT)
        out = None
    elif case == "norm_matrix":
        red = L.reduce(L.R_NORM2)
        out = None
    elif case == "submat_oob":
        nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_SUBMAT, a=0, r0=60, c0=0, nr=10, nc=4)]
        out = None
        red = L.reduce(L.R_ACCU)
    elif case == "submat_of_expr":
        nodes = nodes + [L.node(L.N_SUBMAT, a=2, r0=0, c0=0, nr=4, nc=4)]
        out = None
        red = L.reduce(L.R_ACCU)
    elif case == "out_shape":
        out = L.mat(BASE + (1 << 30), 0, 32, 64)
    elif case == "alias_trans":
        lv = [L.mat(BASE, 0, 64, 64), L.mat(BASE + (1 << 26), 0, 64, 64)]
        nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_TRANS, a=0), L.node(L.N_LEAF, leaf=1),
                 L.node(L.N_PLUS, a=1, b=2)]
        out = L.mat(BASE, 0, 64, 64)
    elif case == "alias_shifted":
        out = L.mat(BASE + 4, 0, 64, 32)
    elif case == "int_scalar":
        lv = mats(L, 2, dtype=L.I32)
        out = L.mat(BASE + (1 << 30), L.I32, 64, 32)
        nodes = nodes + [L.node(L.N_SCAL_TIMES, a=2, k=1e12)]
    elif case == "empty_tree":
        t = L.coot_tree(0, 0, None)
        with pytest.raises(L.CootError, match=status):
            L.coot_signature(t, lv, out, red)
        return
    elif case == "bad_ld":
        lv = [L.mat(BASE, 0, 64, 32, ld=10), L.mat(BASE + 4096, 0, 64, 32)]
    with pytest.raises(L.CootError, match=status):
        L.coot_signature(L.make_tree(nodes), lv, out, red)


def test_in_place_alias_is_accepted(L):
    # B = B + 3*A with out == B: an identical untransposed read may alias
    nodes = [L.node(L.N_LEAF, leaf=1), L.node(L.N_LEAF, leaf=0), L.node(L.N_SCAL_TIMES, a=1, k=3.0),
             L.node(L.N_PLUS, a=0, b=2)]
    lv = mats(L, 2)
    L.coot_signature(L.make_tree(nodes), lv, lv[1], L.reduce())


def _tree_from_rpn(L, prog, shape, dtype):
    """Build a node list from an RPN string (host-side helper for compile tests)."""
    st, nodes = [], []
    leaves = {}
    for tok in prog.split():
        if len(tok) == 1 and tok.isalpha():
            li = ord(tok) - ord("A")
            leaves[li] = True
            nodes.append(L.node(L.N_LEAF, leaf=li))
            st.append(("m", len(nodes) - 1))
        elif tok.startswith("#"):
            st.append(("k", float(tok[1:])))
        elif tok in ("+", "-", "%", "/", "*"):
            y, x = st.pop(), st.pop()
            if x[0] == "k" or y[0] == "k":
                k, m, pre = (x[1], y[1], True) if x[0] == "k" else (y[1], x[1], False)
                op = {"+": L.N_SCAL_PLUS, "*": L.N_SCAL_TIMES, "-": L.N_SCAL_MINUS_PRE if pre else L.N_SCAL_MINUS_POST,
                      "/": L.N_SCAL_DIV_PRE if pre else L.N_SCAL_DIV_POST}[tok]
                nodes.append(L.node(op, a=m, k=k))
            else:
                op = {"+": L.N_PLUS, "-": L.N_MINUS, "%": L.N_SCHUR, "/": L.N_DIV}[tok]
                nodes.append(L.node(op, a=x[1], b=y[1]))
            st.append(("m", len(nodes) - 1))
        elif tok.startswith("submat:"):
            r0, c0, nr, nc = map(int, tok.split(":")[1:])
            nodes.append(L.node(L.N_SUBMAT, a=st.pop()[1], r0=r0, c0=c0, nr=nr, nc=nc))
            st.append(("m", len(nodes) - 1))
        else:
            op = {"exp": L.N_EXP, "log": L.N_LOG, "abs": L.N_ABS, "square": L.N_SQUARE, "sqrt": L.N_SQRT,
                  "neg": L.N_NEG, "trans": L.N_TRANS}[tok]
            nodes.append(L.node(op, a=st.pop()[1]))
            st.append(("m", len(nodes) - 1))
    n_leaves = max(leaves) + 1
    code = L.DTYPE_CODE[dtype]
    lv = [L.mat(BASE + i * (1 << 28), code, *shape) for i in range(n_leaves)]
    return L.make_tree(nodes), lv


@pytest.mark.parametrize("prog,red,dtype", [
    ("#0.5 A * B C exp % +", "R_ACCU", "f32"),
    ("#2 A * B +", "R_NONE", "f64"),
    ("A B % C +", "R_NONE", "i32"),
    ("A trans B +", "R_NONE", "f32"),
    ("A B - exp #1 C abs + /", "R_NONE", "f64"),
    ("A B - square", "R_SUM0", "f32"),
    ("A", "R_VAR", "bf16"),
    ("A B - exp #1 C abs + / D % E - abs sqrt F %", "R_NONE", "f32"),
    ("A B % C +", "R_INDEX_MAX1", "f32"),
    ("A trans B +", "R_MIN0", "f64"),
    ("A B + exp", "R_PROD", "bf16"),
    ("A trans B %", "R_STDDEV1", "f32"),
    ("A B % C +", "R_CUMSUM0", "f32"),
    ("A B %", "R_CUMSUM1", "i32"),
    ("A exp", "R_CUMSUM1", "f16"),
    ("A trans B %", "R_INDEX_MAX1", "bf16"),
    ("A trans B +", "R_SUM1", "f64"),
])
def test_generated_kernels_compile_for_sm103a(L, prog, red, dtype):
    shape = (256, 256)
    t, lv = _tree_from_rpn(L, prog, shape, dtype)
    out = None
    r = {"R_ACCU": L.reduce(L.R_ACCU), "R_NONE": L.reduce(), "R_SUM0": L.reduce(L.R_SUM, 0),
         "R_VAR": L.reduce(L.R_VAR), "R_INDEX_MAX1": L.reduce(L.R_INDEX_MAX, 1), "R_MIN0": L.reduce(L.R_MIN, 0),
         "R_PROD": L.reduce(L.R_PROD), "R_STDDEV1": L.reduce(L.R_STDDEV, 1),
         "R_CUMSUM0": L.reduce(L.R_CUMSUM, 0), "R_CUMSUM1": L.reduce(L.R_CUMSUM, 1),
         "R_SUM1": L.reduce(L.R_SUM, 1)}[red]
    if red == "R_NONE" or red.startswith("R_CUMSUM"):
        out = L.mat(BASE + (1 << 34), L.DTYPE_CODE[dtype], *shape)
    src = L.coot_codegen(t, lv, out, r)
    assert 'extern "C" __global__' in src
    n = L.coot_compile(t, lv, out, r)
    assert n > 1000


def test_nvrtc_failure_is_reported(L, monkeypatch):
    t, lv = _tree_from_rpn(L, "A B +", (8, 8), "f32")
    monkeypatch.setenv("COOT_JIT_FAIL", "1")
    with pytest.raises(L.CootError, match="COOT_ERR_JIT"):
        L.coot_compile(t, lv, None, L.reduce(L.R_ACCU))
    monkeypatch.setenv("COOT_JIT_FAIL", "0")
    assert L.coot_compile(t, lv, None, L.reduce(L.R_ACCU)) > 0


def test_context_creation_without_gpu_fails_cleanly(L):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.CootError, match="COOT_ERR_CUDA|COOT_ERR_INVALID"):
        L.coot_ctx_create(0, 0)


def test_row_programs_carry_the_kernels_the_launcher_names(L):
    # the launcher picks these kernels by name: the one-pass row scan for
    # cumsum along dim 1, and the row walk with transposed reads for a
    # reduction along dim 1 whose transposed reads are no more than its
    # direct streams (more transposed reads stay on the tiles)
    shape = (256, 256)
    t, lv = _tree_from_rpn(L, "A B %", shape, "f32")
    out = L.mat(BASE + (1 << 34), L.DTYPE_CODE["f32"], *shape)
    buf = L.coot_codegen(t, lv, out, L.reduce(L.R_CUMSUM, 1))
    assert "coot_scanp_v1u16w8" in buf and "scanp_kernel<" in buf
    t, lv = _tree_from_rpn(L, "A trans B %", shape, "f32")
    buf = L.coot_codegen(t, lv, None, L.reduce(L.R_SUM, 1))
    assert "row_kernel<" in buf and "coot_row_v1u16" in buf and "tilev_kernel<" not in buf
    t, lv = _tree_from_rpn(L, "A trans B trans +", shape, "f32")
    buf = L.coot_codegen(t, lv, None, L.reduce(L.R_SUM, 1))
    assert "row_kernel<" not in buf and "tile" in buf
