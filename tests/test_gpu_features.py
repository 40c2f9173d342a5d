"""Batched persistent evaluation, CUDA-graph chains, the fused adjoint behind
torch.autograd, and the kernel cache -- each checked against the oracle or
against the single-call path."""
import glob
import os

import numpy as np
import pytest
import torch

import coot_rpn
import oracle
import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L
from paper_2508_11385_gb300 import workloads
from paper_2508_11385_gb300.autograd import loss_l2_schur, scalar

pytestmark = pytest.mark.gpu

BATCH_TREE = [L.node(L.N_LEAF, leaf=0), L.node(L.N_LEAF, leaf=1), L.node(L.N_SCHUR, a=0, b=1),
              L.node(L.N_LEAF, leaf=2), L.node(L.N_TRANS, a=3), L.node(L.N_SCAL_TIMES, a=4, k=0.1),
              L.node(L.N_PLUS, a=2, b=5)]
BATCH_PROG = "A B % C trans #0.1 * +"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batch(n_problems, lo=4, hi=80, empty=False, red=L.R_ACCU):
    rows, cols, A, B, C, pools = workloads.batching(n_problems, device="cuda", lo=lo, hi=hi)
    if empty:  # a 0 x c problem
        A[1] = A[1][:0, :]
        B[1] = B[1][:0, :]
        C[1] = C[1][:, :0]
    outs = [torch.empty((a.shape[1], a.shape[0]), dtype=torch.float32, device="cuda").t() for a in A]
    probs = (L.coot_mat * (3 * n_problems))()
    for q in range(n_problems):
        probs[3 * q] = coot.Mat(A[q]).cmat()
        probs[3 * q + 1] = coot.Mat(B[q]).cmat()
        probs[3 * q + 2] = coot.Mat(C[q]).cmat()
    outm = (L.coot_mat * n_problems)(*[coot.Mat(o).cmat() for o in outs])
    return A, B, C, outs, probs, outm, pools


@pytest.mark.parametrize("empty", [False, True])
@pytest.mark.parametrize("red", [L.R_ACCU, L.R_MEAN])
def test_batched_matches_oracle_per_problem(empty, red):
    n = 400
    A, B, C, outs, probs, outm, _ = _batch(n, empty=empty)
    ctx = coot.context()
    res = torch.empty(n, dtype=torch.float32, device="cuda")
    tree = L.make_tree(BATCH_TREE)
    plan = L.coot_batch_create(ctx, tree, n, 3, probs, outm, L.reduce(red))
    s = torch.cuda.current_stream().cuda_stream
    L.coot_batch_run(plan, res.data_ptr(), s)
    torch.cuda.synchronize()
    first = res.clone()
    first_out = [o.clone() for o in outs[:20]]
    L.coot_batch_run(plan, res.data_ptr(), s)  # the queue and counters reset themselves
    torch.cuda.synchronize()
    torch.testing.assert_close(first, res, rtol=0, atol=0, equal_nan=True)
    assert all(torch.equal(a, b) for a, b in zip(first_out, outs[:20]))
    L.coot_batch_destroy(plan)
    tok = "accu" if red == L.R_ACCU else "mean"
    for q in range(n):
        hs = parity.host([A[q], B[q], C[q]])
        if A[q].numel() == 0:
            v = res[q].item()
            assert (v == 0.0) if red == L.R_ACCU else np.isnan(v)
            continue
        ry = oracle.evaluate(BATCH_PROG, hs, "f32")
        parity.compare_matrix(outs[q], ry, "f32", "problem %d" % q)
        rr = oracle.evaluate(BATCH_PROG + " " + tok, hs, "f32")
        parity.compare_reduction(res[q:q + 1], rr, "f32", "problem %d" % q)


def test_batched_equals_single_calls():
    n = 64
    A, B, C, outs, probs, outm, _ = _batch(n, lo=4, hi=300)
    ctx = coot.context()
    res = torch.empty(n, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    L.coot_eval_batched(ctx, L.make_tree(BATCH_TREE), n, 3, probs, outm, L.reduce(L.R_ACCU), res.data_ptr(), s)
    torch.cuda.synchronize()
    for q in range(n):
        a, b, c = coot.Mat(A[q]), coot.Mat(B[q]), coot.Mat(C[q])
        y, r = coot.evaluate(a % b + 0.1 * coot.trans(c), reduction=coot.accu(a % b + 0.1 * coot.trans(c)),
                             materialise=True)
        torch.cuda.synchronize()
        assert torch.equal(y, outs[q])  # element-wise: bitwise identical
        # the reduction order differs (tile partials vs block partials): both are compensated
        assert abs(r.item() - res[q].item()) <= 2e-6 * abs(r.item()) + 1e-6


def _mixed_problems():
    """Problems that exercise every path of the flat batched kernel: taller
    than one work item (row chunks), wider than one (column chunks), tiny,
    empty, views with a column stride above their row count (non-contiguous
    items) and an output view with its own column stride."""
    g = workloads.generator(41, "cuda")
    shapes = [(5000, 3), (3, 5000), (4097, 2), (513, 40), (4, 4), (1, 1), (0, 7), (33, 65), (250, 251)]
    A, B, C, outs = [], [], [], []
    for q, (r, c) in enumerate(shapes):
        if q % 3 == 2:  # strided views: ld = r + 5
            A.append(workloads.normal(r + 5, c, "f32", g, "cuda")[:r, :])
            B.append(workloads.normal(r + 5, c, "f32", g, "cuda")[2:2 + r, :])
            C.append(workloads.normal(c + 3, r, "f32", g, "cuda")[1:1 + c, :])
            outs.append(torch.empty((c, r + 7), dtype=torch.float32, device="cuda").t()[3:3 + r, :])
        else:
            A.append(workloads.normal(r, c, "f32", g, "cuda"))
            B.append(workloads.normal(r, c, "f32", g, "cuda"))
            C.append(workloads.normal(c, r, "f32", g, "cuda"))
            outs.append(torch.empty((c, r), dtype=torch.float32, device="cuda").t())
    n = len(shapes)
    probs = (L.coot_mat * (3 * n))()
    for q in range(n):
        probs[3 * q] = coot.Mat(A[q]).cmat()
        probs[3 * q + 1] = coot.Mat(B[q]).cmat()
        probs[3 * q + 2] = coot.Mat(C[q]).cmat()
    outm = (L.coot_mat * n)(*[coot.Mat(o).cmat() for o in outs])
    return A, B, C, outs, probs, outm


@pytest.mark.parametrize("kernel", ["flat", "tile"])
def test_batched_mixed_shapes_match_oracle(kernel, monkeypatch):
    if kernel == "tile":
        monkeypatch.setenv("COOT_BATCH_KERNEL", "tile")
    else:
        monkeypatch.delenv("COOT_BATCH_KERNEL", raising=False)
    A, B, C, outs, probs, outm = _mixed_problems()
    n = len(A)
    ctx = coot.context()
    res = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    plan = L.coot_batch_create(ctx, L.make_tree(BATCH_TREE), n, 3, probs, outm, L.reduce(L.R_ACCU))
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the queue and the per-problem counters reset themselves
        for o in outs:
            o.fill_(float("nan"))
        L.coot_batch_run(plan, res.data_ptr(), s)
        torch.cuda.synchronize()
        for q in range(n):
            hs = parity.host([A[q], B[q], C[q]])
            if A[q].numel() == 0:
                assert res[q].item() == 0.0
                continue
            parity.compare_matrix(outs[q], oracle.evaluate(BATCH_PROG, hs, "f32"), "f32", "%s problem %d" % (kernel, q))
            parity.compare_reduction(res[q:q + 1], oracle.evaluate(BATCH_PROG + " accu", hs, "f32"), "f32",
                                     "%s problem %d" % (kernel, q))
    info = L.coot_last_launch(ctx)
    assert info["kernel"] == ("coot_batch" if kernel == "tile" else "coot_batchf")
    L.coot_batch_destroy(plan)


def test_batch_rejects_mismatched_problem():
    A, B, C, outs, probs, outm, _ = _batch(8)
    bad = L.mat(probs[3 * 5 + 1].data, L.F32, probs[3 * 5 + 1].n_rows + 1, probs[3 * 5 + 1].n_cols,
                probs[3 * 5 + 1].ld + 1)
    probs[3 * 5 + 1] = bad
    with pytest.raises(L.CootError, match="problem 5"):
        L.coot_batch_create(coot.context(), L.make_tree(BATCH_TREE), 8, 3, probs, outm, L.reduce(L.R_ACCU))


# The chain of 20 evaluations cycling the six large-tree shapes: 2*X+B,
# X%B+C, trans(X)+B, exp(A-B)/(1+abs(X)), sum(square(X-B),0) (the squares are
# kept as the next X) and accu over an interior submatrix view of X (X passes
# on unchanged).  X enters the exp shape as its C operand so that the values
# stay finite over the whole chain.  (RPN over the step's leaves, the step's
# leaves, output kind.)
def _chain_steps(n):
    r0, nv = n // 8, n // 2
    return [
        ("#2 A * B +", "XB", "mat"),
        ("A B % C +", "XBC", "mat"),
        ("A trans B +", "XB", "mat"),
        ("A B - exp #1 C abs + /", "ABX", "mat"),
        ("A B - square sum:0", "XB", "mat+sum0"),
        ("A submat:%d:%d:%d:%d accu" % (r0, r0, nv, nv), "X", "accu"),
    ]


def test_graph_chain_of_the_six_shapes_matches_the_oracle_step_by_step():
    n = 192
    A, B, C = (parity.rand(n, n, "f32", seed=s) for s in (1, 2, 3))
    steps = _chain_steps(n)
    X = [A]
    sides, calls, progs = {}, [], []
    for k in range(20):
        prog, names, kind = steps[k % 6]
        ten = [{"X": X[k], "A": A, "B": B, "C": C}[c] for c in names]
        e, _ = coot_rpn.build(prog.replace(" sum:0", "").replace(" accu", ""), ten)
        tree, lm, cm = coot.lower(e)
        if kind == "accu":
            sides[k] = torch.empty((), dtype=torch.float32, device="cuda")
            calls.append((tree, cm, None, L.reduce(L.R_ACCU), sides[k]))
            X.append(X[k])  # the view's accu leaves X as it is
        else:
            out = torch.empty((n, n), dtype=torch.float32, device="cuda").t()
            X.append(out)
            if kind == "mat+sum0":
                sides[k] = torch.empty((1, n), dtype=torch.float32, device="cuda")
                calls.append((tree, cm, coot.Mat(out).cmat(), L.reduce(L.R_SUM, 0), sides[k]))
            else:
                calls.append((tree, cm, coot.Mat(out).cmat(), L.reduce(), None))
        progs.append((prog, names, kind))
    ctx = coot.context()
    s = torch.cuda.Stream()

    def run():
        for tree, cm, om, red, side in calls:
            L.coot_eval(ctx, tree, cm, om, red, None if side is None else side.data_ptr(), s.cuda_stream)

    outs = lambda: [x for x in X[1:]] + [sides[k] for k in sorted(sides)]

    def clear():
        for t in outs():
            t.fill_(float("nan"))

    s.wait_stream(torch.cuda.current_stream())  # the inputs were written on the current stream
    run()  # compiles and tunes every step
    torch.cuda.synchronize()
    eager = [t.clone() for t in outs()]
    s.wait_stream(torch.cuda.current_stream())
    L.coot_graph_begin(ctx, s.cuda_stream)
    run()
    g = L.coot_graph_end(ctx, s.cuda_stream)
    clear()
    torch.cuda.synchronize()
    L.coot_graph_launch(g, s.cuda_stream)
    torch.cuda.synchronize()
    L.coot_graph_destroy(g)
    for a, b in zip(eager, outs()):
        assert torch.equal(a, b), "graph replay differs from the eager chain"
    # every replayed step against the oracle, on the host copy of that step's
    # replayed input
    for k, (prog, names, kind) in enumerate(progs):
        hs = parity.host([{"X": X[k], "A": A, "B": B, "C": C}[c] for c in names])
        what = "chain step %d: %s" % (k, prog)
        if kind == "accu":
            parity.compare_reduction(sides[k], oracle.evaluate(prog, hs, "f32"), "f32", what)
            continue
        tree_prog = prog.replace(" sum:0", "")
        parity.compare_matrix(X[k + 1], oracle.evaluate(tree_prog, hs, "f32"), "f32", what)
        if kind == "mat+sum0":
            parity.compare_reduction(sides[k], oracle.evaluate(prog, hs, "f32"), "f32", what)


def test_capture_of_an_uncompiled_tree_is_refused():
    n = 64
    A = parity.rand(n, n, "f32", seed=9)
    ctx = coot.context()
    s = torch.cuda.Stream()
    # a tree this process has never compiled (a unique scalar count)
    e = coot.Mat(A)
    for _ in range(13):
        e = 1.0 + e
    tree, lm, cm = coot.lower(coot.sqrt(coot.abs(e)))
    out = torch.empty((n, n), dtype=torch.float32, device="cuda").t()
    L.coot_graph_begin(ctx, s.cuda_stream)
    with pytest.raises(L.CootError, match="coot_warmup"):
        L.coot_eval(ctx, tree, cm, coot.Mat(out).cmat(), L.reduce(), None, s.cuda_stream)
    try:
        L.coot_graph_end(ctx, s.cuda_stream)
    except L.CootError:
        pass
    torch.cuda.synchronize()


@pytest.mark.parametrize("n", [64, 333])
def test_adjoint_matches_oracle_gradient(n):
    W, X, Y = workloads.differentiation(n=n, device="cuda")
    Wp, Xp = W.clone().requires_grad_(True), X.clone().requires_grad_(True)
    loss = loss_l2_schur(Wp, Xp, Y, 1e-3)
    loss.backward()
    torch.cuda.synchronize()
    prog = "A B % C - square #0.001 A square * + accu"
    hs = parity.host([W, X, Y])
    lo, (gW, gX, _), (aW, aX, _) = oracle.grad(prog, hs, "f32")
    # the loss under the suite's FP32 reduction tolerance (1e-6 relative plus
    # the tree's propagated element bounds)
    rf = oracle.evaluate(prog, hs, "f32")
    assert abs(rf.value[0, 0] - lo) <= 1e-15 * abs(lo)  # the gradient sweep's loss is the forward's
    parity.compare_reduction(loss.detach(), rf, "f32", "loss at %d x %d" % (n, n))
    u = 2.0 ** -24
    for g, ref, ab in ((Wp.grad, gW, aW), (Xp.grad, gX, aX)):
        gg = g.double().cpu().numpy()
        # ~10 FP32 roundings along each gradient term
        assert np.all(np.abs(gg - ref) <= 16 * u * ab + 1e-30)


def test_autograd_of_general_trees_matches_torch():
    n = 200
    A = parity.rand(n, 50, "f64", seed=1, kind="uniform", lo=0.5, hi=2.0).requires_grad_(True)
    B = parity.rand(n, 50, "f64", seed=2, kind="uniform", lo=0.5, hi=2.0).requires_grad_(True)
    f = lambda a, b: coot.mean(coot.sqrt(coot.exp(0.5 * a) / (1 + b)) - coot.log(a % b), -1)
    loss = scalar(f, A, B)
    loss.backward()
    A2 = A.detach().clone().requires_grad_(True)
    B2 = B.detach().clone().requires_grad_(True)
    ref = (torch.sqrt(torch.exp(0.5 * A2) / (1 + B2)) - torch.log(A2 * B2)).mean()
    ref.backward()
    assert abs(loss.item() - ref.item()) <= 1e-13 * abs(ref.item())
    assert torch.allclose(A.grad, A2.grad, rtol=1e-12, atol=1e-15)
    assert torch.allclose(B.grad, B2.grad, rtol=1e-12, atol=1e-15)


def test_disk_cache_corruption_recompiles(tmp_path, monkeypatch):
    monkeypatch.setenv("COOT_CACHE_DIR", str(tmp_path))
    ctx = L.coot_ctx_create(0, 0)
    try:
        A = parity.rand(100, 10, "f32", seed=4)
        e = 3.0 - coot.sqrt(coot.abs(coot.Mat(A)))
        tree, lm, cm = coot.lower(e)
        out = torch.empty((10, 100), dtype=torch.float32, device="cuda").t()
        s = torch.cuda.current_stream().cuda_stream
        L.coot_eval(ctx, tree, cm, coot.Mat(out).cmat(), L.reduce(), None, s)
        torch.cuda.synchronize()
        ref = out.clone()
        files = glob.glob(str(tmp_path / "*.cubin"))
        assert len(files) == 1
        with open(files[0], "r+b") as f:  # flip payload bytes
            f.seek(200)
            f.write(b"\x00\xff" * 32)
    finally:
        L.coot_ctx_destroy(ctx)
    ctx = L.coot_ctx_create(0, 0)
    try:
        out.zero_()
        L.coot_eval(ctx, tree, cm, coot.Mat(out).cmat(), L.reduce(), None, s)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        # truncated entry
        with open(files[0], "r+b") as f:
            f.truncate(100)
    finally:
        L.coot_ctx_destroy(ctx)
    ctx = L.coot_ctx_create(0, 0)
    try:
        out.zero_()
        L.coot_eval(ctx, tree, cm, coot.Mat(out).cmat(), L.reduce(), None, s)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        L.coot_ctx_destroy(ctx)
