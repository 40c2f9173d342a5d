"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (autotuned context): element-wise results on sampled output
blocks (an element depends only on the inputs at the same index, or the
transposed index for trans reads, so a block of the inputs gives the oracle
that block of the output), reductions against the oracle over all elements."""
import numpy as np
import pytest
import torch

import oracle
import parity
import paper_2508_11385_gb300 as coot
from paper_2508_11385_gb300 import lib as L
from paper_2508_11385_gb300 import workloads

pytestmark = pytest.mark.gpu

import bench  # noqa: E402  (the benchmark's tree list and prepared calls)


@pytest.fixture(scope="module")
def tuned_ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = L.coot_ctx_create(0, L.CTX_TUNE)
    yield ctx
    L.coot_ctx_destroy(ctx)


def _blocks(n, b=48):
    return [(0, 0), (n - b, n - b), (n // 2 - 7, 123), (1000, n - b)]


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
def test_large_trees_full_size(tuned_ctx, dtype):
    n = bench.N_MAIN
    leaves = workloads.large_trees(dtype, n=n, device="cuda")
    host_cache = {}
    for name, prog, _ in bench.TREES:
        if dtype == "i32" and "exp" in prog:
            continue
        if dtype != "f32" and name.startswith("L"):
            continue
        c = bench.Call(prog, leaves, True, ctx=tuned_ctx)
        c(torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        res = c.result()
        toks = prog.split()
        used = sorted({t for t in toks if len(t) == 1 and "A" <= t <= "H"})
        if toks[-1] == "sum:0":
            cols = [0, 1, n // 2, n - 1]
            for j in cols:
                sub = [leaves[ord(t) - 65][:, j:j + 1] for t in used]
                rr = oracle.evaluate(prog, parity.host(sub), dtype)
                parity.compare_reduction(res[:, j:j + 1], rr, dtype, name)
            continue
        if toks[-1] == "accu":
            rr = oracle.evaluate(prog, parity.host([leaves[0]]), dtype)
            parity.compare_reduction(res, rr, dtype, name)
            continue
        b = 48
        for r0, c0 in _blocks(n, b):
            sub = []
            for t in used:
                x = leaves[ord(t) - 65]
                if "trans" in toks and t == "A":
                    sub.append(x[c0:c0 + b, r0:r0 + b])
                else:
                    sub.append(x[r0:r0 + b, c0:c0 + b])
            ry = oracle.evaluate(prog, parity.host(sub), dtype)
            parity.compare_matrix(res[r0:r0 + b, c0:c0 + b], ry, dtype, "%s block (%d,%d)" % (name, r0, c0))
    del leaves
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_precision_reductions_full_size(dtype):
    n = 1 << 28
    x, y = workloads.precision(dtype, n=n, device="cuda")
    X, Y = coot.Mat(x), coot.Mat(y)
    hx, hy = parity.host([x, y])
    for prog, red in (("A accu", coot.accu(X)), ("A B dot", coot.dot(X, Y)), ("A norm", coot.norm(X)),
                      ("A var", coot.var(X))):
        r = red.eval()
        torch.cuda.synchronize()
        rr = oracle.evaluate(prog, [hx, hy], dtype)
        parity.compare_reduction(r, rr, dtype, "%s %s" % (dtype, prog))
    del x, y
    torch.cuda.empty_cache()


def test_fp64_var_full_size():
    n = 1 << 28
    x, _ = workloads.precision("f64", n=n, device="cuda")
    r = coot.var(coot.Mat(x)).eval()
    torch.cuda.synchronize()
    rr = oracle.evaluate("A var", parity.host([x]), "f64")
    parity.compare_reduction(r, rr, "f64", "f64 var")
    del x
    torch.cuda.empty_cache()


def test_batching_full_size_sampled():
    npb = 50000
    rows, cols, A, B, C, pools = workloads.batching(npb, device="cuda")
    outs = [torch.empty((c, r), dtype=torch.float32, device="cuda").t() for r, c in zip(rows.tolist(), cols.tolist())]
    probs = (L.coot_mat * (3 * npb))()
    for q in range(npb):
        probs[3 * q] = coot.Mat(A[q]).cmat()
        probs[3 * q + 1] = coot.Mat(B[q]).cmat()
        probs[3 * q + 2] = coot.Mat(C[q]).cmat()
    outm = (L.coot_mat * npb)(*[coot.Mat(o).cmat() for o in outs])
    res = torch.empty(npb, dtype=torch.float32, device="cuda")
    nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_LEAF, leaf=1), L.node(L.N_SCHUR, a=0, b=1),
             L.node(L.N_LEAF, leaf=2), L.node(L.N_TRANS, a=3), L.node(L.N_SCAL_TIMES, a=4, k=0.1),
             L.node(L.N_PLUS, a=2, b=5)]
    plan = L.coot_batch_create(coot.context(), L.make_tree(nodes), npb, 3, probs, outm, L.reduce(L.R_ACCU))
    L.coot_batch_run(plan, res.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    L.coot_batch_destroy(plan)
    assert torch.isfinite(res).all()
    rng = np.random.default_rng(0)
    for q in sorted(set(rng.integers(0, npb, 300).tolist()) | {0, npb - 1}):
        hs = parity.host([A[q], B[q], C[q]])
        ry = oracle.evaluate("A B % C trans #0.1 * +", hs, "f32")
        parity.compare_matrix(outs[q], ry, "f32", "problem %d" % q)
        rr = oracle.evaluate("A B % C trans #0.1 * + accu", hs, "f32")
        parity.compare_reduction(res[q:q + 1], rr, "f32", "problem %d" % q)


def test_differentiation_full_size_sampled():
    from paper_2508_11385_gb300.autograd import loss_l2_schur

    W, X, Y = workloads.differentiation(device="cuda")
    Wp, Xp = W.clone().requires_grad_(True), X.clone().requires_grad_(True)
    loss = loss_l2_schur(Wp, Xp, Y, 1e-3)
    loss.backward()
    torch.cuda.synchronize()
    prog = "A B % C - square #0.001 A square * + accu"
    rr = oracle.evaluate(prog, parity.host([W, X, Y]), "f32")
    parity.compare_reduction(loss.detach(), rr, "f32", "loss")
    u = 2.0 ** -24
    n, b = W.shape[0], 64
    for r0, c0 in [(0, 0), (n - b, n - b), (1234, 2345)]:
        blk = [t[r0:r0 + b, c0:c0 + b] for t in (W, X, Y)]
        _, (gW, gX, _), (aW, aX, _) = oracle.grad(prog, parity.host(blk), "f32")
        for g, ref, ab in ((Wp.grad, gW, aW), (Xp.grad, gX, aX)):
            gg = g[r0:r0 + b, c0:c0 + b].double().cpu().numpy()
            assert np.all(np.abs(gg - ref) <= 16 * u * ab + 1e-30)


def test_stored_tuning_names_its_kernel(tmp_path, monkeypatch, capfd):
    # the tuning file stores the chosen kernel's name beside its index; an
    # entry whose name no longer matches the program's kernel at that index
    # (a program whose variant list changed) is ignored and the call re-tuned
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setenv("COOT_CACHE_DIR", str(tmp_path))
    leaves = workloads.large_trees("f32", n=1024, n_leaves=3, device="cuda")
    prog = "A B % C + sum:1"
    sp = torch.cuda.current_stream().cuda_stream

    def run(flags):
        ctx = L.coot_ctx_create(0, flags)
        try:
            bench.Call(prog, leaves, True, ctx=ctx)(sp)
            torch.cuda.synchronize()
        finally:
            L.coot_ctx_destroy(ctx)

    run(L.CTX_TUNE)
    files = list(tmp_path.glob("tune-*.txt"))
    assert len(files) == 1
    lines = [ln for ln in files[0].read_text().splitlines() if ln.strip()]
    assert lines and all(len(ln.split("\t")[1].split()) == 5 for ln in lines)
    assert all(ln.split()[-1].startswith("coot_") for ln in lines)
    capfd.readouterr()
    run(L.CTX_TUNE | L.CTX_LOG)  # the stored entry is used: no candidates timed
    assert "candidate" not in capfd.readouterr().err
    files[0].write_text("".join(ln.rsplit(" ", 1)[0] + " coot_no_such_kernel\n" for ln in lines))
    run(L.CTX_TUNE | L.CTX_LOG)  # a stale name: tuned again
    assert "candidate" in capfd.readouterr().err
