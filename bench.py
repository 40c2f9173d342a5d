#!/usr/bin/env python
"""Benchmark: fused expression-tree evaluation on GB300, effective HBM GB/s.

Workload (one "step"): the large memory-bound trees on FP32 8192 x 8192
column-major matrices A..F drawn normal(0,1) -- the six tree shapes
  2*A+B,  A%B+C,  trans(A)+B,  exp(A-B)/(1+abs(C)),  sum(square(A-B),0),
  accu(A.submat(1000,1000,5095,5095))
and the depth ladder
  L4 = exp(A-B)/(1+abs(C)) % D, L5 = L4 - E, L6 = abs(L5), L7 = sqrt(L6),
  L8 = L7 % F
each evaluated once by one fused kernel.  value = sum of algorithmic bytes
(distinct operand bytes read + bytes written) / device time of the step.

Besides the headline line the JSON carries: the unfused one-kernel-per-op
path on the same trees (GB/s and the speed-up per tree), FP64 and INT32
variants, the batched workload (exprs/s), the CUDA-graph chain, the fused
adjoint, the roofline of the dominant kernel against the measured HBM copy
peak, SM clocks sampled during the timed region, an end-to-end number through
host buffers, and the FP64 CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused-expr effective HBM GB/s (fraction of peak) vs unfused per-op; batched exprs/s"
N_MAIN = 8192
FALLBACK_HBM = 6800.0

# (name, RPN program over A..F, depth) -- the config-2 shapes and the ladder
TREES = [
    ("axpy", "#2 A * B +", 2),
    ("schur_plus", "A B % C +", 2),
    ("trans_plus", "A trans B +", 2),
    ("exp_div", "A B - exp #1 C abs + /", 4),
    ("colsum_sq", "A B - square sum:0", 3),
    ("accu_submat", "A submat:1000:1000:4096:4096 accu", 2),
    ("L4", "A B - exp #1 C abs + / D %", 5),
    ("L5", "A B - exp #1 C abs + / D % E -", 6),
    ("L6", "A B - exp #1 C abs + / D % E - abs", 7),
    ("L7", "A B - exp #1 C abs + / D % E - abs sqrt", 8),
    ("L8", "A B - exp #1 C abs + / D % E - abs sqrt F %", 9),
]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured", d
    except Exception:
        return FALLBACK_HBM, "fallback", {}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def reduce_max(x, world, device=None):
    """max over ranks (replicas: a barrier and a max of the timings only)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(per_rank_units, per_rank_seconds):
    """Whole-job throughput of independent replicas: all units over the
    slowest rank's time."""
    return sum(per_rank_units) / max(per_rank_seconds)


# ---------------------------------------------------------------------------
# the program-string front end used by the bench (same trees as the tests)
# ---------------------------------------------------------------------------
def build_expr(program, mats):
    import paper_2508_11385_gb300 as coot

    st, red = [], None
    for tok in program.split():
        if len(tok) == 1 and "A" <= tok <= "H":
            st.append(mats[ord(tok) - ord("A")])
        elif tok.startswith("#"):
            st.append(float(tok[1:]))
        elif tok in ("+", "-", "%", "/", "*"):
            y, x = st.pop(), st.pop()
            st.append({"+": lambda a, b: a + b, "-": lambda a, b: a - b, "%": lambda a, b: a % b,
                       "/": lambda a, b: a / b, "*": lambda a, b: a * b}[tok](x, y))
        elif tok in ("exp", "log", "abs", "square", "sqrt", "trans"):
            st.append(getattr(coot, tok)(st.pop()))
        elif tok == "neg":
            st.append(-st.pop())
        elif tok.startswith("submat:"):
            r0, c0, nr, nc = map(int, tok.split(":")[1:])
            st.append(st.pop().submat(r0, c0, r0 + nr - 1, c0 + nc - 1))
        elif tok == "accu":
            red = coot.accu(st[-1])
        elif tok == "sum:0":
            red = coot.sum(st[-1], 0)
        elif tok == "sum:1":
            red = coot.sum(st[-1], 1)
        elif tok == "mean":
            red = coot.mean(st[-1], -1)
        elif tok == "norm":
            red = coot.norm(st[-1])
        elif tok == "norm:fro":
            red = coot.norm(st[-1], "fro")
        elif tok in ("var", "var:1"):
            red = coot.var(st[-1], 1 if tok == "var:1" else 0)
        elif tok in ("stddev", "stddev:1"):
            red = coot.stddev(st[-1], 1 if tok == "stddev:1" else 0)
        elif tok.partition(":")[0] in ("min", "max", "index_min", "index_max", "prod"):
            head, _, d = tok.partition(":")
            red = getattr(coot, head)(st[-1], int(d) if d else -1)
        elif tok.startswith("each_col:"):
            st.append(coot.broadcast_col(st.pop(), int(tok.split(":")[1])))
        elif tok.startswith("each_row:"):
            st.append(coot.broadcast_row(st.pop(), int(tok.split(":")[1])))
        elif tok == "diag" or tok.startswith("diag:"):
            st.append(st.pop().diag(int(tok.split(":")[1]) if ":" in tok else 0))
        elif tok.partition(":")[0] == "cumsum":
            d = tok.partition(":")[2]
            red = coot.cumsum(st[-1], int(d) if d else None)
        elif tok.partition(":")[0] in ("vardim", "stddevdim"):
            head, _, rest = tok.partition(":")
            d, nt = map(int, rest.split(":"))
            red = (coot.var if head == "vardim" else coot.stddev)(st[-1], nt, d)
        elif tok == "dot":
            b, a = st.pop(), st.pop()
            red = coot.dot(a, b)
            st.append(red.expr)
        else:
            raise ValueError(tok)
    return st[-1], red


class Call:
    """A prepared C-ABI call: descriptor, leaf matrices, output, reduction."""

    def __init__(self, program, tensors, fused=True, ctx=None):
        import torch

        import paper_2508_11385_gb300 as coot
        from paper_2508_11385_gb300 import expr as E
        from paper_2508_11385_gb300 import lib as L

        self.L, self.coot = L, coot
        mats = [coot.Mat(t) for t in tensors]
        e, red = build_expr(program, mats)
        self.tree, self.leaf_mats, self.cmats = E.lower(e)
        self.fused = fused
        nr, nc = e.shape
        dt = self.leaf_mats[0].dtype
        dev = tensors[0].device
        if red is None or red.kind == L.R_CUMSUM:
            # element-wise result, or a scan written where it would be
            self.out_t = torch.empty((nc, nr), dtype=tensors[0].dtype, device=dev).t()
            self.out_m = coot.Mat(self.out_t).cmat()
            self.red = L.reduce() if red is None else L.reduce(red.kind, red.dim)
            self.red_t = None
        else:
            self.out_t, self.out_m = None, None
            self.red = L.reduce(red.kind, red.dim, red.norm_type)
            acc = torch.int64 if red.kind in (L.R_INDEX_MIN, L.R_INDEX_MAX) else E._ACC[dt]
            if red.dim == 0:
                self.red_t = torch.empty((1, nc), dtype=acc, device=dev)
            elif red.dim == 1:
                self.red_t = torch.empty((nr, 1), dtype=acc, device=dev)
            else:
                self.red_t = torch.empty((), dtype=acc, device=dev)
        self.ctx = E.context(dev) if ctx is None else ctx
        self.red_ptr = self.red_t.data_ptr() if self.red_t is not None else None
        self.fn = L.coot_eval if fused else L.coot_eval_unfused
        self.leaf_tensors = [m.tensor for m in self.leaf_mats]

    def __call__(self, stream_ptr):
        self.fn(self.ctx, self.tree, self.cmats, self.out_m, self.red, self.red_ptr, stream_ptr)

    def info(self):
        return self.L.coot_last_launch(self.ctx)

    def result(self):
        return self.out_t if self.red_t is None else self.red_t


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        # the raw samples: $COOT_CLOCKS_CSV, else a file in the temporary directory
        self.path = path or os.environ.get("COOT_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), "cootgb_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform

    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, timeout=10).stdout.decode()
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Model Name") and v.strip():
                return v.strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            if k.strip() in ("model name", "Model") and v.strip():
                return v.strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_rate(host, n, budget_s, parallel):
    """GB/s of the oracle over the workload's trees at n x n (the view scaled
    with n), repeated until about budget_s of evaluation time."""
    import oracle

    scale = n / N_MAIN
    done_bytes, t_total, evals = 0, 0.0, 0
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s:
        for name, prog, _ in TREES:
            p = prog.replace("submat:1000:1000:4096:4096",
                             "submat:%d:%d:%d:%d" % (int(1000 * scale), int(1000 * scale),
                                                    int(4096 * scale), int(4096 * scale)))
            t0 = time.perf_counter()
            oracle.evaluate(p, host, "f32", parallel=parallel)
            t_total += time.perf_counter() - t0
            done_bytes += algorithmic_bytes(p, n, 4)
            evals += 1
        if evals >= len(TREES) and time.perf_counter() - t_start > budget_s * 0.5:
            break
    return done_bytes / t_total / 1e9, evals, t_total


def cpu_baseline(n=2048, budget_s=20.0):
    """The FP64 oracle on a bounded sample of the workload: single-threaded,
    and (when the OpenMP build exists) with its element-wise loops on all
    host cores.  `value` and `cores` are the all-core run's when there is one."""
    import oracle
    from paper_2508_11385_gb300 import workloads

    oracle.build()
    leaves = workloads.large_trees("f32", n=n, device="cpu")
    host = [workloads.to_numpy_colmajor(t) for t in leaves]
    scale = n / N_MAIN
    v1, e1, t1 = _oracle_rate(host, n, budget_s / 2, False)
    out = {"value": v1, "unit": "GB/s", "cores": 1, "kind": "oracle", "host_cpus": os.cpu_count(),
           "cpu_model": cpu_model(), "single_thread": {"value": v1, "cores": 1, "evals": e1, "seconds": round(t1, 2)}}
    try:
        cores = oracle.threads(parallel=True)
        vp, ep, tp = _oracle_rate(host, n, budget_s / 2, True)
        out.update({"value": vp, "cores": cores,
                    "all_cores": {"value": vp, "cores": cores, "evals": ep, "seconds": round(tp, 2)}})
    except oracle.OracleError as e:
        out["all_cores"] = {"unavailable": str(e)}
    out["sample"] = ("the %d trees of the workload at %dx%d FP32 (1/%d of the elements); C FP64 oracle, "
                     "single-threaded (%d evaluations) and with its element-wise loops on %s threads "
                     "(reductions sequential, results bit-identical)" % (
                         len(TREES), n, n, int(1 / scale ** 2), e1, out["cores"] if "all_cores" in out and
                         "value" in out["all_cores"] else "no"))
    return out


def algorithmic_bytes(program, n, esz):
    """distinct operand bytes read + bytes written, for the workload's programs"""
    toks = program.split()
    leaves = {t for t in toks if len(t) == 1 and "A" <= t <= "H"}
    if any(t.startswith("submat:") for t in toks):
        nr, nc = [int(x) for x in [t for t in toks if t.startswith("submat:")][0].split(":")[3:5]]
        return nr * nc * esz + 4
    b = len(leaves) * n * n * esz
    if toks[-1] == "sum:0":
        return b + n * 4
    if toks[-1] == "accu":
        return b + 4
    return b + n * n * esz


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_side(args):
    """One side workload alone (for profiling): prints its JSON."""
    import torch

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__

    __graft_entry__.build()
    os.environ.setdefault("COOT_TUNE", "on")
    stream = torch.cuda.current_stream(dev)
    fn = {"batched": lambda: bench_batched(args, dev, stream), "adjoint": lambda: bench_adjoint(dev, stream),
          "precision": lambda: bench_precision(dev, stream, errors=args.precision_errors),
          "graph_chain": lambda: bench_graph(dev, stream), "stats": lambda: bench_stats(args, dev, stream),
          "gemm": lambda: bench_gemm(args, dev, stream), "e2e": lambda: bench_e2e(args, dev, stream),
          "e2e_zero_copy": lambda: bench_e2e(args, dev, stream, zero_copy=True),
          "probe": lambda: bench_probe(dev)}[args.only]
    print(json.dumps({args.only: fn()}))


def bench_e2e(args, dev, stream, zero_copy=False):
    """The end-to-end measurement of the headline step alone (the trees'
    calls prepared and tuned first, untimed)."""
    import torch

    from paper_2508_11385_gb300 import workloads

    leaves = workloads.large_trees("f32", n=args.n, device=dev)
    calls = [(name, prog, depth, Call(prog, leaves, True)) for name, prog, depth in TREES]
    for _ in range(2):
        for _, _, _, c in calls:
            c(stream.cuda_stream)
    torch.cuda.synchronize()
    if zero_copy:
        return run_e2e_zero_copy(calls, leaves, stream, max(2, min(args.steps, 5)))
    return run_e2e(calls, leaves, stream, max(2, min(args.steps, 5)), dev, args.h2d_streams)


def run_prog(args):
    """One RPN program alone over the workload's leaves (for profiling): A..F
    are FP32 n x n; a leaf followed by each_col:n / each_row:n is cut to a
    column / row.  Default launch configuration (no tuning unless COOT_TUNE
    is set): `steps` calls timed after `warmup`."""
    import torch

    from paper_2508_11385_gb300 import workloads

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__

    __graft_entry__.build()
    stream = torch.cuda.current_stream(dev)
    lv = workloads.large_trees(args.prog_dtype, n=args.n, n_leaves=6, device=dev, m=args.prog_cols)
    toks = args.prog.split()
    for i, t in enumerate(toks[:-1]):
        if len(t) == 1 and "A" <= t <= "F":
            li = ord(t) - ord("A")
            if toks[i + 1].startswith("each_col:"):
                lv[li] = lv[li][:, :1]
            elif toks[i + 1].startswith("each_row:"):
                lv[li] = lv[li][:1, :]
    c = Call(args.prog, lv)
    sp = stream.cuda_stream
    for _ in range(args.warmup):
        c(sp)
    torch.cuda.synchronize()
    flush = None
    if args.flush:  # every call alone after a buffer twice the L2 size is read through L2
        flush = torch.empty(2 * torch.cuda.get_device_properties(dev).L2_cache_size, dtype=torch.uint8, device=dev)
    ms = time_calls(lambda: c(sp), stream, reps=args.steps, warm=0, flush=flush)
    info = c.info()
    print(json.dumps({"prog": args.prog, "ms": round(ms, 4), "gbs": round(info["algorithmic_bytes"] / ms / 1e6, 1),
                      "kernel": info["kernel"], "grid": info["grid"], "block": info["block"]}))


def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2508_11385_gb300 import lib as L
    from paper_2508_11385_gb300 import workloads

    os.environ.setdefault("COOT_TUNE", "on")
    n = args.n
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    leaves = workloads.large_trees("f32", n=n, device=dev)
    calls = [(name, prog, depth, Call(prog, leaves, True)) for name, prog, depth in TREES
             if not args.only or name == args.only]
    # warm the JIT and tuning caches (excluded from timing, as the paper's startup is)
    for _, _, _, c in calls:
        c(sp)
    torch.cuda.synchronize()
    bytes_per, kernel_of = {}, {}
    launches_per_step = 0
    for name, _, _, c in calls:
        c(sp)
        info = c.info()
        bytes_per[name] = info["algorithmic_bytes"]
        kernel_of[name] = "%s grid %d x %d" % (info["kernel"], info["grid"], info["block"])
    torch.cuda.synchronize()
    for name, _, _, c in calls:
        c(sp)
        launches_per_step += c.info()["n_launches"]
    torch.cuda.synchronize()

    # timed region: K steps, events around every tree's launch on its stream;
    # the clock sampler starts first and the W warm-up steps run right before
    # the timed ones, so the GPU is busy and at speed when timing starts
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in calls]
          for _ in range(args.steps)]
    clock = ClockSampler(local)
    clock.start()
    time.sleep(0.2)
    for _ in range(args.warmup):
        for _, _, _, c in calls:
            c(sp)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        for i, (_, _, _, c) in enumerate(calls):
            ev[k][i][0].record(stream)
            c(sp)
            ev[k][i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clock.stop()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    total_ms = reduce_max(total_ms, world, dev)
    step_bytes = sum(bytes_per.values())
    per_tree_ms = {name: statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
                   for i, (name, _, _, _) in enumerate(calls)}
    value = world * step_bytes * args.steps / (total_ms / 1e3) / 1e9
    peak, peak_kind, peaks = load_peaks()

    # dominant kernel: largest share of the step
    dom = max(per_tree_ms, key=per_tree_ms.get)
    dom_call = [c for name, _, _, c in calls if name == dom][0]
    dom_call(sp)
    torch.cuda.synchronize()
    dom_info = dom_call.info()
    achieved = bytes_per[dom] / (per_tree_ms[dom] / 1e3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            ent = tr.get(dom)
            if ent and ent.get("headers_sha") == headers_sha():
                traffic = ent["dram_bytes_per_launch"]
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": dom_info["kernel"],
                "tree": dom, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s"}

    # end to end through host buffers: H2D of each tree's operands, eval, D2H of
    # its result (copy engines); and the kernels reading and writing pinned host
    # memory directly.  `value` is the faster route's, both are listed.
    e2e = None
    probe = None
    if rank == 0 and not args.quick:
        try:
            probe = bench_probe(dev)
        except Exception as ex:  # reported, not hidden
            probe = {"error": repr(ex)[:300]}
        e2e = run_e2e(calls, leaves, stream, max(2, min(args.steps, 5)), dev, args.h2d_streams)
        try:
            zc = run_e2e_zero_copy(calls, leaves, stream, max(2, min(args.steps, 5)))
        except Exception as ex:  # reported, not hidden
            zc = {"error": repr(ex)[:300]}
        e2e = {"route": "copy engines", **e2e, "copy_engines": dict(e2e), "zero_copy": zc}
        if zc.get("value") and zc.get("results_equal_device_run") and zc["value"] > e2e["value"]:
            e2e.update({"route": "zero copy", "value": zc["value"], "h2d_bytes_per_step": zc["h2d_bytes_per_step"],
                        "d2h_bytes_per_step": zc["d2h_bytes_per_step"], "note": zc["note"]})
        if probe and probe.get("host_read_gbs"):
            # the host link as kernels see it (probed): reads and writes overlap,
            # so a step takes at least the longer of the two
            t = max(e2e["h2d_bytes_per_step"] / (probe["host_read_gbs"] * 1e9),
                    e2e["d2h_bytes_per_step"] / (probe["host_write_gbs"] * 1e9))
            bound = (e2e["h2d_bytes_per_step"] + e2e["d2h_bytes_per_step"]) / t / 1e9
            e2e["roofline"] = {"bound": "host link", "bound_gbs": round(bound, 1),
                               "frac": round(e2e["value"] / bound, 4),
                               "peaks": "probed kernel read %.1f / write %.1f GB/s of pinned host memory" % (
                                   probe["host_read_gbs"], probe["host_write_gbs"])}

    extras = {}
    if rank == 0 and not args.quick:
        extras = run_extras(args, leaves, calls, per_tree_ms, bytes_per, dev, stream, peak, probe)

    out = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded normal(0,1) FP32 matrices generated on the device)",
        "config": {"workload": "large memory-bound trees, FP32 %dx%d A..F: 6 shapes + depth ladder L4-L8" % (n, n),
                   "trees": [t[0] for t in TREES], "l2": "inputs larger than L2 (each operand %d MiB; between two runs of a "
                   "tree the others stream GBs); the per-tree side comparisons read a buffer twice the "
                   "L2 size before every timed call" % (n * n * 4 >> 20), "parallelism": "replicas" if world > 1 else "single GPU"},
        "frac_of_peak": round(value / world / peak, 4),
        "peak_gbs": peak,
        "roofline": roofline,
        "per_tree": {name: {"ms": round(per_tree_ms[name], 4), "gbs": round(bytes_per[name] / per_tree_ms[name] / 1e6, 1),
                            "bytes": bytes_per[name], "kernel": kernel_of[name]} for name in per_tree_ms},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    out.update(extras)
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# the device sources the streaming kernels (str, col, row, tile, scan, batch,
# adj) are compiled from; the GEMM header is not among them
STREAMING_HEADERS = ("coot_params.h", "coot_dev.cuh", "coot_kernels.cuh")


def headers_sha():
    """Hash of the streaming kernels' device sources: a stored ncu traffic
    figure is used only while they are unchanged."""
    h = hashlib.sha256()
    for name in STREAMING_HEADERS:
        h.update(open(os.path.join(ROOT, "paper_2508_11385_gb300", "csrc", "dev", name), "rb").read())
    return h.hexdigest()[:16]


def time_calls(fn, stream, reps=10, warm=2, flush=None):
    """Device time of one call: `reps` calls enqueued back to back between two
    events (the host prepares call k+1 while the GPU runs call k, so host
    overhead is not counted), averaged; the median of three such batches.
    With `flush` (a device buffer larger than L2), every call is timed alone
    after the buffer is read through L2 (its clean lines replace the cache's
    contents, so no dirty line is written back inside the timed call), and the
    median is returned: operands
    that fit in L2 are then read from HBM, as in the headline step."""
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    if flush is not None:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush.sum(dtype=torch.int32)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)
    ts = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / reps)
    return statistics.median(ts)


def run_e2e(calls, leaves, stream, reps, dev, h2d_streams=1):
    """Every tree of every step through host buffers: H2D of its operands from
    pinned host memory, the fused C-ABI call, D2H of its result.  Two device
    copies of the operands and of the prepared calls alternate, so the next
    tree's operands move host->device (on `h2d_streams` copy streams, the
    operands dealt out in turn) while the current tree runs (the bench
    stream) and the previous result moves device->host (one more stream);
    events order each buffer's reuse."""
    import torch

    # column-major device matrices are transposes of contiguous buffers: copy
    # the buffers whole (one cudaMemcpyAsync each, pinned host memory)
    def dense(t):
        return t.t() if t.dim() == 2 and t.t().is_contiguous() else t

    leaves2 = [torch.empty_like(t) for t in leaves]
    sets = [(leaves, [c for _, _, _, c in calls]),
            (leaves2, [Call(prog, leaves2, fused=True) for _, prog, _, _ in calls])]
    host = [dense(t).cpu().pin_memory() for t in leaves]
    h_out = {}
    for name, _, _, c in calls:
        r = dense(c.result())
        h_out[name] = torch.empty(r.shape, dtype=r.dtype).pin_memory()
    name_to_leaf = {}
    for name, prog, _, c in calls:
        used = sorted({t for t in prog.split() if len(t) == 1 and "A" <= t <= "H"})
        name_to_leaf[name] = [ord(t) - ord("A") for t in used]
    sp = stream.cuda_stream
    for c in sets[1][1]:  # the second set's calls prepared once, untimed
        c(sp)
    torch.cuda.synchronize()
    s_h2ds = [torch.cuda.Stream(device=dev) for _ in range(max(1, h2d_streams))]
    s_d2h = torch.cuda.Stream(device=dev)
    seq = [i for _ in range(reps) for i in range(len(calls))]
    kdone, ddone = [None] * len(seq), [None] * len(seq)
    bytes_alg = h2d = d2h = 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for s_h2d in s_h2ds:
        s_h2d.wait_stream(stream)
    for q, i in enumerate(seq):
        name = calls[i][0]
        lv, cs = sets[q % 2]
        c = cs[i]
        for k, li in enumerate(name_to_leaf[name]):
            s_h2d = s_h2ds[k % len(s_h2ds)]
            if q >= 2:
                s_h2d.wait_event(kdone[q - 2])  # this set's operands were read by step q - 2
            with torch.cuda.stream(s_h2d):
                dense(lv[li]).copy_(host[li], non_blocking=True)
            h2d += host[li].numel() * host[li].element_size()
        for s_h2d in s_h2ds:
            stream.wait_event(s_h2d.record_event())
        if q >= 2:
            stream.wait_event(ddone[q - 2])  # this set's results were read by step q - 2
        c(sp)
        kdone[q] = stream.record_event()
        bytes_alg += c.info()["algorithmic_bytes"]
        s_d2h.wait_event(kdone[q])
        with torch.cuda.stream(s_d2h):
            r = dense(c.result())
            h_out[name].copy_(r, non_blocking=True)
            d2h += r.numel() * r.element_size()
        ddone[q] = s_d2h.record_event()
    for s_h2d in s_h2ds:
        stream.wait_stream(s_h2d)
    stream.wait_stream(s_d2h)
    b.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    del sets, leaves2
    torch.cuda.empty_cache()
    return {"value": round(bytes_alg / sec / 1e9, 1), "unit": "GB/s", "h2d_bytes_per_step": h2d // reps,
            "d2h_bytes_per_step": d2h // reps, "steps": reps,
            "h2d_streams": len(s_h2ds),
            "note": "per tree: pinned host->device copy of its operands, the fused call, device->host copy of Y or "
                    "the reduction, pipelined over two device buffer sets (operand copies on %d stream(s), the "
                    "calls on the bench stream, result copies on one more); value = algorithmic bytes / wall "
                    "time of the whole sequence" % len(s_h2ds)}


def torch_eager_fn(program, tensors):
    """The same tree as eager torch calls, one call per op (the RPN program
    over A..F read as the column-major tensors given)."""
    import torch

    toks = program.split()

    def run():
        st = []
        for tok in toks:
            if len(tok) == 1 and "A" <= tok <= "H":
                st.append(tensors[ord(tok) - ord("A")])
            elif tok.startswith("#"):
                st.append(float(tok[1:]))
            elif tok in ("+", "-", "%", "/", "*"):
                y, x = st.pop(), st.pop()
                st.append({"+": lambda a, b: a + b, "-": lambda a, b: a - b, "%": lambda a, b: a * b,
                           "/": lambda a, b: a / b, "*": lambda a, b: a * b}[tok](x, y))
            elif tok == "trans":
                st.append(st.pop().t())
            elif tok in ("exp", "abs", "sqrt", "square", "log"):
                st.append(getattr(torch, tok)(st.pop()))
            elif tok.startswith("submat:"):
                r0, c0, nr, nc = map(int, tok.split(":")[1:])
                st.append(st.pop()[r0:r0 + nr, c0:c0 + nc])
            elif tok == "accu":
                st.append(torch.sum(st.pop()))
            elif tok == "sum:0":
                st.append(torch.sum(st.pop(), dim=0))
            else:
                raise ValueError(tok)
        return st[-1]

    return run


def bench_probe(dev):
    """Arithmetic and memory rates of the device (coot_probe_device: small
    hand-written kernels timed with CUDA events), in T operations/s and GB/s."""
    from paper_2508_11385_gb300 import lib as L

    r = L.coot_probe_device(dev.index if dev.index is not None else 0)
    out = {k: round(r[k] / 1e12, 4) for k in ("f32_add", "f32_fma", "f32_div", "f32_exp", "f64_add", "f64_fma",
                                             "f64_div", "f64_exp")}
    out.update({"read_gbs": round(r["read_gbs"], 1), "copy_gbs": round(r["copy_gbs"], 1),
                "host_read_gbs": round(r["host_read_gbs"], 1), "host_write_gbs": round(r["host_write_gbs"], 1),
                "l2_bytes": r["l2_bytes"], "sms": r["sms"], "sm_clock_khz": r["sm_clock_khz"],
                "buffer_bytes": r["buffer_bytes"],
                "unit": "T operations/s for f32_* / f64_* (exp: one exp + one FMA per step); GB/s for read/copy",
                "how": "8 independent chains per thread, grid = SMs x occupancy, best of 3 CUDA-event timings; "
                       "16-byte vector read / copy over a buffer of 8x L2, best of 5"})
    return out


# FP64 operations per element of a program (the reduction's accumulation
# included); abs, trans and views use no FP64 arithmetic
_F64_OPS = {"+": "add", "-": "add", "%": "mul", "*": "mul", "/": "div", "exp": "exp", "square": "mul",
            "sqrt": "div", "accu": "add", "sum:0": "add", "sum:1": "add"}


def f64_alu_bound_ms(program, n_elements, probe):
    """Time the FP64 pipe needs for `program` over n_elements: the sum over
    its FP64 operations of n_elements / probed rate (add and mul at the add
    and FMA rates, div at the division rate, exp at the exp+FMA step rate
    less one FMA)."""
    fma = probe["f64_fma"] * 1e12
    per = {"add": 1 / (probe["f64_add"] * 1e12), "mul": 1 / fma, "div": 1 / (probe["f64_div"] * 1e12),
           "exp": max(1 / (probe["f64_exp"] * 1e12) - 1 / fma, 0.0)}
    ops = [_F64_OPS[t] for t in program.split() if t in _F64_OPS]
    return n_elements * sum(per[o] for o in ops) * 1e3, ops


def run_e2e_zero_copy(calls, leaves, stream, reps):
    """The same trees through host buffers without copy-engine copies: the
    operands, Y and the reductions live in pinned host memory, and the fused
    kernels read and write them directly (on a Grace-Blackwell node over
    NVLink-C2C; pinned host memory has a device address under unified
    addressing).  Each byte still crosses the host-device link once per step,
    inside the timed region."""
    import ctypes

    import torch

    def dense(t):
        return t.t() if t.dim() == 2 and t.t().is_contiguous() else t

    def pinned_like(t):
        d = dense(t)
        h = torch.empty(d.shape, dtype=d.dtype).pin_memory()
        return h.t() if d is not t else h

    host = [pinned_like(t) for t in leaves]
    for h, t in zip(host, leaves):
        dense(h).copy_(dense(t))
    hcalls, h2d, d2h = [], 0, 0
    for name, prog, _, c in calls:
        L = c.L
        cm = (L.coot_mat * len(c.cmats))()
        used = set()
        for i, m in enumerate(c.cmats):
            # the same matrix descriptor with the pinned host copy's address
            li = [k for k, t in enumerate(leaves) if t.data_ptr() <= (m.data or 0) < t.data_ptr() + t.numel() *
                  t.element_size()][0]
            off = (m.data - leaves[li].data_ptr())
            cm[i] = L.coot_mat(host[li].data_ptr() + off, m.dtype, m.rs, m.n_rows, m.n_cols, m.ld)
            used.add(li)
        h2d += sum(leaves[li].numel() * leaves[li].element_size() for li in used)
        out_h = pinned_like(c.out_t) if c.out_t is not None else None
        out_m = None
        if out_h is not None:
            om = c.out_m
            out_m = L.coot_mat(out_h.data_ptr(), om.dtype, om.rs, om.n_rows, om.n_cols, om.ld)
            d2h += out_h.numel() * out_h.element_size()
        red_h = torch.empty(c.red_t.shape, dtype=c.red_t.dtype).pin_memory() if c.red_t is not None else None
        if red_h is not None:
            d2h += red_h.numel() * red_h.element_size()
        hcalls.append((c, cm, out_m, red_h, out_h))
    sp = stream.cuda_stream

    def step():
        b = 0
        for c, cm, out_m, red_h, _ in hcalls:
            L = c.L
            L._check(L._lib.coot_eval(c.ctx, ctypes.byref(c.tree), cm, len(c.cmats),
                                      ctypes.byref(out_m) if out_m is not None else None, c.red,
                                      red_h.data_ptr() if red_h is not None else None, sp))
            b += c.info()["algorithmic_bytes"]
        return b

    step()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    nbytes = 0
    for _ in range(reps):
        nbytes += step()
    e.record(stream)
    torch.cuda.synchronize()
    sec = a.elapsed_time(e) / 1e3
    # the results arrived in host memory: check one against the device run
    ok = True
    for (c, _, _, red_h, out_h) in hcalls:
        ref = c.result()
        got = out_h if out_h is not None else red_h
        if not torch.equal(got.to(ref.device).reshape(ref.shape), ref):
            ok = False
    del host
    return {"value": round(nbytes / sec / 1e9, 1), "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": reps, "results_equal_device_run": ok,
            "note": "operands, Y and reductions in pinned host memory, read and written by the fused kernels "
                    "directly (NVLink-C2C); no copy-engine copies"}


def run_extras(args, leaves, calls, per_tree_ms, bytes_per, dev, stream, peak, probe=None):
    import torch

    import paper_2508_11385_gb300 as coot
    from paper_2508_11385_gb300 import lib as L
    from paper_2508_11385_gb300 import workloads

    sp = stream.cuda_stream
    res = {}
    if probe is None:
        try:
            probe = bench_probe(dev)
        except Exception as e:  # reported, not hidden
            probe = {"error": repr(e)[:300]}
    res["probe"] = probe
    if "error" in probe:
        probe = None
    # L2 is refilled with clean lines before every timed call of the per-tree comparisons,
    # so that the 64 MiB view is read from HBM as in the headline step
    flush = torch.empty(2 * torch.cuda.get_device_properties(dev).L2_cache_size, dtype=torch.uint8, device=dev)
    # ---- unfused per-op baseline on the same trees
    unf = {}
    for name, prog, depth, _ in calls:
        c = Call(prog, leaves, fused=False)
        ms = time_calls(lambda: c(sp), stream, reps=max(5, args.steps // 4), flush=flush)
        unf[name] = {"ms": round(ms, 4), "gbs": round(bytes_per[name] / ms / 1e6, 1),
                     "speedup_fused": round(ms / per_tree_ms[name], 2), "depth": depth}
    deep = [unf[n]["speedup_fused"] for n, _, d, _ in calls if d >= 4]
    res["unfused"] = {"per_tree": unf, "geomean_speedup_depth_ge4": round(math.exp(sum(map(math.log, deep)) / len(deep)), 2),
                      "min_speedup_depth_ge4": min(deep)}
    # ---- torch eager: the same ops as torch calls on the same column-major tensors
    te = {}
    for name, prog, depth, _ in calls:
        fn = torch_eager_fn(prog, leaves)
        ms = time_calls(lambda: fn(), stream, reps=max(5, args.steps // 4), flush=flush)
        te[name] = {"ms": round(ms, 4), "gbs": round(bytes_per[name] / ms / 1e6, 1),
                    "speedup_fused": round(ms / per_tree_ms[name], 2), "depth": depth}
    deep = [te[n]["speedup_fused"] for n, _, d, _ in calls if d >= 4]
    res["torch_eager"] = {"per_tree": te, "geomean_speedup_depth_ge4": round(math.exp(sum(map(math.log, deep)) / len(deep)), 2),
                          "note": "each tree as eager torch calls (one kernel per op, temporaries allocated by "
                                  "torch's caching allocator), L2 refilled with clean lines before every timed call"}
    torch.cuda.empty_cache()
    # ---- FP64 / INT32 variants of the six shapes
    del_names = ["axpy", "schur_plus", "trans_plus", "exp_div", "colsum_sq", "accu_submat"]
    for dt in ("f64", "i32"):
        lv = workloads.large_trees(dt, n=args.n, n_leaves=3, device=dev)
        d = {}
        for name, prog, _, _ in calls:
            if name not in del_names or (dt == "i32" and "exp" in prog):
                continue
            c = Call(prog, lv, fused=True)
            c(sp)
            torch.cuda.synchronize()
            ms = time_calls(lambda: c(sp), stream, reps=5, flush=flush)
            b = c.info()["algorithmic_bytes"]
            cu = Call(prog, lv, fused=False)
            msu = time_calls(lambda: cu(sp), stream, reps=3, flush=flush)
            d[name] = {"ms": round(ms, 4), "gbs": round(b / ms / 1e6, 1), "unfused_ms": round(msu, 4)}
            if dt == "f64" and probe is not None:
                # roofline against the larger of the HBM time and the FP64-pipe time
                toks = prog.split()
                sub = [t for t in toks if t.startswith("submat:")]
                ne = (int(sub[0].split(":")[3]) * int(sub[0].split(":")[4])) if sub else args.n * args.n
                alu_ms, ops = f64_alu_bound_ms(prog, ne, probe)
                hbm_ms = b / (peak * 1e6)
                bound_ms = max(alu_ms, hbm_ms)
                d[name]["roofline"] = {"bound": "alu" if alu_ms > hbm_ms else "hbm", "bound_ms": round(bound_ms, 4),
                                       "alu_ms": round(alu_ms, 4), "hbm_ms": round(hbm_ms, 4),
                                       "frac": round(bound_ms / ms, 4), "f64_ops_per_element": ops}
        res[dt] = d
        del lv
        torch.cuda.empty_cache()
    del flush
    # ---- batched: 50,000 problems, Y = A % B + 0.1*trans(C), accu(Y)
    try:
        res["batched"] = bench_batched(args, dev, stream)
    except Exception as e:  # reported, not hidden
        res["batched"] = {"error": repr(e)[:300]}
    torch.cuda.empty_cache()
    try:
        res["graph_chain"] = bench_graph(dev, stream)
    except Exception as e:
        res["graph_chain"] = {"error": repr(e)[:300]}
    try:
        res["adjoint"] = bench_adjoint(dev, stream)
    except Exception as e:
        res["adjoint"] = {"error": repr(e)[:300]}
    try:
        res["precision"] = bench_precision(dev, stream, errors=args.precision_errors)
    except Exception as e:
        res["precision"] = {"error": repr(e)[:300]}
    try:
        res["stats"] = bench_stats(args, dev, stream)
    except Exception as e:
        res["stats"] = {"error": repr(e)[:300]}
    try:
        res["gemm"] = bench_gemm(args, dev, stream)
    except Exception as e:
        res["gemm"] = {"error": repr(e)[:300]}
    return res


STATS = ["accu", "min", "index_max", "prod", "stddev", "sum:0", "min:0", "index_max:0", "prod:0", "vardim:0:0",
         "sum:1", "max:1", "index_min:1", "prod:1", "stddevdim:1:1", "cumsum:0", "cumsum:1"]
STATS_T = ["accu", "sum:0", "index_min:0", "vardim:0:0", "sum:1", "max:1", "prod:1", "vardim:1:1", "cumsum:0", "cumsum:1"]


def bench_gemm(args, dev, stream):
    """trans(X) * Y at 8192^3 BF16 (the paper's implicit-transpose form) with
    a fused epilogue Y = 2 * P + C, through the C ABI; TFLOP/s against the
    measured cuBLAS BF16 peak (burst), beside torch.matmul on the same
    operands."""
    import torch

    import paper_2508_11385_gb300 as coot
    from paper_2508_11385_gb300 import expr as E
    from paper_2508_11385_gb300 import lib as L
    from paper_2508_11385_gb300 import workloads

    _, _, peaks = load_peaks()
    bf_peak = float(peaks.get("bf16_tflops", 1900.0))
    g = workloads.generator(8, dev)
    n = 8192
    X = workloads.normal(n, n, "bf16", g, dev)
    Y = workloads.normal(n, n, "bf16", g, dev)
    Cm = workloads.normal(n, n, "bf16", g, dev)
    out = torch.empty((n, n), dtype=torch.bfloat16, device=dev).t()
    sp = stream.cuda_stream
    ctx = E.context(dev)
    res = {}
    for name, e in (("trans(X)*Y", coot.trans(coot.Mat(X)) * coot.Mat(Y)),
                    ("2*trans(X)*Y + C (fused)", 2 * (coot.trans(coot.Mat(X)) * coot.Mat(Y)) + coot.Mat(Cm)),
                    ("X*Y", coot.Mat(X) * coot.Mat(Y))):
        coot.evaluate(e, out=out)
        torch.cuda.synchronize()
        ms = time_calls(lambda: coot.evaluate(e, out=out), stream, reps=5, warm=1)
        tf = 2.0 * n ** 3 / (ms / 1e3) / 1e12
        res[name] = {"ms": round(ms, 3), "tflops": round(tf, 1), "frac": round(tf / bf_peak, 3),
                     "kernel": L.coot_last_launch(ctx)["kernel"]}
    xt = X.t()
    torch.matmul(xt, Y)
    torch.cuda.synchronize()
    ms = time_calls(lambda: torch.matmul(xt, Y), stream, reps=5, warm=1)
    res["torch.matmul (cuBLAS), same operands"] = {"ms": round(ms, 3), "tflops": round(2.0 * n ** 3 / (ms / 1e3) / 1e12, 1)}
    # FP32 operands on the CUDA cores, beside cuBLAS SGEMM (TF32 off) on the same operands
    xf, yf = X.float(), Y.float()
    outf = torch.empty((n, n), dtype=torch.float32, device=dev).t()
    ef = coot.trans(coot.Mat(xf)) * coot.Mat(yf)
    coot.evaluate(ef, out=outf)
    torch.cuda.synchronize()
    ms = time_calls(lambda: coot.evaluate(ef, out=outf), stream, reps=3, warm=1)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x FMA x max SM clock
    tf = 2.0 * n ** 3 / (ms / 1e3) / 1e12
    res["trans(X)*Y FP32 (CUDA cores)"] = {"ms": round(ms, 3), "tflops": round(tf, 1), "frac": round(tf / fp32_peak, 3),
                                          "bound": "alu", "peak_tflops": round(fp32_peak, 1),
                                          "kernel": L.coot_last_launch(ctx)["kernel"]}
    allow = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    xft = xf.t()
    torch.matmul(xft, yf)
    torch.cuda.synchronize()
    ms = time_calls(lambda: torch.matmul(xft, yf), stream, reps=3, warm=1)
    torch.backends.cuda.matmul.allow_tf32 = allow
    res["torch.matmul FP32 (cuBLAS, TF32 off), same operands"] = {"ms": round(ms, 3),
                                                                   "tflops": round(2.0 * n ** 3 / (ms / 1e3) / 1e12, 1)}
    del xf, yf, outf
    res["peak"] = {"bf16_tflops": bf_peak, "source": "MEASURED_PEAKS.json bf16_tflops (burst)",
                   "path": "BF16: persistent tcgen05 kernel (TMA loads, accumulator in tensor memory), every "
                           "operand layout; mma.sync m16n8k16 only for unaligned operands. FP32: CUDA-core "
                           "kernel, peak derived from FP32 lanes x 2 x max SM clock"}
    del X, Y, Cm, out
    torch.cuda.empty_cache()
    return res


def bench_stats(args, dev, stream, peak=None):
    """Statistics fused onto Y = A % B + C at n x n FP32 (three reads), each
    through a prepared C-ABI call; accu is the additive reference.  Also the
    transposed form Y = trans(A) % B + C along both dims."""
    import torch

    from paper_2508_11385_gb300 import workloads

    peak = peak or load_peaks()[0]
    lv = workloads.large_trees("f32", n=args.n, n_leaves=3, device=dev)
    sp = stream.cuda_stream
    out = {}
    progs = [("A B % C + " + r, r) for r in STATS]
    progs += [("A trans B % C + " + r, "trans " + r) for r in STATS_T]
    # broadcasting: A n x n, B a column, C a row, each repeated over A
    n = args.n
    bv = [lv[0], lv[1][:, :1], lv[2][:1, :]]
    views = [("A B each_col:%d %% C each_row:%d +" % (n, n), "each_col % each_row + (Y)"),
             ("A B each_col:%d %% C each_row:%d + accu" % (n, n), "each_col % each_row + accu"),
             ("A B each_col:%d - square sum:1" % n, "each_col - square sum:1")]
    for prog, name in progs + [(p, "views " + nm) for p, nm in views]:
        c = Call(prog, bv if name.startswith("views") else lv)
        c(sp)
        torch.cuda.synchronize()
        ms = time_calls(lambda: c(sp), stream, reps=10)
        info = c.info()
        gbs = info["algorithmic_bytes"] / ms / 1e6
        out[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 3),
                     "kernel": info["kernel"], "launches": info["n_launches"]}
    del lv, bv
    torch.cuda.empty_cache()
    # cubes: 512 x 512 x 256 FP32 (256 MiB each), reductions within and across
    # slices, each a prepared C-ABI call on the cube's matrix re-view
    import paper_2508_11385_gb300 as coot
    from paper_2508_11385_gb300 import expr as E
    from paper_2508_11385_gb300 import lib as L

    g = workloads.generator(7, dev)
    cq = [coot.cube_empty(512, 512, 256, torch.float32, dev) for _ in range(2)]
    for t in cq:
        t.copy_(torch.randn(t.shape, generator=g, device=dev))
    Q, R = coot.Cube(cq[0]), coot.Cube(cq[1])
    cube_b = 2 * cq[0].numel() * 4
    ctx = E.context(dev)
    for name, mode, dim, nseg, nout in (("cube sum(Q%R, 0)", "cols", 0, 0, 512 * 256),
                                        ("cube sum(Q%R, 1) per slice", "cols", 1, 256, 512 * 256),
                                        ("cube sum(Q%R, 2) across slices", "elems", 1, 0, 512 * 512)):
        e = Q.to_expr(mode) % R.to_expr(mode)
        tree, _, cm = E.lower(e)
        red = L.reduce(L.R_SUM, dim, 0, nseg)
        res = torch.empty(nout, dtype=torch.float32, device=dev)
        fn = lambda: L.coot_eval(ctx, tree, cm, None, red, res.data_ptr(), sp)
        fn()
        torch.cuda.synchronize()
        ms = time_calls(fn, stream, reps=10)
        info = L.coot_last_launch(ctx)
        gbs = info["algorithmic_bytes"] / ms / 1e6
        out[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 3), "kernel": info["kernel"]}
    # each_slice: 256 problems of one persistent batch kernel
    e0 = Q.slice(0) % R.slice(0)
    tree, _, _ = E.lower(e0)
    probs = (L.coot_mat * 512)()
    for q in range(256):
        probs[2 * q] = E.Mat(cq[0][:, :, q]).cmat()
        probs[2 * q + 1] = E.Mat(cq[1][:, :, q]).cmat()
    plan = L.coot_batch_create(ctx, tree, 256, 2, probs, None, L.reduce(L.R_ACCU))
    res = torch.empty(256, dtype=torch.float32, device=dev)
    fn = lambda: L.coot_batch_run(plan, res.data_ptr(), sp)
    fn()
    torch.cuda.synchronize()
    ms = time_calls(fn, stream, reps=10)
    gbs = (cube_b + 256 * 4) / ms / 1e6
    out["cube each_slice accu(Q%R), batched"] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
    L.coot_batch_destroy(plan)
    del cq, Q, R
    torch.cuda.empty_cache()
    return out


def bench_batched(args, dev, stream):
    import torch

    import paper_2508_11385_gb300 as coot
    from paper_2508_11385_gb300 import lib as L
    from paper_2508_11385_gb300 import workloads
    from paper_2508_11385_gb300.expr import context

    npb = args.batch_problems
    rows, cols, A, B, C, pools = workloads.batching(npb, device=dev)
    outs = [torch.empty((c, r), dtype=torch.float32, device=dev).t() for r, c in zip(rows.tolist(), cols.tolist())]
    nodes = [L.node(L.N_LEAF, leaf=0), L.node(L.N_LEAF, leaf=1), L.node(L.N_SCHUR, a=0, b=1),
             L.node(L.N_LEAF, leaf=2), L.node(L.N_TRANS, a=3), L.node(L.N_SCAL_TIMES, a=4, k=0.1),
             L.node(L.N_PLUS, a=2, b=5)]
    tree = L.make_tree(nodes)
    probs = (L.coot_mat * (3 * npb))()
    for q in range(npb):
        probs[3 * q] = coot.Mat(A[q]).cmat()
        probs[3 * q + 1] = coot.Mat(B[q]).cmat()
        probs[3 * q + 2] = coot.Mat(C[q]).cmat()
    outm = (L.coot_mat * npb)(*[coot.Mat(o).cmat() for o in outs])
    red_out = torch.empty(npb, dtype=torch.float32, device=dev)
    ctx = context(dev)
    t0 = time.perf_counter()
    plan = L.coot_batch_create(ctx, tree, npb, 3, probs, outm, L.reduce(L.R_ACCU))
    plan_s = time.perf_counter() - t0
    sp = stream.cuda_stream
    ms = time_calls(lambda: L.coot_batch_run(plan, red_out.data_ptr(), sp), stream, reps=10)
    info = L.coot_last_launch(ctx)
    # 50,000 separate fused launches of the same tree (first 2,000 timed, scaled)
    nsep = min(npb, args.batch_separate)
    if nsep == 0:
        L.coot_batch_destroy(plan)
        return {"n_problems": npb, "ms": round(ms, 4), "exprs_per_s": round(npb / (ms / 1e3), 1),
                "gbs": round(info["algorithmic_bytes"] / ms / 1e6, 1)}
    sep = []
    for q in range(nsep):
        cm = [probs[3 * q], probs[3 * q + 1], probs[3 * q + 2]]
        sep.append((cm, outm[q]))
    r1 = torch.empty((), dtype=torch.float32, device=dev)

    def separate():
        for cm, om in sep:
            L.coot_eval(ctx, tree, cm, om, L.reduce(L.R_ACCU), r1.data_ptr(), sp)

    sep_ms = time_calls(separate, stream, reps=1, warm=1) * npb / nsep
    L.coot_batch_destroy(plan)
    total_elems = int((rows * cols).sum())
    return {"n_problems": npb, "elements": total_elems, "ms": round(ms, 4),
            "exprs_per_s": round(npb / (ms / 1e3), 1), "gbs": round(info["algorithmic_bytes"] / ms / 1e6, 1),
            "algorithmic_bytes": info["algorithmic_bytes"], "plan_create_s": round(plan_s, 3),
            "separate_launches_ms": round(sep_ms, 2), "separate_exprs_per_s": round(npb / (sep_ms / 1e3), 1),
            "speedup_vs_separate": round(sep_ms / ms, 2)}


def bench_graph(dev, stream):
    import torch

    import paper_2508_11385_gb300 as coot
    from paper_2508_11385_gb300 import lib as L
    from paper_2508_11385_gb300 import workloads
    from paper_2508_11385_gb300.expr import context

    A, B, C = workloads.graph_chain(device=dev)
    n = A.shape[0]
    s = torch.cuda.Stream(device=dev)
    X = [torch.empty((n, n), dtype=torch.float32, device=dev).t() for _ in range(21)]
    X[0].copy_(A)
    # the six large-tree shapes; X enters exp(A-B)/(1+abs(C)) as its C operand
    # so that the chain stays finite (as A it overflows FP32 after two cycles)
    shapes = ["#2 X * B +", "X B % C +", "X trans B +", "A B - exp #1 X abs + /", "X B - square", "X"]
    reds = [None, None, None, None, "sum:0", "accu"]
    side = torch.empty((1, n), dtype=torch.float32, device=dev)
    scal = torch.empty((), dtype=torch.float32, device=dev)
    calls = []
    for k in range(20):
        j = k % 6
        if j == 3:
            prog = shapes[j].replace("X", "C")
            ten = [A, B, X[k]]
        else:
            prog = shapes[j].replace("X", "A")
            ten = [X[k], B, C]
        mats = [coot.Mat(t) for t in ten]
        if j == 5:  # accu over the square 2048x2048 view (the whole matrix), X passes through
            e = mats[0].submat(0, 0, n - 1, n - 1)
            tree, lm, cm = coot.lower(e)
            calls.append((tree, cm, coot.Mat(X[k + 1]).cmat(), L.reduce(L.R_ACCU), scal.data_ptr()))
            continue
        e, _ = build_expr(prog, mats)
        tree, lm, cm = coot.lower(e)
        red = L.reduce(L.R_SUM, 0) if reds[j] == "sum:0" else L.reduce()
        calls.append((tree, cm, coot.Mat(X[k + 1]).cmat(), red, side.data_ptr() if reds[j] else None))
    ctx = context(dev)

    def eager(fn=L.coot_eval):
        for tree, cm, om, red, rp in calls:
            fn(ctx, tree, cm, om, red, rp, s.cuda_stream)

    eager()
    torch.cuda.synchronize()
    L.coot_graph_begin(ctx, s.cuda_stream)
    eager()
    g = L.coot_graph_end(ctx, s.cuda_stream)
    ms_graph = time_calls(lambda: L.coot_graph_launch(g, s.cuda_stream), s, reps=20)
    ms_eager = time_calls(eager, s, reps=20)
    ms_unfused = time_calls(lambda: eager(L.coot_eval_unfused), s, reps=5)
    L.coot_graph_destroy(g)
    return {"evals": 20, "n": n, "graph_ms": round(ms_graph, 4), "eager_ms": round(ms_eager, 4),
            "unfused_ms": round(ms_unfused, 4), "graph_exprs_per_s": round(20 / (ms_graph / 1e3), 1),
            "eager_exprs_per_s": round(20 / (ms_eager / 1e3), 1),
            "unfused_exprs_per_s": round(20 / (ms_unfused / 1e3), 1),
            "note": "2048^2 FP32 operands (16 MiB) are L2-resident across the chain"}


def bench_adjoint(dev, stream):
    import torch

    import paper_2508_11385_gb300 as coot
    from paper_2508_11385_gb300 import autograd as AG
    from paper_2508_11385_gb300 import workloads

    W, X, Y = workloads.differentiation(device=dev)
    Wp = W.clone().requires_grad_(True)
    Xp = X.clone().requires_grad_(True)
    f = AG.Loss(lambda w, x, y: coot.accu(coot.square(w % x - y)) + 1e-3 * coot.accu(coot.square(w)), W, X, Y)
    r = torch.empty((), dtype=torch.float32, device=dev)
    one = torch.ones((), dtype=torch.float32, device=dev)
    gW, gX = torch.empty_like(W), torch.empty_like(X)
    from paper_2508_11385_gb300 import lib as L
    from paper_2508_11385_gb300.expr import context

    # kernel times: each C-ABI call captured in a CUDA graph and replayed, so
    # no Python work sits between launches
    f.forward(W, X, Y, out=r)
    f.backward(one, W, X, Y, grads=[gW, gX, None])
    torch.cuda.synchronize()
    ctx = context(dev)
    gs = torch.cuda.Stream(device=dev)
    graphs = []
    for fn in (lambda: f.forward(W, X, Y, out=r), lambda: f.backward(one, W, X, Y, grads=[gW, gX, None])):
        with torch.cuda.stream(gs):
            L.coot_graph_begin(ctx, gs.cuda_stream)
            for _ in range(10):
                fn()
            graphs.append(L.coot_graph_end(ctx, gs.cuda_stream))
    ms_fwd = time_calls(lambda: L.coot_graph_launch(graphs[0], gs.cuda_stream), gs, reps=10) / 10
    ms_bwd = time_calls(lambda: L.coot_graph_launch(graphs[1], gs.cuda_stream), gs, reps=10) / 10
    for g in graphs:
        L.coot_graph_destroy(g)

    # one training step each: gradients set to None first (as zero_grad does),
    # so no step adds into the previous step's gradients
    W2 = W.clone().requires_grad_(True)
    X2 = X.clone().requires_grad_(True)

    def fused():
        Wp.grad = None
        Xp.grad = None
        loss = AG.loss_l2_schur(Wp, Xp, Y, 1e-3)
        loss.backward()
        return loss

    def torch_ref():
        W2.grad = None
        X2.grad = None
        loss = ((W2 * X2 - Y) ** 2).sum() + 1e-3 * (W2 ** 2).sum()
        loss.backward()

    ms_f = time_calls(fused, stream, reps=10)
    ms_t = time_calls(torch_ref, stream, reps=10)
    # host time of one fused step (the GPU is idle-waited before and after)
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for _ in range(20):
        fused()
    host_ms = (time.perf_counter() - h0) / 20 * 1e3
    torch.cuda.synchronize()
    n = W.numel()
    return {"n": W.shape[0], "fwd_kernel_ms": round(ms_fwd, 4), "fwd_gbs": round(12 * n / ms_fwd / 1e6, 1),
            "adjoint_kernel_ms": round(ms_bwd, 4), "adjoint_gbs": round(20 * n / ms_bwd / 1e6, 1),
            "autograd_step_ms": round(ms_f, 4), "autograd_step_host_ms": round(host_ms, 4),
            "step_over_kernels": round(ms_f / (ms_fwd + ms_bwd), 2), "torch_autograd_ms": round(ms_t, 4),
            "speedup_vs_torch_autograd": round(ms_t / ms_f, 2), "algorithmic_bytes_fwd_bwd": 32 * n,
            "note": "fwd reads W, X, Y (12N bytes); the adjoint reads them again and writes dW, dX (20N)"}


def bench_precision(dev, stream, errors=False):
    """Reductions over 2^28-element signed-lognormal vectors (FP32/BF16/FP16,
    and FP64 var), through prepared C-ABI calls.  With errors=True also the
    relative error of each result against the FP64 oracle, for float-float
    (default), Kahan and plain FP32 accumulation."""
    import torch

    from paper_2508_11385_gb300 import workloads

    out = {}
    n = 1 << 28
    sp = stream.cuda_stream
    progs = [("accu", "A accu"), ("dot", "A B dot"), ("norm", "A norm"), ("var", "A var")]
    for dt in ("f32", "bf16", "f16", "f64"):
        x, y = workloads.precision(dt, n=n, device=dev)
        host = None
        if errors:
            import oracle

            host = [workloads.to_numpy_colmajor(t) for t in (x, y)]
        d = {}
        for name, prog in progs:
            if dt == "f64" and name != "var":
                continue
            c = Call(prog, [x, y])
            c(sp)
            torch.cuda.synchronize()
            ms = time_calls(lambda: c(sp), stream, reps=10)
            info = c.info()
            ent = {"ms": round(ms, 4), "gbs": round(info["algorithmic_bytes"] / ms / 1e6, 1), "kernel": info["kernel"]}
            if errors:
                ref = float(oracle.evaluate(prog, host, dt).value[0, 0])
                ent["rel_err"] = abs(float(c.result().item()) - ref) / abs(ref)
                if dt != "f64":
                    for mode in ("kahan", "plain"):
                        os.environ["COOT_ACCUM"] = mode
                        try:
                            c2 = Call(prog, [x, y])
                            c2(sp)
                            torch.cuda.synchronize()
                            ent["rel_err_" + mode] = abs(float(c2.result().item()) - ref) / abs(ref)
                        finally:
                            del os.environ["COOT_ACCUM"]
            d[name] = ent
        out[dt] = d
        del x, y, host
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2508_11385_gb300 import workloads

    oracle.build()
    n = 2048
    scale = n / N_MAIN
    leaves = workloads.large_trees("f32", n=n, device="cpu")
    host = [workloads.to_numpy_colmajor(t) for t in leaves]
    try:
        cores, parallel = oracle.threads(parallel=True), True
    except oracle.OracleError:
        cores, parallel = 1, False

    def step():
        b = 0
        for _, prog, _ in TREES:
            p = prog.replace("submat:1000:1000:4096:4096", "submat:%d:%d:%d:%d" % (
                int(1000 * scale), int(1000 * scale), int(4096 * scale), int(4096 * scale)))
            oracle.evaluate(p, host, "f32", parallel=parallel)
            b += algorithmic_bytes(p, n, 4)
        return b

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        total += step()
    sec = time.perf_counter() - t0
    value = total / sec / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3 / args.steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (same recipe, host-generated)",
           "config": {"workload": "large memory-bound trees, FP32 storage: 6 shapes + depth ladder L4-L8 "
                                  "(bounded sample %dx%d per step)" % (n, n), "trees": [t[0] for t in TREES]},
           "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
                            "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
                            "sample": "%d steps of the %d trees at %dx%d, element-wise loops on %d thread(s)" % (
                                args.steps, len(TREES), n, n, cores)},
           "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_MAIN)
    ap.add_argument("--batch-problems", type=int, default=50000)
    ap.add_argument("--batch-separate", type=int, default=2000,
                    help="problems timed as separate launches for the comparison (0: skip)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--quick", action="store_true", help="headline only (no side workloads)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--precision-errors", action="store_true",
                    help="also report each precision result's error against the FP64 oracle (slow)")
    ap.add_argument("--h2d-streams", type=int, default=1,
                    help="copy streams for the host->device operand copies of the end-to-end measurement")
    ap.add_argument("--only", default=None, help="time one tree of the workload (profiling); implies --quick")
    ap.add_argument("--prog", default=None, help="time one RPN program over the workload's leaves (profiling)")
    ap.add_argument("--flush", action="store_true", help="--prog: time every call after refilling the L2 with clean lines")
    ap.add_argument("--prog-dtype", default="f32", choices=["f32", "f64", "bf16", "f16", "i32"],
                    help="--prog: storage type of the leaves")
    ap.add_argument("--prog-cols", type=int, default=None, help="--prog: columns of the leaves (default n)")
    args = ap.parse_args()
    if args.prog:
        run_prog(args)
        return
    if args.only:
        side = ("batched", "adjoint", "precision", "graph_chain", "stats", "gemm", "e2e", "e2e_zero_copy", "probe")
        if args.only not in [t[0] for t in TREES] + list(side):
            ap.error("--only: one of %s" % ", ".join([t[0] for t in TREES] + list(side)))
        args.quick = True
        args.no_cpu = True
        if args.only in side:
            run_side(args)
            return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
