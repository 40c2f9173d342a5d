"""Host logic of bench.py that needs no GPU: the clock sampler, run against a
stand-in `nvidia-smi` on PATH that prints the queried CSV columns the way the
real tool does, and the bounded oracle baseline."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

# index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
ROWS = [
    "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1100.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
]


def _fake_smi(tmp_path, rows, loop=True):
    script = tmp_path / "nvidia-smi"
    body = "\n".join("echo '%s'" % r for r in rows)
    if loop:  # -lms: keep printing until terminated, like the real tool
        body = "while true; do\n%s\nsleep 0.05\ndone" % body
    script.write_text("#!/bin/sh\n" + body + "\n")
    script.chmod(script.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_reads_median_max_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, ROWS) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0, path=str(tmp_path / "clocks.csv"))
    cs.start()
    time.sleep(0.4)
    out = cs.stop()
    assert out["samples"] >= 3
    assert out["sm_mhz"] == 2070.0  # median of 2070, 2055, 2070, ...
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_throttling(tmp_path, monkeypatch):
    rows = ["0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active"] * 3
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0, path=str(tmp_path / "clocks.csv"))
    cs.start()
    time.sleep(0.3)
    out = cs.stop()
    assert out["sm_mhz"] == 1500.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory: no nvidia-smi
    cs = bench.ClockSampler(0, path=str(tmp_path / "clocks.csv"))
    cs.start()
    out = cs.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_clock_samples_default_outside_the_repository(monkeypatch):
    monkeypatch.delenv("COOT_CLOCKS_CSV", raising=False)
    path = bench.ClockSampler(0).path
    assert not os.path.abspath(path).startswith(ROOT + os.sep)
    monkeypatch.setenv("COOT_CLOCKS_CSV", "/tmp/x.csv")
    assert bench.ClockSampler(0).path == "/tmp/x.csv"


@pytest.mark.parametrize("budget", [0.5])
def test_cpu_baseline_is_bounded_and_labelled(orc, budget):
    t0 = time.time()
    out = bench.cpu_baseline(n=256, budget_s=budget)
    assert time.time() - t0 < 60
    assert out["kind"] == "oracle" and out["unit"] == "GB/s" and out["value"] > 0 and "256x256" in out["sample"]
    assert out["single_thread"]["cores"] == 1 and out["single_thread"]["value"] > 0
    assert out["host_cpus"] == os.cpu_count() and out["cpu_model"]
    if "value" in out["all_cores"]:  # the OpenMP build exists
        assert out["cores"] == out["all_cores"]["cores"] >= 1 and out["value"] == out["all_cores"]["value"]


def test_algorithmic_bytes_of_the_workload_trees():
    # distinct operand bytes read plus bytes written, FP32 at 8192 x 8192:
    # axpy 12N, A%B+C 16N, trans(A)+B 12N, exp_div 16N, the depth ladder
    # 20N / 24N / 24N / 24N / 28N, the column sums 8N + 4 n, the view 4 * 4096^2 + 4
    n = 8192
    N = n * n
    want = {"axpy": 12 * N, "schur_plus": 16 * N, "trans_plus": 12 * N, "exp_div": 16 * N,
            "colsum_sq": 8 * N + 4 * n, "accu_submat": 4 * 4096 * 4096 + 4, "L4": 20 * N, "L5": 24 * N,
            "L6": 24 * N, "L7": 24 * N, "L8": 28 * N}
    got = {name: bench.algorithmic_bytes(prog, n, 4) for name, prog, _ in bench.TREES}
    assert got == want


def test_f64_alu_bound_counts_the_trees_fp64_operations():
    # rates in T operations/s: add 1, fma 2, div 0.5, exp+fma 0.25 -> exp alone 1/0.25 - 1/2 = 3.5 ps
    probe = {"f64_add": 1.0, "f64_fma": 2.0, "f64_div": 0.5, "f64_exp": 0.25}
    n = 10 ** 6
    ms, ops = bench.f64_alu_bound_ms("A B - exp #1 C abs + /", n, probe)
    assert ops == ["add", "exp", "add", "div"]  # abs uses no FP64 arithmetic
    want = n * (1.0 + 3.5 + 1.0 + 2.0) * 1e-12 * 1e3
    assert abs(ms - want) <= 1e-12 * want
    ms, ops = bench.f64_alu_bound_ms("A B - square sum:0", n, probe)
    assert ops == ["add", "mul", "add"]
    assert abs(ms - n * (1.0 + 0.5 + 1.0) * 1e-9) <= 1e-15
    ms, ops = bench.f64_alu_bound_ms("A submat:1:1:4:4 accu", 16, probe)
    assert ops == ["add"]


def test_torch_eager_trees_match_the_oracle():
    """The torch-eager baseline computes the same trees as the library (on CPU
    tensors here, column-major like the workload's leaves)."""
    import numpy as np

    import oracle
    from paper_2508_11385_gb300 import workloads

    n = 48
    lv = workloads.large_trees("f32", n=n, device="cpu")
    host = [workloads.to_numpy_colmajor(t) for t in lv]
    for name, prog, _ in bench.TREES:
        p = prog.replace("submat:1000:1000:4096:4096", "submat:5:7:30:31")
        y = bench.torch_eager_fn(p, lv)()
        r = oracle.evaluate(p, host, "f32")
        g = y.double().numpy().reshape(r.value.shape) if y.dim() > 0 else np.array([[y.item()]])
        # FP32 eager arithmetic against the FP64 oracle: within the oracle's
        # propagated FP32 bound plus the FP32 summation of up to n*n terms
        tol = r.bound + 1e-6 * np.abs(r.value) + (n * n) * 2.0 ** -24 * np.abs(r.value)
        assert np.all(np.abs(g - r.value) <= tol), name
