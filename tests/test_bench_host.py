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
