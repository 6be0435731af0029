"""Host-side parts of bench.py on the CPU: the oracle arm's JSON line, the
clock sampler's parsing of nvidia-smi output, and the traffic lookup."""
import json
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "solves/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2
    assert d["config"]["workload"] == bench.solve_workload_label("tiny")
    assert d["config"]["step"] == "one whole solve"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_workloads_say_unavailable():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "serve", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and "unavailable" in d


FAKE_SMI = """#!/bin/sh
i=0
while [ $i -lt 200 ]; do
  echo "0, {sm}, 2070, 900.5, 0x0, Not Active, {hwt}, Not Active, Active"
  i=$((i+1))
  sleep 0.05
done
"""


@pytest.mark.parametrize("sm,hwt,reasons", [(2070, "Not Active", ["sw_power_cap"]),
                                            (1500, "Active",
                                             ["hw_thermal_slowdown", "sw_power_cap"])])
def test_clock_sampler_parses_samples(tmp_path, monkeypatch, sm, hwt, reasons):
    smi = tmp_path / "nvidia-smi"
    smi.write_text(FAKE_SMI.format(sm=sm, hwt=hwt))
    smi.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.ClockSampler(0)
    c.start()
    time.sleep(0.6)
    r = c.stop()
    assert r["sm_mhz"] == sm and r["sm_max_mhz"] == 2070 and r["reasons"] == reasons
    assert r["samples"] >= 2
    assert not os.path.exists(c.path)            # the temporary sample file is removed


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["unsampled"]


def test_traffic_entry_follows_its_sources():
    """A committed DRAM-traffic figure is used only for its own workload and
    while the sources it was captured on are unchanged."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    for name, e in t.items():
        current = bench.kernel_source_hash(e.get("sources")) == e["source_hash"]
        got = bench.committed_traffic(name, e["workload"])
        assert (got is not None) == current
        assert bench.committed_traffic(name, e["workload"] + "-other") is None
    assert bench.committed_traffic("no_such_kernel") is None


def test_recorded_full_solve_time_comes_from_the_golden():
    from types import SimpleNamespace
    rec = bench.recorded_full_solve("city", SimpleNamespace(n=200_000))
    with open(os.path.join(ROOT, "tests", "golden", "city_oracle.json")) as f:
        gold = json.load(f)
    assert rec["seconds"] == gold["oracle_seconds"] and rec["seconds"] > 1000
    assert bench.recorded_full_solve("city", SimpleNamespace(n=1000)) is None   # other size
    assert bench.recorded_full_solve("no_such_workload", SimpleNamespace(n=5)) is None


def test_reference_arm_headline_line():
    """The default workload's oracle arm: whole small requests of the serving
    stream on one core, with the headline metric and config."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.HEADLINE_METRIC
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert "serving stream of 8 requests" in d["config"]["workload"]
    assert d["cpu_baseline"]["cores"] == 1 and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_default_arguments():
    a = bench.parse([])
    assert (a.workload, a.steps, a.per_step, a.large) == ("headline", 20, 4, "100000x1000")
    assert a.warmup >= 3


def test_scan_workload_arguments_and_reference_arm():
    a = bench.parse(["--workload", "scan", "--scan-of", "large", "--scan-n", "200000"])
    assert (a.workload, a.scan_of, a.scan_n) == ("scan", "large", 200000)
    b = bench.parse(["--workload", "scan"])
    assert (b.scan_of, b.scan_n) == ("city", 0)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "scan", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and "unavailable" in d
