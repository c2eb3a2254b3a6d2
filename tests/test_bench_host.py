"""bench.py's host-side contract, without a GPU: the reference arm's JSON line
(the FP64 oracle on the host cores) and the clock sampler's window, fed with
stamped nvidia-smi lines instead of a running nvidia-smi."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "plain", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "rollout-steps/s"
    assert d["unit"] == "rollout-steps/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "candidates" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["candidates"] == 1024 and d["config"]["horizon"] == 40


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def line(mhz, hw="Not Active", power_cap="Not Active"):
    return f"0, {mhz}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {power_cap}"


def test_clock_window_keeps_only_samples_inside_the_timed_region():
    c = bench.ClockSampler(0)
    c.p = _Done()
    c.lines = [(0.0, line(1200, hw="Active")),       # before the region: ignored
               (1.0, line(2070)), (1.05, line(2055)), (1.10, line(2070, power_cap="Active")),
               (5.0, line(900))]                   # after the region: ignored
    r = c.stop(0.9, 1.2)
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_window_falls_back_to_the_nearest_sample():
    c = bench.ClockSampler(0)
    c.p = _Done()
    c.lines = [(0.0, line(1500)), (2.0, line(2070)), (9.0, line(800))]
    r = c.stop(2.3, 2.4)                           # a region shorter than the sampling period
    assert r["samples"] == 1 and r["sm_mhz"] == 2070.0


def test_clock_sampler_without_nvidia_smi_reports_nothing():
    c = bench.ClockSampler(0)
    assert c.stop(0.0, 1.0) is None


def test_omp_threads_follows_the_environment(monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "3")
    assert bench.omp_threads() == 3
    monkeypatch.delenv("OMP_NUM_THREADS")
    assert bench.omp_threads() == len(os.sched_getaffinity(0))
