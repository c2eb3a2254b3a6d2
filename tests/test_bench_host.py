"""bench.py's host-side contract, without a GPU: the reference arm's JSON line
(the FP64 oracle on the host cores) and the clock sampler's window, fed with
stamped nvidia-smi lines instead of a running nvidia-smi."""
import json
import os
import subprocess
import sys

import numpy as np
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


def _count(name):
    import gen
    import oracle
    w = {"plain": gen.workload_plain, "scaled": gen.workload_scaled, "paper": gen.workload_paper}[name](0)
    N = min(w.N, 1024)
    x0 = w.x0[:N] if w.x0.ndim == 2 else w.x0
    return oracle.count_ops(w.vehicle, w.cost, oracle.Terrain.of(w.terrain), x0, w.ctrl[:, :N], w.dt, w.n_sub)


@pytest.mark.parametrize("name", ["plain", "scaled", "paper"])
def test_roofline_flops_are_the_oracles_count(name):
    """The roofline's numerator is the oracle's counted work per Euler step
    (additions, subtractions, multiplications, divisions), not a hand count."""
    c = _count(name)
    n = c["euler_steps"]
    assert abs((c["add"] + c["mul"] + c["div"]) / n - bench.FLOPS_PER_SUBSTEP[name]) < 5e-4
    # the model's structure per Euler step (Sec. IV-A..IV-C): one slip angle
    # per wheel; a tire square root per wheel and the goal test's; sines of
    # the three angles and of the ESM's |phi| + phibar; cosines of the three
    # angles, of each wheel's steering angle and of the pitch in the ESM
    assert c["atan2"] == 4 * n
    assert 5 * n <= c["sqrt"] <= 5 * n + 1024
    assert 4 * n <= c["sin"] <= 4 * n + 1024
    assert 8 * n <= c["cos"] <= 8 * n + 1024
    assert c["div"] == 30 * n


def test_flop_count_scales_with_the_horizon():
    import gen
    import oracle
    w = gen.workload_plain(0, N=16, H=8)
    t = oracle.Terrain.of(w.terrain)
    a = oracle.count_ops(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    b = oracle.count_ops(w.vehicle, w.cost, t, w.x0, np.concatenate([w.ctrl, w.ctrl]), w.dt, w.n_sub)
    assert b["euler_steps"] == 2 * a["euler_steps"]
    per_a = (a["add"] + a["mul"] + a["div"]) / a["euler_steps"]
    per_b = (b["add"] + b["mul"] + b["div"]) / b["euler_steps"]
    assert abs(per_a - per_b) < 2.0      # the terminal cost and liftoff branches aside


def test_fp32_peak_from_unit_counts_and_clock():
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9


def test_traffic_record_holds_only_for_the_captured_plan_kernel(tmp_path, monkeypatch):
    """The committed DRAM-traffic figure is reported while what the plan
    kernel is compiled from still hashes to the captured value, and only for
    the captured workload; a changed source drops it."""
    for rel in bench.PLAN_KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, rel)), rel
    fake = tmp_path / "repo"                # a copy of the plan kernel's sources
    for rel in bench.PLAN_KERNEL_SOURCES:
        dst = fake / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(fake))
    (fake / "profiles").mkdir()
    (fake / "profiles" / "plan_kernel_traffic.txt").write_text(
        "# a capture\nsources_sha256: %s\ndram_bytes_per_launch: 1234\nworkload: scaled\n"
        % bench.kernel_sources_sha256())
    assert bench.recorded_traffic("scaled") == 1234
    assert bench.recorded_traffic("paper") is None
    p = fake / "paper_2603_20525_gb300" / "csrc" / "srb_model.cuh"
    p.write_bytes(p.read_bytes() + b"\n")
    assert bench.recorded_traffic("scaled") is None
