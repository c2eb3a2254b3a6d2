"""Benchmark of the GB300 rollout planner (one JSON line on rank 0).

A step is one plan: the fused sm_103a kernel rolls every candidate of the
workload forward (SRB model, terrain, suspension, tire, ESM, cost) and reduces
to the best feasible candidate, through the C-ABI (atp_plan).  The default
workload is the scaled rollout: 16384 candidates, horizon 100 at dt = 0.02 s
(4 Euler steps of 5 ms), per-candidate initial speed 5-15 m/s, on a
1024 x 1024 heightmap at 0.1 m.

  value  rollout-steps/s (candidates x control steps per second) of the whole
         job, device-timed with CUDA events per step, L2 flushed between steps
  e2e    the same metric with host buffers: pinned host -> device copy of the
         step's candidates and initial states, the plan, device -> host copy
         of the result, all inside the timed region
  --impl reference   the FP64 CPU oracle on the same workload (host cores)

Under torchrun each rank runs an independent replica of the workload on its
own GPU (weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FP32 work of one Euler step of one candidate: the additions,
# subtractions, multiplications and divisions of the oracle's model, counted by
# its counting scalar (oracle.count_ops) over the first 1024 candidates of each
# workload; tests/test_bench_host.py recounts them.  A fused multiply-add is
# two of these.  The elementary functions of a step (5 sqrt, 4 sin, 8 cos and
# 4 atan2 in the oracle's form) are not in the count.
FLOPS_PER_SUBSTEP = {"plain": 623.762, "scaled": 623.070, "paper": 622.553}
FP32_LANES_PER_SM = 128         # FP32 units per Blackwell SM (4 sub-partitions x 32)


def device_sm_count(device=0) -> int:
    """Streaming multiprocessors of the GPU, from the device properties."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def max_sm_mhz(index=0):
    """The GPU's maximum SM clock (nvidia-smi clocks.max.sm), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(index)], capture_output=True, text=True, timeout=30).stdout
        return float(out.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None


def fp32_peak_tflops(sms, mhz):
    """SMs x 128 FP32 lanes x 2 flops (fused multiply-add) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


# what the plan kernel is compiled from: its translation unit, the headers it
# includes and the module that holds the compile flags
PLAN_KERNEL_SOURCES = ("paper_2603_20525_gb300/csrc/plan_kernel.cu", "paper_2603_20525_gb300/csrc/plan_kernel.cuh",
                       "paper_2603_20525_gb300/csrc/plan_tail.cuh", "paper_2603_20525_gb300/csrc/srb_model.cuh",
                       "paper_2603_20525_gb300/csrc/fastmath.cuh", "include/atp.h",
                       "paper_2603_20525_gb300/build.py")


def kernel_sources_sha256():
    """SHA-256 of the plan kernel's sources, in the order listed."""
    import hashlib
    h = hashlib.sha256()
    for rel in PLAN_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(workload):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel sources changed since the capture or it covers another workload."""
    path = os.path.join(ROOT, "profiles", "plan_kernel_traffic.txt")
    try:
        kv = dict(l.split(":", 1) for l in open(path) if ":" in l and not l.startswith("#"))
    except OSError:
        return None
    kv = {k.strip(): v.strip() for k, v in kv.items()}
    if kv.get("sources_sha256") != kernel_sources_sha256() or kv.get("workload") != workload:
        return None
    return int(kv["dram_bytes_per_launch"])


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks: the job's time is its slowest rank's.
    One rank (or no process group) returns x."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size: int, units_per_rank: float, ms: float) -> float:
    """Weak scaling: every rank runs units_per_rank; the job's rate is all
    ranks' units over the slowest rank's time (ms)."""
    return world_size * units_per_rank / (ms / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms, each sample
    stamped on arrival so that only those taken inside the timed region count."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.index), "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None
            return
        t0 = time.perf_counter()             # wait for the sampler to run
        while not self.lines and time.perf_counter() - t0 < 5.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.p.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t_begin, t_end):
        """Summary of the samples stamped in [t_begin, t_end] (perf_counter
        seconds); the nearest sample when none falls inside."""
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [l for t, l in self.lines if t_begin <= t <= t_end]
        if not inside and self.lines:
            inside = [min(self.lines, key=lambda tl: abs(tl[0] - 0.5 * (t_begin + t_end)))[1]]
        for l in inside:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm),
                    reasons=sorted(reasons), window="samples stamped inside the timed region")


def make_workload(name):
    import gen
    if name == "scaled":
        return gen.workload_scaled(0)
    if name == "plain":
        return gen.workload_plain(0)
    if name == "paper":
        return gen.workload_paper(0)
    raise SystemExit(f"unknown workload {name}")


def workload_config(w, name):
    return {"workload": f"{name}: {w.N} candidates x H={w.H} at dt={w.dt} s "
                        f"({w.n_sub} Euler steps of {1000 * w.dt / w.n_sub:g} ms), "
                        f"{w.terrain.nx}x{w.terrain.ny} heightmap at {w.terrain.cell} m",
            "candidates": w.N, "horizon": w.H, "dt": w.dt, "n_sub": w.n_sub,
            "terrain": [w.terrain.ny, w.terrain.nx], "cell_m": w.terrain.cell,
            "vehicle": ("MRZR parameters (appendix)" if name == "paper" else
                        "1000 kg, wheelbase 2.5 m, track 1.5 m, CoM 0.6 m, 40 kN/m, 3 kN s/m"),
            "l2": "flushed between steps (256 MB write)"}


def omp_threads() -> int:
    """Threads the oracle's OpenMP loops run with: OMP_NUM_THREADS if set,
    else one per CPU this process may run on (libgomp's default)."""
    env = os.environ.get("OMP_NUM_THREADS", "").split(",")[0].strip()
    if env.isdigit() and int(env) > 0:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, w, name, budget_s=120.0):
    """The FP64 CPU oracle, as it stands, on the same workload.  Each step
    plans a prefix of the candidates, sized from one timed full plan so that
    the whole --steps/--warmup run takes about budget_s seconds."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    t = oracle.Terrain.of(w.terrain)
    cores = omp_threads()
    t0 = time.perf_counter()
    oracle.plan(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    t_full = time.perf_counter() - t0
    n_runs = max(1, args.steps + args.warmup)
    m = int(min(w.N, max(256, w.N * budget_s / (n_runs * t_full))))
    x0 = w.x0[:m] if w.x0.ndim == 2 else w.x0
    ctrl = np.ascontiguousarray(w.ctrl[:, :m])
    for _ in range(args.warmup):
        oracle.plan(w.vehicle, w.cost, t, x0, ctrl, w.dt, w.n_sub)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.plan(w.vehicle, w.cost, t, x0, ctrl, w.dt, w.n_sub)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = m * w.H / (ms / 1000)
    unit = "rollout-steps/s"
    sample = (f"each step the first {m} of the workload's {w.N} candidates (all {w.H} steps), "
              f"FP64 C oracle, OpenMP over candidates")
    print(json.dumps({
        "impl": "reference", "metric": "rollout-steps/s", "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, name),
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "substeps_per_s": value * w.n_sub,
    }), flush=True)


def cpu_baseline(w, budget_s=10.0):
    """The oracle on a bounded sample: whole plans of the workload repeated
    for about budget_s seconds on every host core."""
    import oracle
    t = oracle.Terrain.of(w.terrain)
    oracle.plan(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.plan(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 200:
            break
    out = {"value": n * w.N * w.H / el, "unit": "rollout-steps/s", "cores": omp_threads(),
           "kind": "oracle",
           "sample": f"{n} whole plans of the workload ({n * w.N} candidates, {el:.1f} s), FP64"}
    # the same oracle on one thread, over the first 1024 candidates
    m = min(w.N, 1024)
    x0 = w.x0[:m] if w.x0.ndim == 2 else w.x0
    ctrl = np.ascontiguousarray(w.ctrl[:, :m])
    n1, t0 = 0, time.perf_counter()
    while True:
        oracle.plan(w.vehicle, w.cost, t, x0, ctrl, w.dt, w.n_sub, nthreads=1)
        n1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= budget_s / 2 or n1 >= 200:
            break
    out["single_thread"] = {"value": n1 * m * w.H / el1, "unit": "rollout-steps/s", "cores": 1,
                            "sample": f"{n1} plans of the first {m} candidates ({el1:.1f} s), FP64"}
    # the plain configuration (1024 candidates x H = 40 x 10 Euler steps), whole plans
    import gen
    wp = gen.workload_plain(0)
    tp = oracle.Terrain.of(wp.terrain)
    n2, t0 = 0, time.perf_counter()
    while True:
        oracle.plan(wp.vehicle, wp.cost, tp, wp.x0, wp.ctrl, wp.dt, wp.n_sub)
        n2 += 1
        el2 = time.perf_counter() - t0
        if el2 >= budget_s / 4 or n2 >= 2000:
            break
    out["plain"] = {"value": n2 * wp.N * wp.H / el2, "unit": "rollout-steps/s", "cores": omp_threads(),
                    "ms_per_plan": 1e3 * el2 / n2,
                    "sample": f"{n2} whole plans of the plain workload ({wp.N} x {wp.H} x {wp.n_sub}, "
                              f"{el2:.1f} s), FP64"}
    return out


def run_paper_config(ctx, dev, stream, flush, peak, steps=10, warmup=3):
    """The real-time configuration of Sec. IV-D (204,288 candidates, 16 steps
    of 0.25 s, 800 Euler steps of 5 ms each, steering only) on this GPU, in
    the paper's units: trajectory samples per second and the planner rate.
    The paper's own figures on its hardware are quoted beside it."""
    import gen
    import torch
    w = gen.workload_paper(0)
    ter = ctx.terrain_prepare(torch.as_tensor(w.terrain.heights).to(dev), w.terrain.cell,
                              w.terrain.x0, w.terrain.y0)
    ctrl = torch.as_tensor(w.ctrl).to(dev)
    x0 = [float(v) for v in w.x0]
    outs = ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, want_candidates=False,
                    want_best_margin=False)
    for _ in range(warmup):
        ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, out=outs)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, out=outs)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # terrain staging (a window of the texels in each CTA's shared memory),
    # A/B against the plain kernel on the same plan: same result, its time.
    # A 2 x 2 window stages nothing useful: it is the staged kernel's
    # 512-thread CTAs alone.
    from paper_2603_20525_gb300 import atp
    ref = outs["out"].clone()
    staged = []
    for side in (2, 64, 120):
        ctx.set_option(atp.OPT_STAGE_TERRAIN, side)
        try:
            ms_s = _time(lambda: ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, out=outs),
                         steps, warmup, stream, flush)
        finally:
            ctx.set_option(atp.OPT_STAGE_TERRAIN, 0)
        staged.append({"window_nodes": f"{side} x {side}", "shared_kb": side * side * 16 / 1024,
                       "ms_per_plan": ms_s, "vs_plain": ms_s / ms,
                       "same_result": bool(torch.equal(outs["out"], ref))})
    return {"workload": f"{w.N} candidates x 16 steps of 0.25 s ({w.n_sub} Euler steps of 5 ms "
                        f"each), steering only, {w.terrain.nx}^2 heightmap at {w.terrain.cell} m",
            "terrain_staging": staged,
            "ms_per_plan": ms, "planner_hz": 1000.0 / ms, "samples_per_s": w.N / (ms / 1000),
            "substeps_per_s": w.N * w.H * w.n_sub / (ms / 1000),
            "fp32_tflops": FLOPS_PER_SUBSTEP["paper"] * w.N * w.H * w.n_sub / (ms / 1000) / 1e12,
            "fp32_frac": FLOPS_PER_SUBSTEP["paper"] * w.N * w.H * w.n_sub / (ms / 1000) / 1e12 / peak,
            "paper_context": "80 Hz, over 11 M samples/s on an RTX 5000 Ada Mobile; about 21 M "
                             "samples/s on an RTX 6000 Ada (Sec. IV-D); other hardware"}


def _time(fn, steps, warmup, stream, flush):
    import torch
    for _ in range(warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def run_variants(ctx, dev, stream, flush, steps=10):
    """The other kernels of the library on this GPU: the planar (EST) model on
    the scaled workload (its own 1.5 m level of detail), and the terrain
    preprocessing (Gaussian level of detail and the distance-constraint
    costmap) on a 2048^2 map at 0.1 m."""
    import gen
    import torch
    from paper_2603_20525_gb300 import atp
    out = {}
    w = gen.workload_est(0, N=16384, H=100, dt=0.02, scaled=True)
    ter = ctx.terrain_prepare(torch.as_tensor(w.terrain.heights).to(dev), w.terrain.cell,
                              w.terrain.x0, w.terrain.y0)
    ctrl = torch.as_tensor(w.ctrl).to(dev)
    x0 = torch.as_tensor(np.ascontiguousarray(w.x0.T)).to(dev)
    o = ctx.plan_est(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, want_candidates=False)
    ms = _time(lambda: ctx.plan_est(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, out=o),
               steps, 3, stream, flush)
    out["est_plan"] = {"workload": f"planar model, {w.N} candidates x H={w.H} at dt={w.dt} s "
                                   f"({w.n_sub} Euler steps), 1024^2 map, 1.5 m level of detail",
                       "ms_per_plan": ms, "rollout_steps_per_s": w.N * w.H / (ms / 1e3),
                       "substeps_per_s": w.N * w.H * w.n_sub / (ms / 1e3)}
    # the scaled plan on BF16 texels (8 B per node instead of 16)
    ws = gen.workload_scaled(0)
    ter16 = ctx.terrain_prepare(torch.as_tensor(ws.terrain.heights).to(dev), ws.terrain.cell,
                                ws.terrain.x0, ws.terrain.y0, fmt=atp.BF16X4)
    ctrl16 = torch.as_tensor(ws.ctrl).to(dev)
    x016 = torch.as_tensor(np.ascontiguousarray(ws.x0.T)).to(dev)
    o16 = ctx.plan(ws.vehicle, ws.cost, ter16, x016, ctrl16, ws.dt, ws.n_sub, want_candidates=False,
                   want_best_margin=False)
    ms = _time(lambda: ctx.plan(ws.vehicle, ws.cost, ter16, x016, ctrl16, ws.dt, ws.n_sub, out=o16),
               steps, 3, stream, flush)
    out["bf16_terrain_plan"] = {"workload": "the scaled plan on BF16 texels", "ms_per_plan": ms,
                                "rollout_steps_per_s": ws.N * ws.H / (ms / 1e3)}
    # the plain configuration (1024 candidates x H = 40 at dt = 0.05 s, 10 Euler steps)
    wp = gen.workload_plain(0)
    terp = ctx.terrain_prepare(torch.as_tensor(wp.terrain.heights).to(dev), wp.terrain.cell,
                               wp.terrain.x0, wp.terrain.y0)
    ctrlp = torch.as_tensor(wp.ctrl).to(dev)
    x0p = [float(v) for v in wp.x0]
    op = ctx.plan(wp.vehicle, wp.cost, terp, x0p, ctrlp, wp.dt, wp.n_sub, want_candidates=False,
                  want_best_margin=False)
    ms = _time(lambda: ctx.plan(wp.vehicle, wp.cost, terp, x0p, ctrlp, wp.dt, wp.n_sub, out=op),
               steps, 3, stream, flush)
    out["plain_plan"] = {"workload": f"plain: {wp.N} candidates x H={wp.H} at dt={wp.dt} s "
                                     f"({wp.n_sub} Euler steps), 256^2 map at 0.2 m, "
                                     f"{ctx.plan_lanes(wp.N)} threads per candidate",
                         "ms_per_plan": ms, "rollout_steps_per_s": wp.N * wp.H / (ms / 1e3)}
    t = gen.terrain_tile(2048, 5, lod_sigma=0.0)
    h = torch.as_tensor(t.heights).to(dev)
    sm = torch.empty_like(h)
    for sig in (0.3, 1.5):
        ms = _time(lambda: ctx.lod_smooth(h, t.cell, sig, out=sm), steps, 3, stream, flush)
        out[f"lod_{sig}m"] = {"workload": f"2048^2 at {t.cell} m, sigma {sig} m "
                                          f"(radius {int(4 * sig / t.cell + 0.5)} cells)",
                              "ms": ms, "nodes_per_s": 2048 * 2048 / (ms / 1e3),
                              "hbm_gbs_min_traffic": 4 * 4 * 2048 * 2048 / (ms / 1e3) / 1e9}
    polys = gen.obstacles(t, 5, n=24)
    nv = sum(len(p) for p, _ in polys)
    ms = _time(lambda: ctx.costmap(polys, t.nx, t.ny, t.cell, t.x0, t.y0), steps, 3, stream, flush)
    out["costmap"] = {"workload": f"2048^2 nodes, {len(polys)} perimeters, {nv} edges", "ms": ms,
                      "nodes_per_s": 2048 * 2048 / (ms / 1e3),
                      "note": "each 16 x 16 tile skips the obstacles beyond 2 eps of it (exactly zero "
                              "rate there); the path boundary is evaluated at every node"}
    # the adjoint's configuration: 64 candidates of the plain plan at H = 100, dt = 0.02 s
    wa = gen.workload_plain(0, N=64, H=100, dt=0.02)
    tera = ctx.terrain_prepare(torch.as_tensor(wa.terrain.heights).to(dev), wa.terrain.cell)
    ca = torch.as_tensor(wa.ctrl).to(dev)
    xa = [float(v) for v in wa.x0]
    ms = _time(lambda: ctx.grad(wa.vehicle, wa.cost, tera, xa, ca, wa.dt, wa.n_sub, 10), steps, 3, stream, flush)
    out["adjoint"] = {"workload": "dJ/dctrl of 64 candidates, H = 100, dt = 0.02 s (4 Euler steps), "
                                  "checkpoints every 10 steps", "ms": ms,
                      "candidate_gradients_per_s": 64 / (ms / 1e3)}
    # the sampler: the largest serving request, 32768 candidates x 150 steps
    ctrl_s = torch.empty((150, 32768, 2), dtype=torch.float32, device=dev)
    ms = _time(lambda: ctx.sample(32768, 150, 0.2, 0.3, (1, 2), 3, out=ctrl_s), steps, 3, stream, flush)
    out["sampler"] = {"workload": "32768 candidates x 150 steps, Philox4x64-10 + Box-Muller", "ms": ms,
                      "hbm_gbs": 150 * 32768 * 8 / (ms / 1e3) / 1e9}
    return out


def run_serving(seconds, device, sweep_rates=(), sweep_seconds=10.0):
    """The serving stream: 32 vehicles, each on its own resident 512-2048^2
    tile, Poisson plan requests at 20 Hz per vehicle with N in {1k, 4k, 16k,
    32k}, H uniform in [40, 150], dt in {0.020, 0.025, ..., 0.050} s, warm
    started from the vehicle's previous plan; continuous batching against the
    plain single-plan path replaying the same trace one request at a time."""
    import gen
    from paper_2603_20525_gb300 import serve
    fl = gen.fleet(32, seed=0)
    vehicles = serve.resident_vehicles(fl, device=device)
    srv = serve.Server(vehicles, streams=2, slot_candidates=1 << 17, arena_bytes=2 << 30,
                       device=device)
    srv.serve(serve.poisson_trace(32, 20.0, 0.5, seed=99))          # warm-up
    serve.reset_warm_start(vehicles)
    trace = serve.poisson_trace(32, 20.0, seconds, seed=1)
    served = srv.serve(trace)
    gap_served = srv.max_loop_gap
    serve.reset_warm_start(vehicles)
    plain = srv.sequential(trace)
    gap_plain = srv.max_loop_gap
    same = all(a.best_idx == b.best_idx and a.best_cost == b.best_cost for a, b in zip(served, plain))
    out = {"workload": "32 vehicles x 20 Hz Poisson, N in {1024, 4096, 16384, 32768}, "
                       "H 40-150, dt 0.02-0.05 s, own 512-2048^2 tile at 0.1 m, warm start",
           "trace_s": seconds, "requests": len(trace),
           "served": dict(serve.latency_summary(served),
                          longest_loop_pause_ms=1000 * gap_served[0], at_s=gap_served[1]),
           "plain_sequential": dict(serve.latency_summary(plain),
                                    longest_request_ms=1000 * gap_plain[0], at_s=gap_plain[1]),
           "identical_results": bool(same)}
    # the same 32-vehicle mix at higher request rates, until the plain path
    # falls behind: where continuous batching pays
    sweep = []
    for rate in sweep_rates:
        tr = serve.poisson_trace(32, float(rate), sweep_seconds, seed=1000 + int(rate))
        serve.reset_warm_start(vehicles)
        a = srv.serve(tr)
        serve.reset_warm_start(vehicles)
        b = srv.sequential(tr)
        sa, sb = serve.latency_summary(a), serve.latency_summary(b)
        offered = sum(r.N * r.H for r in tr) / sweep_seconds
        sweep.append({"rate_hz_per_vehicle": rate, "requests": len(tr), "offered_rollout_steps_per_s": offered,
                      "served": {k: sa[k] for k in ("p50_ms", "p99_ms", "max_ms", "mean_batch",
                                                   "rollout_steps_per_s")},
                      "plain_sequential": {k: sb[k] for k in ("p50_ms", "p99_ms", "max_ms",
                                                             "rollout_steps_per_s")},
                      "identical_results": bool(all(x.best_idx == y.best_idx and x.best_cost == y.best_cost
                                                    for x, y in zip(a, b)))})
    if sweep:
        out["rate_sweep"] = {"trace_s": sweep_seconds, "points": sweep}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scaled", choices=["scaled", "plain", "paper"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4],
                    help="threads per candidate (ATP_OPT_LANES; 0 chooses by batch size)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="seconds of the 32-vehicle request stream (0: skip)")
    ap.add_argument("--serve-rates", default="30,40,60,80,100",
                    help="per-vehicle request rates (Hz) of the serving sweep, comma-separated ('' skips)")
    ap.add_argument("--sweep-seconds", type=float, default=6.0, help="seconds of each sweep stream")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = make_workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w, args.workload)

    import torch
    import torch.distributed as dist
    from paper_2603_20525_gb300 import atp

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)            # each rank's own GPU before NCCL comes up
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    ctx = atp.Context(local)
    ctx.set_option(atp.OPT_LANES, args.lanes)
    ctx.reserve(w.N, w.H)
    heights = torch.as_tensor(w.terrain.heights).to(dev)
    ter = ctx.terrain_prepare(heights, w.terrain.cell, w.terrain.x0, w.terrain.y0)
    ctrl = torch.as_tensor(w.ctrl).to(dev)
    per = w.x0.ndim == 2
    x0 = torch.as_tensor(np.ascontiguousarray(w.x0.T)).to(dev) if per else [float(v) for v in w.x0]
    # the planner's outputs: best controls, cost, minimum ESM margin and its step
    # (the optional per-step margins of the best candidate are not asked for)
    outs = ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, want_candidates=False,
                    want_best_margin=False)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step():
        ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, out=outs)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_begin = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                       # evict L2 between steps
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_end = time.perf_counter()
    per_step = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(per_step)
    clk = clocks.stop(t_begin, t_end)
    ms = max_over_ranks(ms, dev)
    units = w.N * w.H
    value = job_rate(ws, units, ms)

    # end to end through the public API with host buffers, double-buffered:
    # the controls and start states of step k+1 are copied from pinned host
    # memory on their own stream while step k computes, as an MPC loop that
    # prepares its next plan would; every step's inputs cross the bus, and its
    # result is read back to pinned host memory, inside the timed region (the
    # L2 flush between steps is inside it too)
    ctrl_h = torch.as_tensor(w.ctrl).pin_memory()
    x0_h = torch.as_tensor(np.ascontiguousarray(w.x0.T)).pin_memory() if per else None
    res_h = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outs.items()}
    copy_stream = torch.cuda.Stream(device=dev)
    bufs = [(torch.empty_like(ctrl), torch.empty_like(x0) if per else None) for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]

    def copy_in(k):
        b = k % 2
        copy_stream.wait_event(consumed[b])
        with torch.cuda.stream(copy_stream):
            bufs[b][0].copy_(ctrl_h, non_blocking=True)
            if per:
                bufs[b][1].copy_(x0_h, non_blocking=True)
        copied[b].record(copy_stream)

    def run_step(k):
        b = k % 2
        flush.zero_()
        stream.wait_event(copied[b])
        o = ctx.plan(w.vehicle, w.cost, ter, bufs[b][1] if per else x0, bufs[b][0], w.dt, w.n_sub,
                     out=outs, stream=stream)
        consumed[b].record(stream)
        for k2, v in o.items():
            res_h[k2].copy_(v, non_blocking=True)

    def e2e_run(n, start=None):
        if start is not None:
            copy_stream.wait_event(start)
        copy_in(0)
        for k in range(n):
            if k + 1 < n:
                copy_in(k + 1)
            run_step(k)

    e2e_run(args.warmup)
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    e2e_run(args.steps, start=t_start)
    t_end.record(stream)
    torch.cuda.synchronize()
    e2e_ms = t_start.elapsed_time(t_end) / args.steps
    e2e_ms = max_over_ranks(e2e_ms, dev)
    h2d = ctrl_h.numel() * 4 + (x0_h.numel() * 4 if per else 0)
    d2h = sum(v.numel() * v.element_size() for v in res_h.values())

    if rank == 0:
        substeps = units * w.n_sub
        flops = FLOPS_PER_SUBSTEP[args.workload]
        achieved = flops * substeps / (ms / 1000) / 1e12
        sms = device_sm_count(local)
        mhz = max_sm_mhz(local) or (clk or {}).get("sm_max_mhz") or 2070.0
        peak = fp32_peak_tflops(sms, mhz)
        line = {
            "metric": "rollout-steps/s", "value": value, "unit": "rollout-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(w, args.workload), threads_per_candidate=ctx.plan_lanes(w.N)),
            "substeps_per_s": value * w.n_sub,
            "latency_ms": {"p50": float(np.percentile(per_step, 50)),
                           "p99": float(np.percentile(per_step, 99))},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(args.workload),
                         "kernel": "plan_kernel (fused rollout + argmin)",
                         "note": f"{flops} algorithmic FP32 flops per Euler step (counted by the "
                                 f"oracle's counting scalar) x {substeps} Euler steps per launch; "
                                 f"peak = {sms} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                                 f"x {mhz:g} MHz (maximum SM clock, nvidia-smi), derived"},
            "e2e": {"value": job_rate(ws, units, e2e_ms), "unit": "rollout-steps/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "overlap": "step k+1's inputs are copied on a second stream while step k runs "
                               "(two device buffers); L2 flush between steps inside the timed region"},
            "gpu_launches": args.steps,
            "clocks": clk,
        }
        # the single-GPU characterisation (the paper configuration, the other
        # kernels, the serving stream) runs at N = 1 only: under torchrun the
        # other ranks would sit idle on their GPUs meanwhile
        if args.workload != "paper" and ws == 1:
            line["paper_configuration"] = run_paper_config(ctx, dev, stream, flush, peak)
            line["other_kernels"] = run_variants(ctx, dev, stream, flush)
        if args.serve_seconds > 0 and ws == 1:
            rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
            line["serving"] = run_serving(args.serve_seconds, local, rates, args.sweep_seconds)
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
