"""The serving loop on the GPU: requests of many vehicles, admitted into
ragged batches on two streams as they arrive, give the same per-request
results as the plain single-plan path run one at a time, and a served plan
agrees with the FP64 oracle."""
import numpy as np
import pytest

import gen
import oracle
from tests.test_gpu_parity import check_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fleet():
    return gen.fleet(8, seed=2, sides=(512,))


def burst_trace():
    from paper_2603_20525_gb300 import serve
    # 8 vehicles at 400 Hz for 0.1 s, then 20 Hz for 1 s: a burst that must batch
    a = serve.poisson_trace(8, 400.0, 0.1, seed=5, sizes=(1024, 4096), h_range=(20, 60))
    b = serve.poisson_trace(8, 20.0, 1.0, seed=6, sizes=(1024, 4096, 16384), h_range=(40, 100))
    reqs = [(r.t_arrive, r.vehicle, r.N, r.H, r.dt) for r in a] + \
           [(0.1 + r.t_arrive, r.vehicle, r.N, r.H, r.dt) for r in b]
    reqs.sort()
    return [serve.Request(i, v, N, H, dt, t) for i, (t, v, N, H, dt) in enumerate(reqs)]


@pytest.mark.parametrize("slots", [1 << 16, 20000])
def test_served_equals_sequential_bitwise(fleet, slots):
    """With ample slots, and with slots so tight that the admission keeps
    requests back (each vehicle's later requests must then wait behind them,
    or the warm starts would differ)."""
    from paper_2603_20525_gb300 import serve
    vehicles = serve.resident_vehicles(fleet)
    srv = serve.Server(vehicles, streams=2, slot_candidates=slots, arena_bytes=256 << 20)
    trace = burst_trace()
    served = srv.serve(trace)
    serve.reset_warm_start(vehicles)
    plain = srv.sequential(trace)
    assert all(np.isfinite(r.t_done) for r in served)
    assert max(r.batch for r in served) > 1                 # batches did form
    for a, b in zip(served, plain):
        assert a.rid == b.rid and a.best_idx == b.best_idx and a.best_cost == b.best_cost
    s = serve.latency_summary(served)
    p = serve.latency_summary(plain)
    print("served", s, "plain", p)
    assert srv.arena.used == 0                               # every block came back


def test_served_plan_matches_oracle(fleet):
    """The first request of a vehicle has no warm start: its candidates are
    re-drawn with the same key and nonce and the plan is compared with the
    oracle's."""
    from paper_2603_20525_gb300 import atp, serve
    vehicles = serve.resident_vehicles(fleet[:2])
    srv = serve.Server(vehicles, streams=2, slot_candidates=1 << 15, arena_bytes=64 << 20)
    trace = [serve.Request(0, 0, 2048, 30, 0.025, 0.0), serve.Request(1, 1, 1024, 40, 0.05, 0.0)]
    rec = srv.serve(trace)
    ctx = atp.Context(0)
    for r, f in zip(rec, fleet[:2]):
        ctrl = ctx.sample(r.N, r.H, 0.2, 0.3, tuple(int(k) for k in f.key), r.rid)
        torch.cuda.synchronize()
        ctrl_h = ctrl.cpu().numpy()
        w = gen.Workload("served", f.terrain, f.vehicle, f.cost, f.x0, ctrl_h,
                         trace[r.rid].dt, gen.n_substeps(trace[r.rid].dt))
        ter = ctx.terrain_prepare(torch.as_tensor(f.terrain.heights).cuda(), f.terrain.cell)
        o = ctx.plan(f.vehicle, f.cost, ter, [float(v) for v in f.x0], ctrl, w.dt, w.n_sub, want_xf=True)
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
        g.update(atp.decode_out(o["out"]))
        g["xf"] = g["xf"].T.copy()
        assert g["best_idx"] == r.best_idx and np.float32(g["best_cost"]) == np.float32(r.best_cost)
        ref = oracle.plan(f.vehicle, f.cost, oracle.Terrain.of(f.terrain), f.x0, ctrl_h, w.dt, w.n_sub)
        check_plan(g, ref, w)
    ctx.close()


def test_largest_serving_request_full_size():
    """The serving mix's largest request at full size: 32768 candidates of
    150 steps at dt = 0.05 s (1500 Euler steps each) on a 2048^2 tile, drawn
    on the device and run through the batch path.  The reduction is checked
    bit-exactly over every output, and every candidate against the oracle."""
    from paper_2603_20525_gb300 import atp
    from tests.test_gpu_parity import check_candidates, lexmin
    f = gen.fleet(1, seed=3, sides=(2048,))[0]
    N, H, dt = 32768, 150, 0.05
    ctx = atp.Context(0)
    t = f.terrain
    ter = ctx.terrain_prepare(torch.as_tensor(t.heights).cuda(), t.cell, t.x0, t.y0)
    ctrl = ctx.sample(N, H, 0.2, 0.3, tuple(int(k) for k in f.key), 7)
    q = dict(veh=f.vehicle, cost=f.cost, terrain=ter, x0=[float(v) for v in f.x0], ctrl=ctrl, dt=dt,
             n_sub=0, out=atp.plan_outputs(N, H, xf=True))
    ctx.plan_batch([q])
    torch.cuda.synchronize()
    o = q["out"]
    g = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
    g.update(atp.decode_out(o["out"]))
    g["xf"] = g["xf"].T.copy()
    assert g["best_idx"] == lexmin(g["cost"], g["flags"])
    assert g["n_feasible"] == int(np.count_nonzero(g["flags"] & 1))
    ws = gen.Workload("serving-largest", f.terrain, f.vehicle, f.cost, f.x0, ctrl.cpu().numpy(), dt,
                      gen.n_substeps(dt))
    check_candidates({k: g[k] for k in ("cost", "margin", "flags", "xf")},
                     oracle.plan(f.vehicle, f.cost, oracle.Terrain.of(f.terrain), f.x0, ws.ctrl, dt, ws.n_sub), ws)
    ctx.close()
