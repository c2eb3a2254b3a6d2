"""The planar (EST) model on the GPU (atp_plan_est through the C-ABI) against
its FP64 oracle on the same seeded inputs: per-candidate cost, lateral-
acceleration margin, flags and final state under the conditioning-aware
protocol of tests/parity.py, the reduction bit-exactly over the GPU's own
outputs, with and without a distance-constraint costmap."""
import numpy as np
import pytest

import gen
import oracle
from tests import parity
from tests.test_gpu_parity import lexmin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_20525_gb300 import atp
    c = atp.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def gpu_est(ctx, w, costmap=None):
    from paper_2603_20525_gb300 import atp
    t = w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, t.x0, t.y0,
                              costmap=None if costmap is None else dev(costmap))
    xarg = dev(np.ascontiguousarray(w.x0.T)) if w.x0.ndim == 2 else [float(v) for v in w.x0]
    o = ctx.plan_est(w.vehicle, w.cost, ter, xarg, dev(w.ctrl), w.dt, w.n_sub, want_xf=True)
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
    r.update(atp.decode_out(o["out"]))
    r["xf"] = r["xf"].T.copy()
    return r


def check_est(g, w, costmap=None):
    ter = oracle.Terrain(w.terrain.heights, w.terrain.cell, w.terrain.x0, w.terrain.y0, costmap=costmap)
    o = oracle.est_plan(w.vehicle, w.cost, ter, w.x0, w.ctrl, w.dt, w.n_sub)
    cond = parity.conditioning(oracle, w.vehicle, w.cost, ter, w.x0, w.ctrl, w.dt, w.n_sub, o, model="est")
    v = parity.classify(g, o, cond, w.vehicle, model="est")
    print("parity", w.name, v["stats"])
    bad = np.nonzero(v["fail"])[0]
    assert bad.size == 0, [(int(j), float(v["err"][j]), float(v["bound"][j])) for j in bad[:5]]
    assert v["stats"]["tail"] <= v["stats"]["cap"], v["stats"]
    if v["stats"]["feasible"] >= 200:
        parity.assert_fp32_level(v["stats"])
    assert v["stats"]["switch_misses"] <= v["stats"]["switch_cap"], v["stats"]
    ck = v["checked"]
    assert np.array_equal(g["flags"][ck], o["flags"][ck])
    assert np.array_equal(g["flags"][~v["near"]] & 1, o["flags"][~v["near"]] & 1)
    # reduction: bit-exact over the GPU's own outputs
    assert g["best_idx"] == lexmin(g["cost"], g["flags"])
    assert g["n_feasible"] == int(np.count_nonzero(g["flags"] & 1))
    assert g["best_cost"] == g["cost"][g["best_idx"]]
    assert g["best_min_margin"] == g["margin"][g["best_idx"]]
    bc = w.ctrl[:, g["best_idx"], :].copy()
    dm = np.float32(w.vehicle["delta_rate_max"])
    bc[:, 0] = np.clip(bc[:, 0], -dm, dm)
    assert np.array_equal(g["best_ctrl"], bc)
    gb, ob = g["best_idx"], o["best"]
    if gb != ob:
        tie = abs(o["J"][gb] - o["J"][ob]) <= (v["bound"][gb] + v["bound"][ob]) * max(abs(o["J"][ob]), 1.0)
        assert tie or not v["checked"][ob], (gb, ob, o["J"][gb], o["J"][ob])
    if v["checked"][gb]:
        sm = o["step_margin"][:, gb] if gb == ob else oracle.est_rollout(
            w.vehicle, w.cost, ter, w.x0[gb] if w.x0.ndim == 2 else w.x0, w.ctrl[:, gb:gb + 1, :], w.dt,
            w.n_sub, want_step_margin=True)["step_margin"][:, 0]
        assert parity.rel(g["best_margin"], sm, parity.margin_floor(w.vehicle, "est")).max() <= v["bound"][gb]
    return v


@pytest.mark.parametrize("seed", [0, 1])
def test_est_plain_parity(ctx, seed):
    w = gen.workload_est(seed)
    check_est(gpu_est(ctx, w), w)


def test_est_scaled_parity_per_candidate_start(ctx):
    w = gen.workload_est(0, N=16384, H=100, dt=0.02, scaled=True)
    check_est(gpu_est(ctx, w), w)


def test_est_with_costmap_and_high_traction(ctx):
    """Obstacles and a path boundary through the costmap at the wheels, and a
    tire with mu > abar / g so that the lateral-acceleration constraint can
    bind (with mu = 0.6 it cannot on level ground).  mu = 1.8 puts the turns
    just past the bound; the protocol is the same as everywhere else."""
    w = gen.workload_est(2, N=2048, H=40)
    w.vehicle = dict(w.vehicle, mu=1.8)
    # constant steering rates from -1 to 1 rad/s: the sharper turns exceed abar
    ctrl = np.zeros((w.H, w.N, 2), np.float32)
    ctrl[:, :, 0] = np.linspace(-1.0, 1.0, w.N, dtype=np.float32)[None, :]
    ctrl[:, :, 1] = w.ctrl[:, :, 1]
    w.ctrl = ctrl
    cm, _ = oracle.costmap(gen.obstacles(w.terrain, 2), w.terrain.nx, w.terrain.ny, w.terrain.cell,
                           w.terrain.x0, w.terrain.y0)
    cm = cm.astype(np.float32)
    g = gpu_est(ctx, w, costmap=cm)
    check_est(g, w, costmap=cm)
    assert np.count_nonzero((g["flags"] & 1) == 0) > 10        # the constraint binds
    assert np.count_nonzero(g["cost"] > 1e5) > 10               # obstacles are hit


@pytest.mark.parametrize("N,H,n_sub", [(1, 1, 1), (33, 7, 3), (65, 40, 10)])
def test_est_ragged_sizes(ctx, N, H, n_sub):
    w = gen.workload_est(4, N=N, H=H)
    w.n_sub = n_sub
    check_est(gpu_est(ctx, w), w)


def test_est_goal_truncation(ctx):
    w = gen.workload_est(6, N=200, H=40)
    w.cost = dict(w.cost, goal_x=12.0)
    g = gpu_est(ctx, w)
    assert np.count_nonzero(g["flags"] & 2) > 100
    check_est(g, w)


def test_est_invalid_arguments(ctx):
    from paper_2603_20525_gb300 import atp
    w = gen.workload_est(0, N=8, H=4)
    ter = ctx.terrain_prepare(dev(w.terrain.heights), w.terrain.cell)
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan_est(w.vehicle, w.cost, ter, [float("nan")] * 7, dev(w.ctrl), w.dt)
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan_est(w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), 0.0)


def test_est_bf16_terrain_against_decoded_oracle(ctx):
    """The planar model on BF16 texels against the oracle fed the same decoded
    terrain (the host restatement of the format), which leaves arithmetic
    error only."""
    from paper_2603_20525_gb300 import atp
    w = gen.workload_est(3)
    t = w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, t.x0, t.y0, fmt=atp.BF16X4)
    o = ctx.plan_est(w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), w.dt, w.n_sub,
                     want_xf=True)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
    g.update(atp.decode_out(o["out"]))
    g["xf"] = g["xf"].T.copy()
    h_dec, gx, gy, _, _ = oracle.bf16_terrain(t.heights, t.cell)
    od = oracle.Terrain(h_dec, t.cell, t.x0, t.y0, gx=gx, gy=gy)
    ref = oracle.est_plan(w.vehicle, w.cost, od, w.x0, w.ctrl, w.dt, w.n_sub)
    cond = parity.conditioning(oracle, w.vehicle, w.cost, od, w.x0, w.ctrl, w.dt, w.n_sub, ref, model="est")
    v = parity.classify(g, ref, cond, w.vehicle, model="est")
    print("est bf16 vs decoded oracle", v["stats"])
    assert v["stats"]["fails"] == 0 and v["stats"]["tail"] <= v["stats"]["cap"]
    assert g["best_idx"] == lexmin(g["cost"], g["flags"])
