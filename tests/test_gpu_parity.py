"""GPU (sm_103a, through the C-ABI) against the FP64 oracle on the same
seeded inputs.  Per-candidate cost, ESM margin, flags and final state follow
the protocol in tests/parity.py; the reduction and the copies are checked
bit-exactly against the GPU's own per-candidate outputs."""
import math

import numpy as np
import pytest

import gen
import oracle
from tests import parity

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


def gpu_plan(ctx, w, x0=None, ctrl=None, terrain=None, want_xf=True):
    from paper_2603_20525_gb300 import atp
    t = terrain or w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, t.x0, t.y0,
                              costmap=None if t.costmap is None else dev(t.costmap))
    x0 = w.x0 if x0 is None else x0
    ctrl = w.ctrl if ctrl is None else ctrl
    xarg = dev(np.ascontiguousarray(x0.T)) if x0.ndim == 2 else [float(v) for v in x0]
    o = ctx.plan(w.vehicle, w.cost, ter, xarg, dev(ctrl), w.dt, w.n_sub, want_xf=want_xf)
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
    r.update(atp.decode_out(o["out"]))
    if "xf" in r:
        r["xf"] = r["xf"].T.copy()
    return r


def oracle_plan(w, x0=None, ctrl=None, terrain=None):
    t = oracle.Terrain.of(terrain or w.terrain)
    return oracle.plan(w.vehicle, w.cost, t, w.x0 if x0 is None else x0,
                       w.ctrl if ctrl is None else ctrl, w.dt, w.n_sub)


def lexmin(cost, flags):
    """Host restatement of the reduction over the GPU's own FP32 outputs."""
    inf = (flags & 1) == 0
    order = np.lexsort((np.arange(len(cost)), cost.astype(np.float32), inf))
    return int(order[0])


def check_candidates(g, o, w, ctrl=None, x0=None):
    """Per-candidate outputs (cost, margin, flags, final state) of the GPU
    against the oracle's on the same candidates."""
    ctrl = w.ctrl if ctrl is None else ctrl
    x0 = w.x0 if x0 is None else x0
    ter = oracle.Terrain.of(w.terrain)
    cond = parity.conditioning(oracle, w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, o)
    v = parity.classify(g, o, cond, w.vehicle)
    print("parity", w.name, v["stats"])
    # every feasible candidate agrees within max(1e-4, KAPPA x the FP32
    # reference's own error), except a capped few that took the other side of
    # a switch
    bad = np.nonzero(v["fail"])[0]
    assert bad.size == 0, [(int(j), float(v["err"][j]), float(v["bound"][j])) for j in bad[:5]]
    assert v["stats"]["tail"] <= v["stats"]["cap"], v["stats"]
    assert v["stats"]["switch_misses"] <= v["stats"]["switch_cap"], v["stats"]
    # the goal, off-map and non-finite bits agree on every candidate that
    # held the bound
    ck = v["checked"]
    assert np.array_equal(g["flags"][ck] & 0xFE, o["flags"][ck] & 0xFE)
    # the feasibility bit (feasible means min U > 0 and finite, Sec. IV-B)
    # agrees on every candidate away from a switch whose FP32 reference stays
    # in range.  Elsewhere FP32 arithmetic does not decide it, and either side
    # is accepted, counted against the switch cap: at the U = 0 switch itself
    # (for an angle within about 2.4e-4 rad of the tipping point 1 - sin
    # rounds to 0 in FP32, while FP64 keeps a margin of order 1e-8), and on a
    # wild candidate, one on which FP32 arithmetic itself (the reference on
    # the same inputs) misses the oracle by more than the largest bound or
    # ends finite where the oracle does not, or the other way round: a
    # tumbling chassis that FP32 and FP64 follow down different paths.
    fe_diff = (g["flags"] & 1) != (o["flags"] & 1)
    sure = ~v["near"] & ~v["wild"]
    assert not (sure & fe_diff).any(), np.nonzero(sure & fe_diff)[0][:5]
    other_side = int((fe_diff & ~sure & ~v["flipped"]).sum())
    print("feasibility decided the other way at a switch or on a wild candidate:", other_side)
    assert v["stats"]["switch_misses"] + other_side <= v["stats"]["switch_cap"], (other_side, v["stats"])
    # over the workload, as accurate as FP32 arithmetic itself
    if v["stats"]["feasible"] >= 200:
        parity.assert_fp32_level(v["stats"])
    return v


def check_plan(g, o, w, ctrl=None, x0=None):
    ctrl = w.ctrl if ctrl is None else ctrl
    x0 = w.x0 if x0 is None else x0
    ter = oracle.Terrain.of(w.terrain)
    v = check_candidates(g, o, w, ctrl, x0)
    # reduction: bit-exact over the GPU's own per-candidate outputs
    assert g["best_idx"] == lexmin(g["cost"], g["flags"])
    assert g["n_feasible"] == int(np.count_nonzero(g["flags"] & 1))
    assert g["best_cost"] == g["cost"][g["best_idx"]]
    assert g["best_min_margin"] == g["margin"][g["best_idx"]]
    # best controls are the chosen candidate's, steering rate clamped
    bc = ctrl[:, g["best_idx"], :].copy()
    dm = np.float32(w.vehicle["delta_rate_max"])
    bc[:, 0] = np.clip(bc[:, 0], -dm, dm)
    assert np.array_equal(g["best_ctrl"], bc)
    # the chosen index equals the oracle's unless the two are tied within
    # their bounds or the oracle's winner is not a checked candidate
    gb, ob = g["best_idx"], o["best"]
    if gb != ob:
        tie = abs(o["J"][gb] - o["J"][ob]) <= (v["bound"][gb] + v["bound"][ob]) * max(abs(o["J"][ob]), 1.0)
        assert tie or not v["checked"][ob], (gb, ob, o["J"][gb], o["J"][ob])
    # per-step margins of the best candidate
    sm = oracle.rollout(w.vehicle, w.cost, ter, x0[gb] if x0.ndim == 2 else x0,
                        ctrl[:, gb:gb + 1, :], w.dt, w.n_sub, want_step_margin=True)["step_margin"][:, 0]
    if v["checked"][gb]:
        U0 = parity.level_esm(w.vehicle)
        assert parity.rel(g["best_margin"], sm, 0.01 * U0).max() <= v["bound"][gb]
    assert g["best_min_step"] == int(np.argmin(g["best_margin"]))
    return v["stats"]


def test_terrain_texels_match_oracle_gradients(ctx):
    w = gen.workload_plain(0)
    t = w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, t.x0, t.y0)
    tex = ter.texels.view(t.ny, t.nx, 4).cpu().numpy()
    ot = oracle.Terrain.of(t)
    assert np.array_equal(tex[..., 0], t.heights)
    np.testing.assert_allclose(tex[..., 1], ot.gx, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(tex[..., 2], ot.gy, rtol=1e-6, atol=1e-6)
    assert np.all(tex[..., 3] == 0)


def test_plain_plan_parity(ctx):
    w = gen.workload_plain(0)
    g = gpu_plan(ctx, w)
    o = oracle_plan(w)
    check_plan(g, o, w)


@pytest.mark.parametrize("seed", [1, 2])
def test_plain_plan_parity_other_seeds(ctx, seed):
    w = gen.workload_plain(seed)
    check_plan(gpu_plan(ctx, w), oracle_plan(w), w)


def test_scaled_plan_parity(ctx):
    """The benchmark workload (16384 candidates, H = 100, per-candidate speed)."""
    w = gen.workload_scaled(0)
    g = gpu_plan(ctx, w)
    o = oracle_plan(w)
    check_plan(g, o, w)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_lanes_option_parity(ctx, lanes):
    """Every thread layout, forced: one thread per candidate, a pair with one
    axle each, a quad with one wheel each, on both workloads and a ragged
    size."""
    from paper_2603_20525_gb300 import atp
    ctx.set_option(atp.OPT_LANES, lanes)
    try:
        for w in (gen.workload_plain(3), gen.workload_scaled(0), gen.workload_plain(4, N=33, H=7)):
            check_plan(gpu_plan(ctx, w), oracle_plan(w), w)
    finally:
        ctx.set_option(atp.OPT_LANES, 0)
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.set_option(atp.OPT_LANES, 3)


@pytest.mark.parametrize("case", ["plain", "goal", "costmap", "tipping"])
def test_every_lane_layout_same_bits(ctx, case):
    """A pair of lanes sums each axle and then the two axles, and a quad
    each axle by one shuffle and then the two axles by another, both in the
    order one lane uses, so the three layouts agree bit for bit.  With the
    goal 8 m ahead of the start, over half of the candidates reach it
    mid-horizon, where two lanes compute the step and discard it and one and
    four lanes skip it; with a costmap the lanes also sum the wheels' cost.
    The paper's configuration (3000 of its candidates) tips most of them
    over: their states diverge to huge and non-finite values, which the
    lanes' split sincos must treat exactly as one lane does."""
    from paper_2603_20525_gb300 import atp
    w = gen.workload_paper(0, N=3000) if case == "tipping" else gen.workload_scaled(3, N=3000, H=30)
    if case == "goal":
        w = gen.Workload(w.name, w.terrain, w.vehicle, dict(w.cost, goal_x=18.0), w.x0,
                         w.ctrl, w.dt, w.n_sub)
    terrain = None
    if case == "costmap":
        t = w.terrain
        xs, ys = t.grid()
        cm = (0.5 + 0.5 * np.sin(0.7 * xs) * np.cos(0.4 * ys)).astype(np.float32)
        terrain = gen.Terrain(t.heights, t.cell, t.x0, t.y0, costmap=cm, name="costmap")
    outs = []
    for lanes in (1, 2, 4):
        ctx.set_option(atp.OPT_LANES, lanes)
        outs.append(gpu_plan(ctx, w, terrain=terrain))
    ctx.set_option(atp.OPT_LANES, 0)
    if case == "goal":
        assert np.count_nonzero(outs[0]["flags"] & 2) > 1000      # ATP_FLAG_DONE
    if case == "tipping":
        assert np.count_nonzero(outs[0]["flags"] & 8) > 1000      # ATP_FLAG_NONFINITE
    for o in outs[1:]:
        for k in ("cost", "margin", "flags", "xf", "best_ctrl", "best_margin"):
            assert outs[0][k].tobytes() == o[k].tobytes(), k
        assert outs[0]["best_idx"] == o["best_idx"]


def test_paper_configuration_full_size(ctx):
    """The real-time configuration of Sec. IV-D at full size: 204,288
    candidates of 16 steps of 0.25 s (800 Euler steps of 5 ms), steering
    only, one thread per candidate.  The reduction is checked bit-exactly
    over all GPU outputs, and every output of every candidate against the
    oracle (about half of them tip over and end non-finite on both sides)."""
    w = gen.workload_paper(0)
    g = gpu_plan(ctx, w)
    assert g["best_idx"] == lexmin(g["cost"], g["flags"])
    assert g["n_feasible"] == int(np.count_nonzero(g["flags"] & 1))
    assert g["best_cost"] == g["cost"][g["best_idx"]]
    check_plan(g, oracle_plan(w), w)


def test_rollout_equals_plan_outputs(ctx):
    w = gen.workload_plain(0, N=300, H=12)
    ter = ctx.terrain_prepare(dev(w.terrain.heights), w.terrain.cell)
    p = ctx.plan(w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), w.dt, w.n_sub,
                 want_xf=True)
    r = ctx.rollout(w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), w.dt, w.n_sub,
                    want_xf=True, want_step_margin=True)
    torch.cuda.synchronize()
    for k in ("cost", "margin", "flags", "xf"):
        assert torch.equal(p[k], r[k]), k
    # consecutive plans on one context reuse the self-resetting scratch
    p2 = ctx.plan(w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), w.dt, w.n_sub)
    torch.cuda.synchronize()
    assert torch.equal(p["out"], p2["out"])


@pytest.mark.parametrize("N,H,n_sub", [(1, 1, 1), (33, 7, 3), (65, 40, 10), (1000, 5, 1)])
def test_ragged_sizes(ctx, N, H, n_sub):
    w = gen.workload_plain(4, N=N, H=H, dt=0.05)
    w.n_sub = n_sub
    check_plan(gpu_plan(ctx, w), oracle_plan(w), w)


@pytest.mark.parametrize("lanes", [1, 2, 4])
@pytest.mark.parametrize("slope_deg", [37.0, -37.0])
def test_steep_cross_slope_with_the_soft_constraint_active(ctx, slope_deg, lanes):
    """A 37-degree cross slope, rising to either side, rolls the chassis to
    |phi| ~ 0.65 rad while it slides down the slope: the ESM is under 10 % of
    its level-ground value, so its soft cost (Sec. IV-B, IV-C) is active at
    every step, for either sign of the roll, in every thread layout."""
    from paper_2603_20525_gb300 import atp
    v = gen.vehicle_baseline()
    c = gen.cost_default(1000.0, 0.0)
    n, cell = 256, 0.5
    ys = np.arange(n) * cell - 64.0
    hts = np.repeat((math.tan(math.radians(slope_deg)) * ys)[:, None], n, axis=1).astype(np.float32)
    ter = gen.Terrain(hts, cell, -10.0, -64.0)
    x0 = gen.settled_state(ter, v, 0.0, 0.0, 0.0, 6.0)
    H, dt, N = 20, 0.05, 1500
    rng = np.random.default_rng(2)
    ctrl = np.stack([rng.normal(0, 0.2, (H, N)), rng.normal(0, 0.3, (H, N))], -1).astype(np.float32)
    w = gen.Workload("cross-slope", ter, v, c, x0, ctrl, dt, gen.n_substeps(dt))
    ctx.set_option(atp.OPT_LANES, lanes)
    try:
        g = gpu_plan(ctx, w)
    finally:
        ctx.set_option(atp.OPT_LANES, 0)
    o = oracle_plan(w)
    U0 = parity.level_esm(v)
    assert np.all(o["margin"] < 0.1 * U0)           # the soft term acts on every candidate
    assert np.all(o["J"] > 1e5)
    check_plan(g, o, w)


def test_all_infeasible_and_ties(ctx):
    w = gen.workload_plain(5, N=96, H=10)
    x0 = np.repeat(w.x0[None, :], w.N, axis=0)
    x0[:, 5] = 1.1                          # rolled past tipping,
    x0[:, 2] += 5.0                          # falling freely for the whole horizon
    ctrl = w.ctrl.copy()
    ctrl[:, 40:48, :] = ctrl[:, 7:8, :]      # duplicates tie with candidate 7
    ww = gen.Workload(w.name, w.terrain, w.vehicle, w.cost, x0, ctrl, w.dt, w.n_sub)
    g = gpu_plan(ctx, ww)
    o = oracle_plan(ww)
    assert g["n_feasible"] == 0 and o["n_feasible"] == 0
    check_plan(g, o, ww, x0=x0, ctrl=ctrl)
    # nothing is feasible: the free fall is smooth, so every candidate's state
    # and cost still agree within the bound
    cond = parity.conditioning(oracle, ww.vehicle, ww.cost, oracle.Terrain.of(ww.terrain), x0, ctrl,
                               ww.dt, ww.n_sub, o)
    v = parity.classify(g, o, cond, ww.vehicle)
    assert np.all(v["ok"])
    assert g["best_idx"] not in range(40, 48)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_goal_truncation_and_offmap(ctx, lanes):
    """Goal truncation (Q4) and off-map lookups in every thread layout: the
    layouts handle a candidate at its goal differently (one and four lanes
    skip the step, two lanes compute and discard it)."""
    from paper_2603_20525_gb300 import atp
    ctx.set_option(atp.OPT_LANES, lanes)
    try:
        w = gen.workload_plain(6, N=200, H=40)
        c = dict(w.cost, goal_x=12.0)            # reached mid-horizon
        ww = gen.Workload(w.name, w.terrain, w.vehicle, c, w.x0, w.ctrl, w.dt, w.n_sub)
        g = gpu_plan(ctx, ww)
        o = oracle_plan(ww)
        assert np.count_nonzero(o["flags"] & oracle.DONE) > 100
        check_plan(g, o, ww)
        # start near the map corner so that candidates leave the map
        x0 = gen.settled_state(w.terrain, w.vehicle, 2.0, 2.0, math.pi * 1.25, 8.0)
        ww = gen.Workload(w.name, w.terrain, w.vehicle, w.cost, x0, w.ctrl, w.dt, w.n_sub)
        g = gpu_plan(ctx, ww)
        o = oracle_plan(ww)
        assert np.count_nonzero(o["flags"] & oracle.OFFMAP) > 100
        check_plan(g, o, ww)
    finally:
        ctx.set_option(atp.OPT_LANES, 0)


def test_nonfinite_controls_are_data(ctx):
    w = gen.workload_plain(7, N=64, H=8)
    ctrl = w.ctrl.copy()
    ctrl[3, 5, 0] = np.nan
    ctrl[2, 9, 1] = np.inf
    g = gpu_plan(ctx, w, ctrl=ctrl)
    for j in (5, 9):
        assert g["flags"][j] & 8 and not g["flags"][j] & 1
        assert np.isinf(g["cost"][j])
    assert g["best_idx"] not in (5, 9)


def test_invalid_arguments_rejected(ctx):
    from paper_2603_20525_gb300 import atp
    w = gen.workload_plain(0, N=8, H=4)
    ter = ctx.terrain_prepare(dev(w.terrain.heights), w.terrain.cell)
    x0 = [float(v) for v in w.x0]
    ctrl = dev(w.ctrl)
    bad = [dict(dt=0.0), dict(dt=float("nan")), dict(n_sub=-1)]
    for b in bad:
        with pytest.raises(atp.AtpError, match="INVALID"):
            ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, b.get("dt", w.dt), b.get("n_sub", 0))
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan(dict(w.vehicle, M=-1.0), w.cost, ter, x0, ctrl, w.dt)
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan(w.vehicle, dict(w.cost, wt=float("inf")), ter, x0, ctrl, w.dt)
    flat = torch.zeros(w.H * w.N * 2 + 1, dtype=torch.float32, device="cuda")
    misaligned = flat[1:].view(w.H, w.N, 2)           # float2 rows 4 bytes off
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan(w.vehicle, w.cost, ter, x0, misaligned, w.dt)
    with pytest.raises(atp.AtpError):
        ctx.terrain_prepare(dev(np.zeros((2, 2), np.float32)), 0.1)
