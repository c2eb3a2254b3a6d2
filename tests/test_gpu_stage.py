"""Terrain staging (ATP_OPT_STAGE_TERRAIN): a window of the texels copied
into each CTA's shared memory, the lookups inside it read from there (the
cached terrain lookups of Sec. IV-D).  The texel values are the same either
way, so a staged plan must give the unstaged one-lane plan's bits: every
candidate output, the argmin and the best candidate's controls and per-step
margins, for windows inside the map, clipped at its edges, covering all of a
small map, and of the smallest side."""
import math

import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu

KEYS = ("cost", "margin", "flags", "xf", "best_ctrl", "best_margin")


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_20525_gb300 import atp
    c = atp.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def plan(ctx, w, stage):
    from paper_2603_20525_gb300 import atp
    ctx.set_option(atp.OPT_LANES, 1)
    ctx.set_option(atp.OPT_STAGE_TERRAIN, stage)
    try:
        t = w.terrain
        ter = ctx.terrain_prepare(dev(t.heights), t.cell, t.x0, t.y0,
                                  costmap=None if t.costmap is None else dev(t.costmap))
        x0 = [float(v) for v in w.x0]
        o = ctx.plan(w.vehicle, w.cost, ter, x0, dev(w.ctrl), w.dt, w.n_sub, want_xf=True)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(atp.OPT_STAGE_TERRAIN, 0)
        ctx.set_option(atp.OPT_LANES, 0)
    r = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
    r.update(atp.decode_out(o["out"]))
    return r


def same_bits(a, b):
    """Equal bytes, NaN payloads included (candidates that tip over end
    with a non-finite state)."""
    return a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes()


def same(a, b):
    for k in KEYS:
        assert same_bits(a[k], b[k]), k
    for k in ("best_idx", "n_feasible", "best_cost", "best_min_margin", "best_min_step"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("side", [2, 64, 120])
def test_staged_plan_same_bits_paper_configuration(ctx, side):
    """The paper's real-time configuration (Sec. IV-D) on 8192 candidates:
    the fan of trajectories starts inside the window and leaves it."""
    w = gen.workload_paper(0, N=8192)
    same(plan(ctx, w, side), plan(ctx, w, 0))


def test_staged_plan_window_clipped_at_the_map_corner(ctx):
    """Start near the map's corner heading off the map: the window is moved
    inside the map, and the candidates leave both the window and the map."""
    w = gen.workload_paper(0, N=4096)
    x0 = gen.settled_state(w.terrain, w.vehicle, 3.0, 3.0, math.pi * 1.2, 6.0)
    wc = gen.Workload(w.name, w.terrain, w.vehicle, w.cost, x0, w.ctrl, w.dt, w.n_sub)
    a, b = plan(ctx, wc, 120), plan(ctx, wc, 0)
    assert np.count_nonzero(a["flags"] & 4) > 0          # some wheels queried off the map
    same(a, b)


def test_staged_plan_window_covers_a_small_map(ctx):
    """A map of 40 x 30 nodes, smaller than the window on both sides: the
    window is the whole map (with a costmap channel)."""
    w = gen.workload_plain(0, N=2048, H=20)
    t = w.terrain
    small = gen.Terrain(np.ascontiguousarray(t.heights[:30, :40]), t.cell, t.x0, t.y0,
                        costmap=np.full((30, 40), 0.5, np.float32), name="small")
    x0 = gen.settled_state(small, w.vehicle, t.x0 + 2.0, t.y0 + 3.0, 0.3, 3.0)
    ws = gen.Workload(w.name, small, w.vehicle, w.cost, x0, w.ctrl, w.dt, w.n_sub)
    same(plan(ctx, ws, 120), plan(ctx, ws, 0))


def test_staged_rollout_same_bits(ctx):
    """atp_rollout with staging: the per-candidate outputs and per-step
    margins of the unstaged one-lane rollout."""
    from paper_2603_20525_gb300 import atp
    w = gen.workload_paper(1, N=3000)
    t = w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, t.x0, t.y0)
    x0 = [float(v) for v in w.x0]
    outs = []
    ctx.set_option(atp.OPT_LANES, 1)
    for stage in (100, 0):
        ctx.set_option(atp.OPT_STAGE_TERRAIN, stage)
        r = ctx.rollout(w.vehicle, w.cost, ter, x0, dev(w.ctrl), w.dt, w.n_sub, want_step_margin=True)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in r.items()})
    ctx.set_option(atp.OPT_STAGE_TERRAIN, 0)
    ctx.set_option(atp.OPT_LANES, 0)
    assert outs[0].keys() == outs[1].keys()
    for k in outs[0]:
        assert same_bits(outs[0][k], outs[1][k]), k


def test_stage_option_values(ctx):
    from paper_2603_20525_gb300 import atp
    for bad in (1, 121, -3):
        with pytest.raises(RuntimeError):
            ctx.set_option(atp.OPT_STAGE_TERRAIN, bad)
    for ok in (0, 2, 120):
        ctx.set_option(atp.OPT_STAGE_TERRAIN, ok)
    ctx.set_option(atp.OPT_STAGE_TERRAIN, 0)
