"""Continuous-batching pieces on the GPU: the candidate sampler against the
oracle's sampler, and the ragged batch kernel against single plans (bit for
bit), alone and in mixes of other plans, and against the FP64 oracle."""
import numpy as np
import pytest

import gen
import oracle
from tests import parity
from tests.test_gpu_parity import check_plan

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


@pytest.mark.parametrize("with_prev", [False, True])
def test_sampler_matches_oracle(ctx, with_prev):
    N, H = 3000, 37
    prev = None
    if with_prev:
        prev = np.stack([np.linspace(-0.3, 0.4, 25), np.linspace(0.1, -0.2, 25)], 1).astype(np.float32)
    g = ctx.sample(N, H, 0.2, 0.3, (12345, 678), 9, prev=None if prev is None else dev(prev), shift=1)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    o = oracle.sample(prev, 1, 0.2, 0.3, (12345, 678), 9, N, H)
    assert np.array_equal(g[:, 0, :], o[:, 0, :].astype(np.float32).astype(np.float64))
    err = np.abs(g - o) / np.maximum(np.abs(o), 0.3)
    assert err.max() < 2e-6, err.max()


def requests_mix():
    """Plans of different vehicles, terrains, sizes, horizons and steps."""
    rs = []
    w = gen.workload_plain(0, N=1000, H=20)
    rs.append(dict(w=w, x0=w.x0, name="plain-1000"))
    w = gen.workload_plain(2, N=333, H=57, dt=0.035)
    rs.append(dict(w=w, x0=w.x0, name="plain-333"))
    t = gen.terrain_tile(512, 3)
    veh = gen.vehicle_mrzr()
    x0 = gen.settled_state(t, veh, 25.0, 25.0, 0.7, 7.0)
    ctrl = gen.candidates(4096, 40, 5)
    w = gen.Workload("tile-4096", t, veh, gen.cost_default(40.0, 40.0), x0, ctrl, 0.025, 5)
    rs.append(dict(w=w, x0=x0, name="tile-4096"))
    w = gen.workload_scaled(1, N=2048, H=30)
    rs.append(dict(w=w, x0=w.x0, name="scaled-2048"))
    # above the four-lane limit: one thread per candidate inside the batch
    w = gen.workload_scaled(2, N=20000, H=12, terrain=w.terrain)
    rs.append(dict(w=w, x0=w.x0, name="scaled-20000"))
    return rs


def prepare(ctx, rs):
    from paper_2603_20525_gb300 import atp
    out = []
    for r in rs:
        w = r["w"]
        ter = ctx.terrain_prepare(dev(w.terrain.heights), w.terrain.cell, w.terrain.x0, w.terrain.y0)
        x0 = dev(np.ascontiguousarray(r["x0"].T)) if r["x0"].ndim == 2 else [float(v) for v in r["x0"]]
        out.append(dict(veh=w.vehicle, cost=w.cost, terrain=ter, x0=x0, ctrl=dev(w.ctrl), dt=w.dt,
                        n_sub=w.n_sub, w=w))
    return out


def fresh_outputs(q, xf=True):
    from paper_2603_20525_gb300 import atp
    H, N, _ = q["ctrl"].shape
    return atp.plan_outputs(N, H, xf=xf)


def same(a, b):
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_batch_equals_single_plans_bitwise(ctx):
    qs = prepare(ctx, requests_mix())
    singles = []
    for q in qs:
        o = fresh_outputs(q)
        ctx.plan(q["veh"], q["cost"], q["terrain"], q["x0"], q["ctrl"], q["dt"], q["n_sub"], out=o)
        singles.append(o)
    for q in qs:
        q["out"] = fresh_outputs(q)
    ctx.plan_batch(qs)
    torch.cuda.synchronize()
    for q, o in zip(qs, singles):
        same(q["out"], o)


def test_alone_and_in_any_mix_bitwise(ctx):
    qs = prepare(ctx, requests_mix())
    target = qs[2]
    target["out"] = fresh_outputs(target)
    ctx.plan_batch([target])
    torch.cuda.synchronize()
    alone = {k: v.clone() for k, v in target["out"].items()}
    rng = np.random.default_rng(0)
    for trial in range(4):
        others = [qs[i] for i in rng.permutation([0, 1, 3, 4])[: trial + 1]]
        mix = others + [target] if trial % 2 else [target] + others
        for q in mix:
            q["out"] = fresh_outputs(q)
        ctx.plan_batch(mix)
        torch.cuda.synchronize()
        same(target["out"], alone)


def test_two_lane_plan_alone_and_in_a_full_batch_bitwise(ctx):
    """A plan that runs two lanes alone (20000 candidates) keeps two lanes in
    a batch that leaves the GPU mostly empty and runs one lane in a batch of
    three such plans (60000 threads at one lane each, past a two-lane plan's
    own 57344); every layout gives the same bits, so it matches atp_plan
    either way."""
    qs = prepare(ctx, requests_mix())
    big = next(q for q in qs if q["ctrl"].shape[1] == 20000)
    assert ctx.plan_lanes(20000) == 2
    single = fresh_outputs(big)
    ctx.plan(big["veh"], big["cost"], big["terrain"], big["x0"], big["ctrl"], big["dt"], big["n_sub"],
             out=single)
    big["out"] = fresh_outputs(big)
    ctx.plan_batch([big])
    torch.cuda.synchronize()
    same(big["out"], single)
    trio = [dict(big, out=fresh_outputs(big)) for _ in range(3)]
    ctx.plan_batch(trio)
    torch.cuda.synchronize()
    for q in trio:
        same(q["out"], single)


def test_four_lane_plan_demoted_in_a_full_batch_bitwise(ctx):
    """A plan that runs four lanes alone (1000 candidates) keeps four in a
    batch that leaves room for them (alone, or ahead of two 20000-candidate
    plans, which then run one lane each) and runs one lane ahead of three of
    them (61000 threads at one lane each, past a two-lane plan's own 57344).
    Every layout gives the same bits, so it matches atp_plan in each."""
    qs = prepare(ctx, requests_mix())
    small = next(q for q in qs if q["ctrl"].shape[1] == 1000)
    big = next(q for q in qs if q["ctrl"].shape[1] == 20000)
    assert ctx.plan_lanes(1000) == 4
    single = fresh_outputs(small)
    ctx.plan(small["veh"], small["cost"], small["terrain"], small["x0"], small["ctrl"], small["dt"],
             small["n_sub"], out=single)
    for n_big in (0, 2, 3):
        mix = [dict(small, out=fresh_outputs(small))] + [dict(big, out=fresh_outputs(big)) for _ in range(n_big)]
        ctx.plan_batch(mix)
        torch.cuda.synchronize()
        same(mix[0]["out"], single)


def test_batched_plan_parity_with_oracle(ctx):
    qs = prepare(ctx, requests_mix())
    for q in qs:
        q["out"] = fresh_outputs(q)
    ctx.plan_batch(qs)
    torch.cuda.synchronize()
    from paper_2603_20525_gb300 import atp
    for q in qs:
        w = q["w"]
        g = {k: v.cpu().numpy() for k, v in q["out"].items() if k != "out"}
        g.update(atp.decode_out(q["out"]["out"]))
        g["xf"] = g["xf"].T.copy()
        o = oracle.plan(w.vehicle, w.cost, oracle.Terrain.of(w.terrain), w.x0, w.ctrl, w.dt, w.n_sub)
        check_plan(g, o, w)


def test_batch_validation(ctx):
    from paper_2603_20525_gb300 import atp
    qs = prepare(ctx, requests_mix())
    for q in qs:
        q["out"] = fresh_outputs(q)
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan_batch([])
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.plan_batch([qs[0]] * 65)
    bad = dict(qs[1], dt=0.0)
    with pytest.raises(atp.AtpError, match="request 1"):
        ctx.plan_batch([qs[0], bad, qs[2]])
