"""Precision variants on the GPU: terrain stored as BF16 (per-8x8-block FP32
height offset plus bf16 residuals and slopes) and the running cost
accumulated in FP64.  The BF16 texels are checked against an independent host
encoding, and a BF16 plan against the oracle fed that decoded terrain (so only
arithmetic error remains); the FP64 accumulation changes the cost only."""
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


def test_bf16_texels_match_host_encoding(ctx):
    from paper_2603_20525_gb300 import atp
    w = gen.workload_plain(0)
    t = w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, fmt=atp.BF16X4)
    raw = ter.texels.view(torch.int32).cpu().numpy().view(np.uint32)
    words = raw[: t.nx * t.ny * 2].reshape(t.ny, t.nx, 2)
    off = (t.nx * t.ny * 8 + 255) // 256 * 256 // 4
    nbx, nby = (t.nx + 7) // 8, (t.ny + 7) // 8
    plane_gpu = raw[off: off + nbx * nby * 4].view(np.float32).reshape(nby, nbx, 4)[..., :3]
    h_dec, gx, gy, (w_res, w_gx, w_gy), plane = oracle.bf16_terrain(t.heights, t.cell)
    assert np.array_equal(plane_gpu, plane)
    assert np.array_equal((words[..., 0] & 0xFFFF).astype(np.uint16), w_res)
    # slopes: FP32 on the device, FP64 on the host, then both rounded to bf16
    for got, want in (((words[..., 0] >> 16).astype(np.int64), w_gx.astype(np.int64)),
                      ((words[..., 1] & 0xFFFF).astype(np.int64), w_gy.astype(np.int64))):
        assert np.abs(got - want).max() <= 1 and np.mean(got != want) < 1e-3
    # quantisation of the heights: half a bf16 ulp of the residual
    res = np.abs(bf16_plane_residual(t.heights, plane))
    assert np.all(np.abs(h_dec - t.heights) <= 2.0 ** -8 * res + 1e-6)
    print("bf16 height quantisation: max", np.abs(h_dec - t.heights).max(), "m")


def bf16_plane_residual(H, plane):
    ny, nx = H.shape
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    P = plane[jj // 8, ii // 8].astype(np.float64)
    return H - (P[..., 0] + P[..., 1] * (ii & 7) + P[..., 2] * (jj & 7))


@pytest.mark.parametrize("seed", [0, 3])
def test_bf16_plan_parity_with_decoded_terrain(ctx, seed):
    from paper_2603_20525_gb300 import atp
    w = gen.workload_plain(seed)
    t = w.terrain
    ter = ctx.terrain_prepare(dev(t.heights), t.cell, fmt=atp.BF16X4)
    o = ctx.plan(w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), w.dt, w.n_sub,
                 want_xf=True)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
    g.update(atp.decode_out(o["out"]))
    g["xf"] = g["xf"].T.copy()
    h_dec, gx, gy, _, _ = oracle.bf16_terrain(t.heights, t.cell)
    dec = gen.Terrain(h_dec, t.cell, t.x0, t.y0, name="bf16-decoded")
    wd = gen.Workload(w.name, dec, w.vehicle, w.cost, w.x0, w.ctrl, w.dt, w.n_sub)
    od = oracle.Terrain(h_dec, t.cell, t.x0, t.y0, gx=gx, gy=gy)
    ref = oracle.plan(w.vehicle, w.cost, od, w.x0, w.ctrl, w.dt, w.n_sub)
    cond = parity.conditioning(oracle, w.vehicle, w.cost, od, w.x0, w.ctrl, w.dt, w.n_sub, ref)
    v = parity.classify(g, ref, cond, w.vehicle)
    print("bf16 vs decoded oracle", v["stats"])
    assert v["stats"]["fails"] == 0 and v["stats"]["tail"] <= v["stats"]["cap"]
    assert v["stats"]["switch_misses"] <= v["stats"]["switch_cap"]
    assert g["best_idx"] == int(np.lexsort((np.arange(w.N), g["cost"], (g["flags"] & 1) == 0))[0])


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_fp64_cost_accumulation_changes_cost_only(ctx, lanes):
    """In every thread layout (each has its own FP64-accumulating kernel),
    and through the batch kernel, which takes the choice at run time."""
    from paper_2603_20525_gb300 import atp
    w = gen.workload_plain(1)
    ter = ctx.terrain_prepare(dev(w.terrain.heights), w.terrain.cell)
    args = (w.vehicle, w.cost, ter, [float(v) for v in w.x0], dev(w.ctrl), w.dt, w.n_sub)
    ctx.set_option(atp.OPT_LANES, lanes)
    try:
        a = ctx.plan(*args, want_xf=True)
        ctx.set_option(atp.OPT_COST_FP64, 1)
        b = ctx.plan(*args, want_xf=True)
        # the batch kernel, with the same forced layout, takes FP64 at run time
        q = dict(veh=w.vehicle, cost=w.cost, terrain=ter, x0=[float(v) for v in w.x0],
                 ctrl=dev(w.ctrl), dt=w.dt, n_sub=w.n_sub, out=atp.plan_outputs(w.N, w.H, xf=True))
        ctx.plan_batch([q])
        torch.cuda.synchronize()
        for k in ("cost", "margin", "flags", "xf"):
            assert torch.equal(q["out"][k], b[k]), k
    finally:
        ctx.set_option(atp.OPT_COST_FP64, 0)
        ctx.set_option(atp.OPT_LANES, 0)
    torch.cuda.synchronize()
    for k in ("margin", "flags", "xf"):
        assert torch.equal(a[k], b[k]), k
    ref = oracle.rollout(w.vehicle, w.cost, oracle.Terrain.of(w.terrain), w.x0, w.ctrl, w.dt, w.n_sub)
    ca, cb = a["cost"].cpu().numpy().astype(np.float64), b["cost"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(ca - cb) / np.abs(cb)) < 2e-6
    # the FP64 sum is at least as close to the oracle on the median candidate
    ea = np.abs(ca - ref["J"]) / ref["J"]
    eb = np.abs(cb - ref["J"]) / ref["J"]
    print("cost error vs oracle: fp32 acc median", np.median(ea), "fp64 acc median", np.median(eb))
    assert np.median(eb) <= np.median(ea) * 1.05
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.set_option(99, 1)


def test_precision_over_64_seeds(ctx):
    """The precision table over 64 seeds of the plain plan (1024 candidates,
    H = 40, dt = 0.05 s), each GPU variant against the FP64 oracle:
      f32        FP32 terrain, FP32 arithmetic and cost accumulation
      f32+acc64  the same with the running cost accumulated in FP64
      bf16       BF16 terrain against the oracle on the FP32 terrain
                 (arithmetic plus quantisation error)
      bf16/dec   BF16 terrain against the oracle on the same decoded terrain
                 (arithmetic error only)
    Per variant: per-field maximum and median relative error over the feasible
    candidates (floors of tests/parity.py), feasibility-flag agreement over
    all candidates and the number of seeds whose chosen candidate agrees."""
    import json
    from paper_2603_20525_gb300 import atp
    fields = ("x", "y", "z", "psi", "theta", "phi", "vx", "vy", "vz", "wx", "wy", "wz", "delta", "J", "margin")
    acc = {k: dict(err=[], feas_agree=0, feas_n=0, argmin=0) for k in ("f32", "f32+acc64", "bf16", "bf16/dec")}
    seeds = 64
    for seed in range(seeds):
        w = gen.workload_plain(seed)
        t = w.terrain
        o32 = oracle.plan(w.vehicle, w.cost, oracle.Terrain.of(t), w.x0, w.ctrl, w.dt, w.n_sub)
        h_dec, gx, gy, _, _ = oracle.bf16_terrain(t.heights, t.cell)
        odec = oracle.plan(w.vehicle, w.cost, oracle.Terrain(h_dec, t.cell, t.x0, t.y0, gx=gx, gy=gy),
                           w.x0, w.ctrl, w.dt, w.n_sub)
        hd, ctrl, x0 = dev(t.heights), dev(w.ctrl), [float(v) for v in w.x0]
        runs = {}
        for fmt, opt in ((atp.F32X4, 0), (atp.F32X4, 1), (atp.BF16X4, 0)):
            ter = ctx.terrain_prepare(hd, t.cell, t.x0, t.y0, fmt=fmt)
            ctx.set_option(atp.OPT_COST_FP64, opt)
            try:
                o = ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, want_xf=True)
                torch.cuda.synchronize()
            finally:
                ctx.set_option(atp.OPT_COST_FP64, 0)
            g = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
            g.update(atp.decode_out(o["out"]))
            g["xf"] = g["xf"].T.copy()
            runs[(fmt, opt)] = g
        for name, g, ref in (("f32", runs[(atp.F32X4, 0)], o32), ("f32+acc64", runs[(atp.F32X4, 1)], o32),
                             ("bf16", runs[(atp.BF16X4, 0)], o32), ("bf16/dec", runs[(atp.BF16X4, 0)], odec)):
            c = parity.compare(g, ref, w.vehicle)
            feas = (ref["flags"] & 1) > 0
            a = acc[name]
            a["err"].append(np.concatenate([c["eX"], c["eJ"][:, None], c["eM"][:, None]], 1)[feas])
            a["feas_agree"] += int(np.sum((g["flags"] & 1) == (ref["flags"] & 1)))
            a["feas_n"] += len(feas)
            a["argmin"] += int(g["best_idx"] == ref["best"])
    table = {}
    for name, a in acc.items():
        e = np.concatenate(a["err"], 0)
        table[name] = dict(max_rel={n: float(v) for n, v in zip(fields, e.max(0))},
                           median_rel={n: float(v) for n, v in zip(fields, np.median(e, 0))},
                           strict=float(np.mean(e.max(1) <= parity.TOL)),
                           feasibility_agreement=a["feas_agree"] / a["feas_n"], argmin_agreement=a["argmin"])
    print(json.dumps(table, indent=1))
    # FP32 arithmetic on FP32 or decoded BF16 terrain: every choice agrees, and
    # every feasibility flag but the odd candidate whose margin crosses zero
    # within FP32 reach (at most 1 in 10^4)
    for name in ("f32", "f32+acc64", "bf16/dec"):
        assert table[name]["feasibility_agreement"] >= 0.9999, name
        assert table[name]["argmin_agreement"] == seeds, name
        assert table[name]["strict"] >= 0.999, name
    # FP64 accumulation moves the cost only
    assert table["f32+acc64"]["median_rel"]["z"] == table["f32"]["median_rel"]["z"]
    # BF16 storage: the quantised terrain is a slightly different problem
    assert table["bf16"]["feasibility_agreement"] >= 0.999
    assert table["bf16"]["argmin_agreement"] >= seeds - 4
