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
    sens = parity.conditioning(oracle, w.vehicle, w.cost, od, w.x0, w.ctrl, w.dt, w.n_sub, ref)
    v = parity.classify(g, ref, sens, w.vehicle)
    print("bf16 vs decoded oracle", v["stats"])
    assert v["stats"]["fails"] == 0 and v["stats"]["tail"] <= v["stats"]["cap"]
    assert v["stats"]["switch_misses"] <= v["stats"]["cap"]
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
