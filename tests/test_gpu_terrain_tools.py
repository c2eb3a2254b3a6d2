"""Terrain preprocessing on the GPU against the FP64 oracle: the Gaussian
level of detail (atp_lod_smooth) and the distance-constraint costmap
(atp_costmap), with tolerances derived from FP32 arithmetic."""
import math

import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24            # FP32 unit roundoff


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_20525_gb300 import atp
    c = atp.Context(0)
    yield c
    c.close()


def raw(n=300, m=257, seed=0):
    """An unsmoothed fBm heightmap with a berm and a ramp (raw plant terrain)."""
    rng = np.random.default_rng(seed)
    f = gen.fbm(max(n, m), 0.1, 0.8, seed, stream=31)[:m, :n]
    f = f + 0.05 * rng.standard_normal(f.shape)
    return np.ascontiguousarray(f, dtype=np.float32)


# Two FP32 passes of n = 2r+1 weighted terms each, weights rounded within a
# few ulp: |error| <= 2 (n + 3) u max|f|.
@pytest.mark.parametrize("cell,sigma", [(0.1, 0.3), (0.1, 1.5), (0.2, 1.5), (0.05, 0.3), (0.1, 0.0)])
def test_lod_matches_oracle(ctx, cell, sigma):
    f = raw()
    g = ctx.lod_smooth(torch.as_tensor(f).cuda(), cell, sigma)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    o = oracle.lod_smooth(f, cell, sigma)
    r = int(4 * sigma / cell + 0.5) if sigma > 0 else 0
    bound = 2 * (2 * r + 1 + 3) * U * np.abs(f).max()
    err = np.abs(g - o).max()
    print("lod", cell, sigma, r, err, bound)
    assert err <= bound
    if sigma == 0:
        assert np.array_equal(g, f.astype(np.float64))


def test_lod_ragged_and_small_maps(ctx):
    for shape in ((1, 1), (3, 700), (700, 3), (65, 33)):
        f = np.random.default_rng(1).normal(0, 1, shape).astype(np.float32)
        g = ctx.lod_smooth(torch.as_tensor(f).cuda(), 0.1, 0.3)
        torch.cuda.synchronize()
        o = oracle.lod_smooth(f, 0.1, 0.3)
        assert np.abs(g.cpu().numpy() - o).max() <= 2 * 28 * U * np.abs(f).max()


def test_lod_rejects_bad_arguments(ctx):
    from paper_2603_20525_gb300 import atp
    f = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(atp.AtpError, match="UNSUPPORTED"):
        ctx.lod_smooth(f, 0.01, 2.0)                  # radius 800 cells
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.lod_smooth(f, 0.1, -1.0)


def band(polys, ter_shape, cell, x0, y0, delta, eps=0.25, sigma=1e6):
    """Largest change of the summed cost when every signed distance moves by
    at most delta: sum over perimeters of sigma (v(s - delta)^2 - v(s)^2)."""
    ny, nx = ter_shape
    tot = np.zeros((ny, nx))
    for p in polys:
        _, s = oracle.costmap([p], nx, ny, cell, x0, y0, eps, sigma)
        v = np.maximum(0.0, 1.0 - s / eps)
        vd = np.maximum(0.0, 1.0 - (s - delta) / eps)
        tot += sigma * (vd * vd - v * v)
    return tot


@pytest.mark.parametrize("which", ["plain", "scaled"])
def test_costmap_matches_oracle(ctx, which):
    t = gen.terrain_plain(0) if which == "plain" else gen.terrain_scaled(1)
    polys = gen.obstacles(t, 3 if which == "plain" else 4, n=6)
    cm, sd = ctx.costmap(polys, t.nx, t.ny, t.cell, t.x0, t.y0, want_sdist=True)
    torch.cuda.synchronize()
    cm, sd = cm.cpu().numpy().astype(np.float64), sd.cpu().numpy().astype(np.float64)
    oc, os_ = oracle.costmap(polys, t.nx, t.ny, t.cell, t.x0, t.y0)
    # FP32 coordinates relative to the map corner: each distance within a few
    # ulp of the map's extent
    extent = max(t.nx, t.ny) * t.cell
    delta = 16 * U * extent
    assert np.abs(sd - os_).max() <= delta
    b = band(polys, (t.ny, t.nx), t.cell, t.x0, t.y0, delta)
    assert np.all(np.abs(cm - oc) <= b + 8 * U * oc + 1e-30)
    assert np.count_nonzero(oc > 0) > 100              # the obstacles cost something


def test_costmap_feeds_a_plan(ctx):
    """The GPU costmap as the texels' cost channel: a plan through obstacles
    avoids them (the best candidate's cost carries no obstacle term) while
    straight candidates that run into one pay for it."""
    w = gen.workload_plain(0, N=2048, H=40)
    t = w.terrain
    box = np.array([[20.0, 24.6], [22.0, 24.6], [22.0, 26.6], [20.0, 26.6]])   # on the nominal path
    cm = ctx.costmap([(box, 0)], t.nx, t.ny, t.cell, t.x0, t.y0)
    ter = ctx.terrain_prepare(torch.as_tensor(t.heights).cuda(), t.cell, t.x0, t.y0, costmap=cm)
    o = ctx.plan(w.vehicle, w.cost, ter, [float(v) for v in w.x0], torch.as_tensor(w.ctrl).cuda(), w.dt,
                 w.n_sub)
    torch.cuda.synchronize()
    cost = o["cost"].cpu().numpy()
    from paper_2603_20525_gb300 import atp
    best = atp.decode_out(o["out"])
    assert cost[0] > 1e5                       # the nominal drives into the box
    assert best["best_cost"] < 1e4


def test_costmap_rejects_bad_perimeters(ctx):
    from paper_2603_20525_gb300 import atp
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.costmap([(np.zeros((1, 2)), 0)], 8, 8, 0.1)
    with pytest.raises(atp.AtpError, match="INVALID"):
        ctx.costmap([(np.zeros((3, 2)), 2)], 8, 8, 0.1)
