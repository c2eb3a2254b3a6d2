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


@pytest.mark.parametrize("sigma", [0.3, 1.5])
def test_lod_ragged_and_small_maps(ctx, sigma):
    """Maps smaller than one CTA's tile and ragged against it, with the
    narrow windows (r = 12 cells) and the wide ones (r = 60)."""
    r = int(4 * sigma / 0.1 + 0.5)
    for shape in ((1, 1), (3, 700), (700, 3), (65, 33), (129, 2049)):
        f = np.random.default_rng(1).normal(0, 1, shape).astype(np.float32)
        g = ctx.lod_smooth(torch.as_tensor(f).cuda(), 0.1, sigma)
        torch.cuda.synchronize()
        o = oracle.lod_smooth(f, 0.1, sigma)
        assert np.abs(g.cpu().numpy() - o).max() <= 2 * (2 * r + 4) * U * np.abs(f).max()


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
    # without the distances, tiles skip the obstacles out of their reach:
    # the same bits
    cm2 = ctx.costmap(polys, t.nx, t.ny, t.cell, t.x0, t.y0)
    torch.cuda.synchronize()
    assert np.array_equal(cm2.cpu().numpy().astype(np.float64), cm)


def scattered(t, seed, n, r_lo, r_hi, on_tile_edges=False):
    """n small convex obstacles over the whole map, optionally centred on the
    corners of the costmap kernel's 16 x 16-node tiles."""
    rng = np.random.default_rng(seed)
    ext_x, ext_y = (t.nx - 1) * t.cell, (t.ny - 1) * t.cell
    out = []
    for _ in range(n):
        if on_tile_edges:
            cx = t.x0 + 16 * t.cell * rng.integers(1, max(2, t.nx // 16))
            cy = t.y0 + 16 * t.cell * rng.integers(1, max(2, t.ny // 16))
        else:
            cx, cy = t.x0 + rng.uniform(0, ext_x), t.y0 + rng.uniform(0, ext_y)
        k = int(rng.integers(3, 10))
        ang = np.sort(rng.uniform(0, 2 * np.pi, k))
        r = rng.uniform(r_lo, r_hi)
        out.append((np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], 1), 0))
    return out


@pytest.mark.parametrize("eps", [0.02, 0.25, 3.0])
@pytest.mark.parametrize("edges", [False, True])
def test_costmap_tile_skipping_keeps_the_bits(ctx, eps, edges):
    """Obstacles skipped per tile add exactly nothing: the costmap without
    distances (tiles skip obstacles beyond reach) equals the one with them
    (every perimeter at every node) bit for bit, for obstacles anywhere, on
    tile corners, larger than a tile, beside and across the path boundary,
    on a ragged map."""
    t = gen.terrain_plain(2)
    polys = scattered(t, 7, 60, 0.05, 0.8, edges) + scattered(t, 8, 4, 2.0, 6.0)
    polys = polys[:30] + gen.obstacles(t, 5, n=0) + polys[30:]        # boundary mid-list
    nx, ny = t.nx - 5, t.ny - 11
    full, _ = ctx.costmap(polys, nx, ny, t.cell, t.x0, t.y0, eps=eps, want_sdist=True)
    skip = ctx.costmap(polys, nx, ny, t.cell, t.x0, t.y0, eps=eps)
    torch.cuda.synchronize()
    full, skip = full.cpu().numpy(), skip.cpu().numpy()
    assert np.count_nonzero(full > 0) > 200
    assert np.array_equal(full.view(np.uint32), skip.view(np.uint32))


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
