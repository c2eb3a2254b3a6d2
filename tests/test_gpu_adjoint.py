"""The hand-written adjoint (atp_grad) on the GPU: gradients of the top-64
candidates of the plain plan at H = 100, dt = 0.02 s against the FP64 tape
adjoint and FP64 central differences; checkpoint-interval invariance; the
autograd Function; gradient refinement."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2603_20525_gb300 import atp
    ctx = atp.Context(0)
    w = gen.workload_plain(0, N=1024, H=100, dt=0.02)
    t = oracle.Terrain.of(w.terrain)
    r = oracle.rollout(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    order = np.lexsort((r["J"], (r["flags"] & 1) == 0))
    top = np.sort(order[:64])
    ctrl = np.ascontiguousarray(w.ctrl[:, top, :])
    ter = ctx.terrain_prepare(torch.as_tensor(w.terrain.heights).cuda(), w.terrain.cell)
    yield dict(ctx=ctx, w=w, t=t, ctrl=ctrl, ter=ter, top=top)
    ctx.close()


def gpu_grad(s, ctrl=None, ckpt=10):
    w = s["w"]
    c = torch.as_tensor(s["ctrl"] if ctrl is None else ctrl).cuda()
    J, G = s["ctx"].grad(w.vehicle, w.cost, s["ter"], [float(v) for v in w.x0], c, w.dt, w.n_sub, ckpt)
    torch.cuda.synchronize()
    return J.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64)


def test_gradient_against_fp64_adjoint(setup):
    s = setup
    w = s["w"]
    Jg, Gg = gpu_grad(s)
    Jo, Go = oracle.grad(w.vehicle, w.cost, s["t"], w.x0, s["ctrl"], w.dt, w.n_sub)
    assert np.max(np.abs(Jg - Jo) / Jo) < 1e-4
    num = np.linalg.norm((Gg - Go).reshape(-1, 64), axis=0)
    den = np.linalg.norm(Go.reshape(-1, 64), axis=0)
    rel = num / den
    print("gradient relative error per candidate: median", np.median(rel), "max", rel.max(),
          "quantiles", np.quantile(rel, [0.5, 0.9, 1.0]))
    cos = np.sum((Gg * Go).reshape(-1, 64), 0) / (np.linalg.norm(Gg.reshape(-1, 64), axis=0) * den)
    print("cosine", np.quantile(cos, [0, 0.1, 0.5]))
    assert np.median(rel) < 1e-4 and np.quantile(rel, 0.9) < 1e-3 and rel.max() < 1e-2
    assert np.quantile(cos, 0.1) > 0.99999


def test_gradient_against_central_differences(setup):
    """FP64 central differences (h = 1e-6) of the oracle's cost, where they are
    stable against h = 1e-5 (away from a kink of the model)."""
    s = setup
    w = s["w"]
    Jg, Gg = gpu_grad(s)
    rng = np.random.default_rng(1)
    ok = tot = 0
    errs = []
    for j in rng.choice(64, 6, replace=False):
        u = s["ctrl"][:, j, :].astype(np.float64)
        for k in rng.choice(w.H, 6, replace=False):
            for c in (0, 1):
                vals = []
                for hstep in (1e-6, 1e-5):
                    up, dn = u.copy(), u.copy()
                    up[k, c] += hstep
                    dn[k, c] -= hstep
                    vals.append((oracle.cost_f64(w.vehicle, w.cost, s["t"], w.x0.astype(np.float64), up,
                                                 w.dt, w.n_sub) -
                                 oracle.cost_f64(w.vehicle, w.cost, s["t"], w.x0.astype(np.float64), dn,
                                                 w.dt, w.n_sub)) / (2 * hstep))
                tot += 1
                if abs(vals[0] - vals[1]) > 1e-3 * max(abs(vals[0]), 1e-2):
                    continue
                ok += 1
                errs.append(abs(Gg[k, j, c] - vals[0]) / max(abs(vals[0]), 1e-1))
    print("FD: smooth", ok, "of", tot, "rel err median", np.median(errs), "max", np.max(errs))
    assert ok >= 0.6 * tot and np.median(errs) < 1e-4 and np.max(errs) < 1e-2


def test_checkpoint_interval_does_not_change_the_result(setup):
    J1, G1 = gpu_grad(setup, ckpt=1)
    J10, G10 = gpu_grad(setup, ckpt=10)
    J100, G100 = gpu_grad(setup, ckpt=100)
    assert np.array_equal(J1, J10) and np.array_equal(J10, J100)
    assert np.array_equal(G1, G10) and np.array_equal(G10, G100)


def test_autograd_function_and_refinement(setup):
    from paper_2603_20525_gb300.autograd import RolloutCost, refine
    s = setup
    w = s["w"]
    x0 = [float(v) for v in w.x0]
    c = torch.as_tensor(s["ctrl"]).cuda().requires_grad_(True)
    J = RolloutCost.apply(c, s["ctx"], w.vehicle, w.cost, s["ter"], x0, w.dt, w.n_sub)
    (2.0 * J.sum()).backward()
    _, G = gpu_grad(s)
    assert np.allclose(c.grad.cpu().numpy(), 2.0 * G)
    ctrl, hist = refine(s["ctx"], w.vehicle, w.cost, s["ter"], x0, torch.as_tensor(s["ctrl"]).cuda(),
                        w.dt, w.n_sub, iters=10)
    h = hist.cpu().numpy()
    assert np.all(np.diff(h, axis=0) <= 0)                       # never worse
    print("refinement: mean cost", h[0].mean(), "->", h[-1].mean(), "improved", np.mean(h[-1] < h[0]))
    assert np.mean(h[-1] < h[0]) > 0.8
    assert float(ctrl[..., 0].abs().max()) <= w.vehicle["delta_rate_max"]


@pytest.mark.parametrize("slope_deg", [37.0, -37.0])
def test_gradient_with_the_esm_soft_term_active(slope_deg):
    """A 37-degree cross slope rolls the chassis to |phi| ~ 0.65 rad, where
    the ESM is under 10 % of its level-ground value and its soft cost is
    active on every step: the GPU adjoint through |phi| and the soft term
    against the FP64 tape adjoint."""
    import math
    from paper_2603_20525_gb300 import atp
    ctx = atp.Context(0)
    try:
        v = gen.vehicle_baseline()
        c = gen.cost_default(1000.0, 0.0)
        n, cell = 256, 0.5
        ys = np.arange(n) * cell - 64.0
        hts = np.repeat((math.tan(math.radians(slope_deg)) * ys)[:, None], n, axis=1).astype(np.float32)
        ter_g = gen.Terrain(hts, cell, -10.0, -64.0)
        x0 = gen.settled_state(ter_g, v, 0.0, 0.0, 0.0, 6.0)
        H, dt, n_sub, K = 20, 0.05, 5, 16
        rng = np.random.default_rng(1)
        ctrl = np.stack([rng.normal(0, 0.2, (H, K)), rng.normal(0, 0.3, (H, K))], -1).astype(np.float32)
        ter = ctx.terrain_prepare(torch.as_tensor(hts).cuda(), cell, -10.0, -64.0)
        J, G = ctx.grad(v, c, ter, [float(q) for q in x0], torch.as_tensor(ctrl).cuda(), dt, n_sub)
        torch.cuda.synchronize()
        Jg, Gg = J.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64)
        t = oracle.Terrain(hts, cell, -10.0, -64.0)
        Jo, Go = oracle.grad(v, c, t, x0, ctrl, dt, n_sub)
        assert Jo.min() > 1e5                        # the soft term dominates the cost
        assert np.max(np.abs(Jg - Jo) / Jo) < 1e-4
        num = np.linalg.norm((Gg - Go).reshape(-1, K), axis=0)
        den = np.linalg.norm(Go.reshape(-1, K), axis=0)
        rel = num / den
        cos = np.sum((Gg * Go).reshape(-1, K), 0) / (np.linalg.norm(Gg.reshape(-1, K), axis=0) * den)
        print("side slope", slope_deg, "gradient relative error: median", np.median(rel), "max", rel.max(),
              "cosine min", cos.min())
        assert np.median(rel) < 1e-4 and rel.max() < 1e-3
        assert cos.min() > 0.99999
    finally:
        ctx.close()
