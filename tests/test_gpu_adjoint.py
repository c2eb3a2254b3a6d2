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



@pytest.mark.parametrize("objective", ["cost", "margin"])
@pytest.mark.parametrize("ckpt", [10, 7])
def test_every_layout_same_bits(setup, objective, ckpt):
    """A small grid walks and recomputes on separate warps, a grid beyond
    one wave on the same quad; a CTA short of candidates leaves quads idle.
    The top-64's gradients, alone (split), as the first 50 (idle quads) and
    as 256 copies in a batch of 16384 (one quad per candidate), are the same
    bits, for a checkpoint interval that divides H and one that does not."""
    w = setup["w"]
    x0 = [float(v) for v in w.x0]

    def grad(ctrl):
        c = torch.as_tensor(np.ascontiguousarray(ctrl)).cuda()
        J, G = setup["ctx"].grad(w.vehicle, w.cost, setup["ter"], x0, c, w.dt, w.n_sub, ckpt,
                                 objective=objective)
        torch.cuda.synchronize()
        return J.cpu().numpy(), G.cpu().numpy()

    c64 = setup["ctrl"]
    J, G = grad(c64)
    J50, G50 = grad(c64[:, :50])
    assert J50.tobytes() == J[:50].tobytes() and G50.tobytes() == G[:, :50].tobytes()
    Jb, Gb = grad(np.tile(c64, (1, 256, 1)))
    assert Jb.tobytes() == np.tile(J, 256).tobytes()
    assert Gb.tobytes() == np.tile(G, (1, 256, 1)).tobytes()

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


def margin_ties(w, t, x0, ctrl, tol=1e-5):
    """Per candidate: is the smallest U_ESM over its states within `tol`
    (relative) of the next smallest?  Where it is, FP32 and FP64 may take the
    minimum at different states, and so their subgradients differ."""
    U0 = oracle.esm(w.vehicle, 0.0, 0.0)
    ties = []
    for j in range(ctrl.shape[1]):
        st, _, _ = oracle.trajectory(w.vehicle, w.cost, t, x0, ctrl[:, j, :], w.dt, w.n_sub)
        U = np.sort([oracle.esm(w.vehicle, float(s[5]), float(s[4])) for s in st])
        ties.append((U[1] - U[0]) / max(abs(U[0]), 0.01 * U0) < tol)
    return np.array(ties)


def compare_margin_gradients(Mg, Gg, Mo, Go, ties, U0):
    K = Mo.shape[0]
    assert np.max(np.abs(Mg - Mo) / np.maximum(np.abs(Mo), 0.01 * U0)) < 1e-4
    num = np.linalg.norm((Gg - Go).reshape(-1, K), axis=0)
    den = np.maximum(np.linalg.norm(Go.reshape(-1, K), axis=0), 1e-12)
    rel = (num / den)[~ties]
    print("margin gradient relative error (no tie): median", np.median(rel), "p90", np.quantile(rel, 0.9),
          "max", rel.max(), "ties", int(ties.sum()), "of", K)
    assert np.mean(~ties) >= 0.75
    assert np.median(rel) < 1e-4 and np.quantile(rel, 0.9) < 1e-3 and rel.max() < 1e-2


def test_margin_gradient_against_fp64_adjoint(setup):
    """atp_grad_margin: d(min U_ESM)/du of the top-64 candidates against the
    FP64 tape adjoint of the oracle's margin, away from ties of the minimum."""
    s = setup
    w = s["w"]
    c = torch.as_tensor(s["ctrl"]).cuda()
    M, G = s["ctx"].grad(w.vehicle, w.cost, s["ter"], [float(v) for v in w.x0], c, w.dt, w.n_sub,
                         objective="margin")
    torch.cuda.synchronize()
    Mo, Go = oracle.grad_margin(w.vehicle, w.cost, s["t"], w.x0, s["ctrl"], w.dt, w.n_sub)
    ties = margin_ties(w, s["t"], w.x0.astype(np.float64), s["ctrl"])
    compare_margin_gradients(M.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64), Mo, Go,
                             ties, oracle.esm(w.vehicle, 0.0, 0.0))
    # a few components against FP64 central differences of the margin
    rng = np.random.default_rng(4)
    Gg = G.cpu().numpy().astype(np.float64)
    checked = 0
    for j in rng.choice(np.nonzero(~ties)[0], 4, replace=False):
        u = s["ctrl"][:, j, :].astype(np.float64)
        for k in rng.choice(20, 4, replace=False):
            vals = []
            for hstep in (1e-6, 1e-5):
                up, dn = u.copy(), u.copy()
                up[k, 1] += hstep
                dn[k, 1] -= hstep
                vals.append((oracle.margin_f64(w.vehicle, w.cost, s["t"], w.x0.astype(np.float64), up, w.dt,
                                               w.n_sub) -
                             oracle.margin_f64(w.vehicle, w.cost, s["t"], w.x0.astype(np.float64), dn, w.dt,
                                               w.n_sub)) / (2 * hstep))
            if abs(vals[0] - vals[1]) > 1e-3 * max(abs(vals[0]), 1e-1):
                continue
            checked += 1
            assert abs(Gg[k, j, 1] - vals[0]) <= 1e-3 * max(abs(vals[0]), 1.0), (j, k, Gg[k, j, 1], vals[0])
    assert checked >= 8


@pytest.mark.parametrize("slope_deg", [37.0, -37.0])
def test_margin_gradient_on_a_steep_cross_slope(slope_deg):
    """Where the margin matters: a 37-degree cross slope, rising to either
    side, the chassis rolled to |phi| ~ 0.65 rad; the margin's gradient
    through |phi| against the FP64 tape adjoint."""
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
        M, G = ctx.grad(v, c, ter, [float(q) for q in x0], torch.as_tensor(ctrl).cuda(), dt, n_sub,
                        objective="margin")
        torch.cuda.synchronize()
        t = oracle.Terrain(hts, cell, -10.0, -64.0)
        Mo, Go = oracle.grad_margin(v, c, t, x0, ctrl, dt, n_sub)
        assert Mo.max() < 0.1 * oracle.esm(v, 0.0, 0.0)            # near the rollover bound
        w = gen.Workload("side-slope", ter_g, v, c, x0, ctrl, dt, n_sub)
        ties = margin_ties(w, t, x0.astype(np.float64), ctrl)
        compare_margin_gradients(M.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64), Mo, Go,
                                 ties, oracle.esm(v, 0.0, 0.0))
    finally:
        ctx.close()


def test_refinement_step_kernels():
    """The three step kernels against their definition: eta from the largest
    gradient component, the clamped trial step, and the per-candidate accept."""
    from paper_2603_20525_gb300 import atp
    ctx = atp.Context(0)
    try:
        rng = np.random.default_rng(7)
        H, K, rate_max = 13, 37, 1.0
        ctrl = rng.normal(0, 0.6, (H, K, 2)).astype(np.float32)
        G = rng.normal(0, 3.0, (H, K, 2)).astype(np.float32)
        c, g = torch.as_tensor(ctrl).cuda(), torch.as_tensor(G).cuda()
        eta = torch.empty(K, dtype=torch.float32, device="cuda")
        ctx.refine_init(g, 0.05, eta)
        trial = torch.empty_like(c)
        ctx.refine_trial(c, g, eta, rate_max, trial)
        torch.cuda.synchronize()
        e = eta.cpu().numpy()
        np.testing.assert_allclose(e, 0.05 / np.abs(G).reshape(H, K, 2).max(axis=(0, 2)), rtol=1e-6)
        want = ctrl.astype(np.float64) - e[None, :, None].astype(np.float64) * G
        want[..., 0] = np.clip(want[..., 0], -rate_max, rate_max)
        np.testing.assert_allclose(trial.cpu().numpy(), want, rtol=1e-6, atol=1e-6)
        cost = torch.as_tensor(rng.uniform(10, 20, K).astype(np.float32)).cuda()
        tcost = cost.clone()
        tcost[::2] -= 1.0                               # even candidates improve
        tcost[5] = float("nan")                         # non-finite: rejected
        tg = torch.as_tensor(rng.normal(0, 1, (H, K, 2)).astype(np.float32)).cuda()
        c0, g0, cost0, e0 = c.clone(), g.clone(), cost.clone(), eta.clone()
        ctx.refine_accept(trial, tcost, tg, c, cost, g, eta)
        torch.cuda.synchronize()
        ok = np.isfinite(tcost.cpu().numpy()) & (tcost.cpu().numpy() < cost0.cpu().numpy())
        assert ok[0] and not ok[1] and not ok[5]
        okt = torch.as_tensor(ok).cuda()
        assert torch.equal(c, torch.where(okt[None, :, None], trial, c0))
        assert torch.equal(g, torch.where(okt[None, :, None], tg, g0))
        assert torch.equal(cost, torch.where(okt, tcost, cost0))
        np.testing.assert_allclose(eta.cpu().numpy(), np.where(ok, 1.5, 0.5) * e0.cpu().numpy(), rtol=1e-7)
    finally:
        ctx.close()


def test_margin_autograd_function(setup):
    from paper_2603_20525_gb300.autograd import RolloutMargin
    s = setup
    w = s["w"]
    x0 = [float(v) for v in w.x0]
    c = torch.as_tensor(s["ctrl"]).cuda().requires_grad_(True)
    m = RolloutMargin.apply(c, s["ctx"], w.vehicle, w.cost, s["ter"], x0, w.dt, w.n_sub)
    (-m.sum()).backward()
    _, G = s["ctx"].grad(w.vehicle, w.cost, s["ter"], x0, torch.as_tensor(s["ctrl"]).cuda(), w.dt, w.n_sub,
                         objective="margin")
    torch.cuda.synchronize()
    assert torch.equal(c.grad, -G)
