"""Pins of the FP64 tape adjoint (oracle/adjoint.cpp): its templated model
reproduces srb.c's cost bit for bit; its gradient matches a closed form on
level ground and FP64 central finite differences (h = 1e-6) on the rough
plain terrain wherever the cost is smooth at that scale."""
import numpy as np
import pytest

import gen
import oracle


def flat(n=512, cell=0.5, x0=-10.0, y0=-128.0):
    return oracle.Terrain(np.zeros((n, n), np.float32), cell, x0, y0)


def test_templated_model_reproduces_srb_c():
    for w in (gen.workload_plain(0, N=16, H=40), gen.workload_plain(3, N=16, H=100, dt=0.02)):
        t = oracle.Terrain.of(w.terrain)
        r = oracle.rollout(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
        J, _ = oracle.grad(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
        assert np.array_equal(J, r["J"])


def test_gradient_closed_form_straight_acceleration():
    """Level ground, straight, tire forces zero, goal far ahead on the x axis:
    x_S = x0 + h sum_s v_s with v_{s+1} = v_s + h a_k, so an acceleration held
    over control step k moves x_S by h^2 sum_{s in k} (S - 1 - s), and the
    terminal cost w_g (x_g - x_S) has d/da_k = -w_g h^2 sum (S - 1 - s).  The
    rear longitudinal constraint force that holds the acceleration also pitches
    the chassis by about 1e-3 rad, which bends the world x velocity at second
    order: the closed form holds to ~2e-5 of the largest component."""
    v = dict(gen.vehicle_baseline(), C=0.0)
    c = gen.cost_default(1000.0, 0.0)
    t = flat()
    x0 = np.zeros(13, np.float32)
    x0[2] = v["hR"]
    x0[6] = 6.0
    H, n_sub, dt = 12, 5, 0.05
    h = dt / n_sub
    ctrl = np.zeros((H, 1, 2), np.float32)
    ctrl[:, 0, 1] = np.linspace(-0.3, 0.4, H).astype(np.float32)
    J, G = oracle.grad(v, c, t, x0, ctrl, dt, n_sub)
    S = H * n_sub
    for k in range(H):
        want = -c["wg"] * h * h * sum(S - 1 - s for s in range(k * n_sub, (k + 1) * n_sub))
        assert G[k, 0, 1] == pytest.approx(want, abs=5e-5 * 0.4275)
        # steering rate: w_c delta_dot^2 is zero at zero rate, and nothing
        # steers without tire forces, so its gradient is zero too
        assert abs(G[k, 0, 0]) < 1e-9


def fd(w, t, j, k, c, step=1e-6):
    u = w.ctrl[:, j, :].astype(np.float64)
    up, dn = u.copy(), u.copy()
    up[k, c] += step
    dn[k, c] -= step
    x0 = (w.x0[j] if w.x0.ndim == 2 else w.x0).astype(np.float64)
    return (oracle.cost_f64(w.vehicle, w.cost, t, x0, up, w.dt, w.n_sub) -
            oracle.cost_f64(w.vehicle, w.cost, t, x0, dn, w.dt, w.n_sub)) / (2 * step)


def test_gradient_against_central_differences():
    """Candidates of the plain workload at H = 100, dt = 0.02 s.  Components
    whose central difference is not stable between h = 1e-6 and h = 1e-5 sit
    on a kink of the model (a contact switch or the steering clamp) and are
    skipped; at least 70 % must be smooth and every smooth one must agree."""
    w = gen.workload_plain(5, N=6, H=100, dt=0.02)
    t = oracle.Terrain.of(w.terrain)
    J, G = oracle.grad(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    rng = np.random.default_rng(0)
    smooth = checked = 0
    for j in range(w.N):
        for k in rng.choice(w.H, 8, replace=False):
            for c in (0, 1):
                a, b = fd(w, t, j, k, c, 1e-6), fd(w, t, j, k, c, 1e-5)
                checked += 1
                if abs(a - b) > 1e-3 * max(abs(a), 1e-2):
                    continue
                smooth += 1
                assert G[k, j, c] == pytest.approx(a, rel=2e-4, abs=2e-4), (j, k, c)
    assert smooth >= 0.7 * checked


@pytest.mark.parametrize("slope_deg", [37.0, -37.0])
def test_gradient_with_the_esm_soft_term_active(slope_deg):
    """A 37-degree cross slope rolls the chassis to |phi| ~ 0.65 rad, to one
    side or the other, where the ESM is under 10 % of its level-ground value
    and its soft cost (Sec. IV-B, IV-C) is active: the gradient through
    |phi| and the soft term against FP64 central differences."""
    import math
    v = gen.vehicle_baseline()
    c = gen.cost_default(1000.0, 0.0)
    n, cell = 256, 0.5
    ys = np.arange(n) * cell - 64.0
    hts = np.repeat((math.tan(math.radians(slope_deg)) * ys)[:, None], n, axis=1).astype(np.float32)
    ter = gen.Terrain(hts, cell, -10.0, -64.0)
    t = oracle.Terrain(hts, cell, -10.0, -64.0)
    x0 = gen.settled_state(ter, v, 0.0, 0.0, 0.0, 6.0)
    H, dt, n_sub = 20, 0.05, 5
    rng = np.random.default_rng(1)
    ctrl = np.stack([rng.normal(0, 0.2, (H, 4)), rng.normal(0, 0.3, (H, 4))], -1).astype(np.float32)
    w = gen.Workload("side-slope", ter, v, c, x0, ctrl, dt, n_sub)
    tr = oracle.trajectory(v, c, t, x0, ctrl[:, 0, :], dt, n_sub)
    states = tr["states"] if isinstance(tr, dict) else tr[0]
    assert np.all(np.sign(states[:, 5]) == math.copysign(1.0, slope_deg))   # rising to the left: positive roll
    u_min = min(oracle.esm(v, float(p), float(q)) for p, q in zip(states[:, 5], states[:, 4]))
    assert u_min < 0.1 * oracle.esm(v, 0.0, 0.0)
    J, G = oracle.grad(v, c, t, x0, ctrl, dt, n_sub)
    smooth = checked = 0
    for j in range(4):
        for k in (0, 3, 7, 12, 18):
            for comp in (0, 1):
                a, b = fd(w, t, j, k, comp, 1e-6), fd(w, t, j, k, comp, 1e-5)
                checked += 1
                if abs(a - b) > 1e-3 * max(abs(a), 1e-2):
                    continue
                smooth += 1
                assert G[k, j, comp] == pytest.approx(a, rel=2e-4, abs=2e-4), (j, k, comp)
    assert smooth >= 0.7 * checked


def fd_margin(w, t, j, k, c, step):
    u = w.ctrl[:, j, :].astype(np.float64)
    up, dn = u.copy(), u.copy()
    up[k, c] += step
    dn[k, c] -= step
    x0 = (w.x0[j] if w.x0.ndim == 2 else w.x0).astype(np.float64)
    return (oracle.margin_f64(w.vehicle, w.cost, t, x0, up, w.dt, w.n_sub) -
            oracle.margin_f64(w.vehicle, w.cost, t, x0, dn, w.dt, w.n_sub)) / (2 * step)


@pytest.mark.parametrize("slope_deg", [0.0, 20.0, -20.0])
def test_margin_gradient_against_central_differences(slope_deg):
    """The ESM margin (min U_ESM over the trajectory, Sec. IV-B) and its tape
    gradient: the margin equals the oracle's, the gradient matches FP64
    central differences wherever the margin is smooth at that scale (the
    state holding the minimum does not change under the step), and it is
    exactly zero for every control applied after that state (causality)."""
    import math
    v = gen.vehicle_baseline()
    c = gen.cost_default(1000.0, 0.0)
    n, cell = 256, 0.5
    ys = np.arange(n) * cell - 64.0
    xs = np.arange(n) * cell - 10.0
    hts = (math.tan(math.radians(slope_deg)) * ys[:, None] + 0.3 * np.sin(xs[None, :] / 1.7)
           + 0.2 * np.cos(ys[:, None] / 2.3)).astype(np.float32)
    ter = gen.Terrain(hts, cell, -10.0, -64.0)
    t = oracle.Terrain(hts, cell, -10.0, -64.0)
    x0 = gen.settled_state(ter, v, 0.0, 0.0, 0.0, 7.0)
    H, dt, n_sub = 20, 0.05, 5
    rng = np.random.default_rng(3)
    ctrl = np.stack([rng.normal(0, 0.4, (H, 4)), rng.normal(0, 0.3, (H, 4))], -1).astype(np.float32)
    w = gen.Workload("margin", ter, v, c, x0, ctrl, dt, n_sub)
    M, G = oracle.grad_margin(v, c, t, x0, ctrl, dt, n_sub)
    r = oracle.rollout(v, c, t, x0, ctrl, dt, n_sub, want_step_margin=True)
    assert np.array_equal(M, r["margin"])
    smooth = checked = 0
    for j in range(4):
        kmin = int(np.argmin(r["step_margin"][:, j]))
        # controls after the minimum's control step cannot move it
        assert np.all(G[kmin + 1:, j, :] == 0.0)
        for k in range(0, kmin + 1, max(1, (kmin + 1) // 5)):
            for comp in (0, 1):
                a, b = fd_margin(w, t, j, k, comp, 1e-6), fd_margin(w, t, j, k, comp, 1e-5)
                checked += 1
                if abs(a - b) > 1e-3 * max(abs(a), 1e-1):
                    continue
                smooth += 1
                assert G[k, j, comp] == pytest.approx(a, rel=2e-4, abs=2e-3), (j, k, comp)
    assert smooth >= 0.6 * checked
    assert np.abs(G).max() > 1.0          # the margin does depend on the controls
