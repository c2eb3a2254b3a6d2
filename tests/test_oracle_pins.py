"""Pins of the FP64 oracle against facts that do not come from the oracle
itself: an independent rotation library, brute-force rigid-body geometry,
rigid-body mechanics in free flight, closed-form small-signal stiffness,
energy bookkeeping, mirror symmetry, the linear-bicycle neutral-steer result,
hand-summed costs and a brute-force argmin.  Each test names the passage of
arxiv 2603.20525 whose reading it fixes."""
import math

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator
from scipy.spatial.transform import Rotation

import gen
import oracle

VEH = gen.vehicle_baseline()


def flat(n=64, cell=0.5, z=0.0, x0=-16.0, y0=-16.0):
    return oracle.Terrain(np.full((n, n), z, dtype=np.float32), cell, x0, y0)


def no_cost(goal=(1e6, 0.0)):
    c = gen.cost_default(*goal)
    c["goal_r"] = 0.0
    return c


def veh(**kw):
    v = dict(VEH)
    v.update(kw)
    return v


def Rbar_phibar(v):
    return math.hypot(v["hR"], 0.5 * v["e"]), math.atan(2.0 * v["hR"] / v["e"])


# ---------------------------------------------------------------------------
# Sec. IV-A rotation matrix (3-2-1) against an independent rotation library
def test_rotation_matches_zyx_composition():
    rng = np.random.default_rng(1)
    for _ in range(50):
        psi, th, ph = rng.uniform(-3, 3), rng.uniform(-1.2, 1.2), rng.uniform(-3, 3)
        R = oracle.rotation(psi, th, ph)
        Rs = Rotation.from_euler("ZYX", [psi, th, ph]).as_matrix()
        assert np.max(np.abs(R - Rs)) < 1e-14


# Sec. III-A sigmoid tire model: odd, slope -C at 0, saturates at -/+ mu
def test_tire_model_limits_and_slope():
    Cc, mu = 6.1, 0.6
    for a in (0.01, 0.1, 0.5, 1.2):
        assert oracle.tire(Cc, mu, -a) == pytest.approx(-oracle.tire(Cc, mu, a), abs=1e-15)
    d = 1e-7
    slope = (oracle.tire(Cc, mu, d) - oracle.tire(Cc, mu, -d)) / (2 * d)
    assert slope == pytest.approx(-Cc, rel=1e-9)
    assert oracle.tire(Cc, mu, 1e6) == pytest.approx(-mu, rel=1e-9)
    assert oracle.tire(Cc, mu, -1e6) == pytest.approx(mu, rel=1e-9)
    assert oracle.tire(0.0, mu, 0.3) == 0.0
    assert oracle.tire(Cc, 0.0, 0.3) == 0.0


# ---------------------------------------------------------------------------
# Sec. IV-B ESM against brute-force rigid-body geometry: rotate the body about
# each support-polygon side edge until the CoM is over it; U = M g (height gain),
# negative once the CoM has crossed the edge.
def esm_bruteforce(v, phi, theta, psi=0.3):
    R = Rotation.from_euler("ZYX", [psi, theta, phi]).as_matrix()
    com = np.zeros(3)
    he = 0.5 * v["e"]
    best = None
    for side in (+1.0, -1.0):
        a = R @ np.array([v["Lf"], side * he, -v["hR"]])
        b = R @ np.array([-v["Lr"], side * he, -v["hR"]])
        u = (a - b) / np.linalg.norm(a - b)
        c0 = a + np.dot(com - a, u) * u          # circle centre on the edge
        r = np.linalg.norm(com - c0)
        zperp = np.array([0, 0, 1.0]) - u[2] * u  # up, projected off the axis
        top = c0[2] + r * np.linalg.norm(zperp)
        dh = top - com[2]
        # the CoM is outside the footprint when it lies beyond the edge, i.e.
        # when the horizontal direction from the edge to the CoM points away
        # from the other wheels
        other = R @ np.array([v["Lf"], -side * he, -v["hR"]])
        n = np.cross(u, [0, 0, 1.0])
        outside = np.sign(np.dot(com - c0, n)) != np.sign(np.dot(other - c0, n))
        Uside = (-1.0 if outside else 1.0) * v["M"] * v["g"] * dh
        best = Uside if best is None else min(best, Uside)
    return best


@pytest.mark.parametrize("vv", [VEH, gen.vehicle_mrzr()])
def test_esm_matches_bruteforce_geometry(vv):
    rng = np.random.default_rng(2)
    for _ in range(200):
        phi = rng.uniform(-1.4, 1.4)
        th = rng.uniform(-0.5, 0.5)
        assert oracle.esm(vv, phi, th) == pytest.approx(esm_bruteforce(vv, phi, th), abs=1e-9)


def test_esm_side_slope_and_tip_points():
    v = VEH
    Rb, pb = Rbar_phibar(v)
    Mg = v["M"] * v["g"]
    assert oracle.esm(v, 0.0, 0.0) == pytest.approx(Mg * (Rb - v["hR"]), rel=1e-13)
    tip = 0.5 * math.pi - pb
    assert abs(oracle.esm(v, tip, 0.0)) < 1e-9
    assert oracle.esm(v, tip - 1e-3, 0.0) > 0 > oracle.esm(v, tip + 1e-3, 0.0)
    # static 15 and 20 degree side slopes, chassis parallel to the slope
    for deg in (15.0, 20.0):
        u = oracle.esm(v, math.radians(deg), 0.0)
        assert u == pytest.approx(esm_bruteforce(v, math.radians(deg), 0.0), abs=1e-9)
        assert 0 < u < oracle.esm(v, 0.0, 0.0)


# ---------------------------------------------------------------------------
# Terrain lookup (reading Q10) against a library bilinear interpolator, and
# exactness on planes and for the gradient of a quadratic.
def test_terrain_bilinear_matches_library():
    rng = np.random.default_rng(3)
    Hm = rng.normal(size=(40, 50)).astype(np.float32)
    t = oracle.Terrain(Hm, 0.25, -3.0, 2.0)
    xs = -3.0 + 0.25 * np.arange(50)
    ys = 2.0 + 0.25 * np.arange(40)
    ref = RegularGridInterpolator((ys, xs), Hm.astype(np.float64), method="linear")
    for _ in range(300):
        x = rng.uniform(xs[0], xs[-1])
        y = rng.uniform(ys[0], ys[-1])
        out, off = t.sample(x, y)
        assert not off
        assert out[0] == pytest.approx(ref([y, x])[0], abs=1e-12)


def test_terrain_plane_exact_and_offmap_clamp():
    a, b, c = 0.5, 0.25, -0.125
    g = gen.terrain_plane(33, 29, 0.25, a, b, c, x0=-4.0, y0=-2.0)
    t = oracle.Terrain.of(g)
    rng = np.random.default_rng(4)
    for _ in range(100):
        x = rng.uniform(-4.0, -4.0 + 32 * 0.25)
        y = rng.uniform(-2.0, -2.0 + 28 * 0.25)
        out, off = t.sample(x, y)
        assert not off
        assert out[0] == pytest.approx(a + b * x + c * y, abs=1e-12)
        assert out[1] == pytest.approx(b, abs=1e-12)
        assert out[2] == pytest.approx(c, abs=1e-12)
    out, off = t.sample(100.0, -50.0)      # clamps to the corner node (nx-1, 0)
    assert off
    assert out[0] == pytest.approx(a + b * 4.0 + c * -2.0, abs=1e-12)


def test_terrain_gradient_exact_for_quadratic_interior():
    cell = 0.25
    xs = cell * np.arange(41)
    Hm = np.tile((xs ** 2).astype(np.float32), (9, 1))
    t = oracle.Terrain(Hm, cell)
    for x in (1.0, 2.3, 5.55, 8.9):
        out, _ = t.sample(x, 1.0)
        assert out[1] == pytest.approx(2 * x, abs=1e-9)
    # one-sided differences on the border nodes
    assert t.gx[0, 0] == pytest.approx((xs[1] ** 2 - xs[0] ** 2) / cell, abs=1e-9)
    assert t.gx[0, -1] == pytest.approx((xs[-1] ** 2 - xs[-2] ** 2) / cell, abs=1e-9)


# ---------------------------------------------------------------------------
# Sec. IV-A suspension extension on a tilted plane (reading Q1): a chassis
# parallel to the plane at perpendicular offset d has chi_i = d at every
# wheel; motion along the plane normal at rate w gives chi_dot = w.
def chassis_on_plane(v, b, c, psi, d, p_xy=(0.3, -0.2), a=0.5):
    n = np.array([-b, -c, 1.0])
    n /= np.linalg.norm(n)
    hx = np.array([math.cos(psi), math.sin(psi), 0.0])
    bx = hx - np.dot(hx, n) * n
    bx /= np.linalg.norm(bx)
    by = np.cross(n, bx)
    R = np.stack([bx, by, n], axis=1)
    yaw, th, ph = Rotation.from_matrix(R).as_euler("ZYX")
    q = np.array([p_xy[0], p_xy[1], a + b * p_xy[0] + c * p_xy[1]])
    p = q + (v["hR"] + d) * n
    xi = np.zeros(13)
    xi[0:3] = p
    xi[3:6] = (yaw, th, ph)
    return xi, R, n


@pytest.mark.parametrize("b,c,psi", [(0.25, 0.0, 0.0), (0.0, -0.25, 0.7), (0.25, 0.125, -2.0),
                                     (-0.375, 0.25, 2.5)])
def test_chi_equals_perpendicular_offset_on_tilted_plane(b, c, psi):
    g = gen.terrain_plane(81, 81, 0.25, 0.5, b, c, x0=-10.0, y0=-10.0)
    t = oracle.Terrain.of(g)
    for d in (0.0, 0.02, -0.03):
        xi, R, n = chassis_on_plane(VEH, b, c, psi, d)
        _, wheel, _ = oracle.evaluate(VEH, no_cost(), t, xi, [0.0, 0.0])
        chi = wheel[:, oracle.WHEEL_FIELDS.index("chi")]
        assert np.max(np.abs(chi - d)) < 1e-12
        # translate along the normal at w = 0.7 m/s (v_B = R^T n w)
        xi2 = xi.copy()
        xi2[6:9] = R.T @ (0.7 * n)
        _, wheel2, _ = oracle.evaluate(VEH, no_cost(), t, xi2, [0.0, 0.0])
        chidot = wheel2[:, oracle.WHEEL_FIELDS.index("chidot")]
        assert np.max(np.abs(chidot - 0.7)) < 1e-12
        # in-plane translation leaves chi unchanged
        xi3 = xi.copy()
        xi3[6:9] = R.T @ (3.0 * R[:, 0] + 1.0 * R[:, 1])
        _, wheel3, _ = oracle.evaluate(VEH, no_cost(), t, xi3, [0.0, 0.0])
        assert np.max(np.abs(wheel3[:, oracle.WHEEL_FIELDS.index("chidot")])) < 1e-12


# ---------------------------------------------------------------------------
# Rigid-body mechanics with every wheel in the air and the rear constraint
# force zeroed (zeta_2 chosen so): translational rows are g_B - omega x v,
# rotational rows are Euler's torque-free equations, position rates are R v,
# attitude rates reproduce omega under the library's rotation.
def test_free_flight_rigid_body_rows():
    rng = np.random.default_rng(5)
    t = flat()
    v = VEH
    J = np.diag([v["Jxx"], v["Jyy"], v["Jzz"]])
    for _ in range(20):
        xi = np.zeros(13)
        xi[0:2] = rng.uniform(-3, 3, 2)
        xi[2] = 5.0                                 # wheels far above the ground
        xi[3:6] = (rng.uniform(-3, 3), rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8))
        xi[6:9] = rng.uniform(-5, 5, 3)
        xi[9:12] = rng.uniform(-2, 2, 3)
        xi[12] = rng.uniform(-0.5, 0.5)
        R = Rotation.from_euler("ZYX", xi[3:6]).as_matrix()
        gB = R.T @ np.array([0.0, 0.0, -v["g"]])
        w, vb = xi[9:12], xi[6:9]
        zeta2 = gB[0] - (w[1] * vb[2] - w[2] * vb[1])       # rear F_x = 0
        xd, wheel, _ = oracle.evaluate(v, no_cost(), t, xi, [0.2, zeta2])
        assert np.all(wheel[:, oracle.WHEEL_FIELDS.index("Fz")] == 0.0)
        np.testing.assert_allclose(xd[0:3], R @ vb, atol=1e-12)
        acc = gB - np.cross(w, vb)
        np.testing.assert_allclose(xd[7:9], acc[1:3], atol=1e-12)
        assert xd[6] == pytest.approx(zeta2, abs=1e-15)
        wdot = np.linalg.solve(J, -np.cross(w, J @ w))
        np.testing.assert_allclose(xd[9:12], wdot, atol=1e-10)
        assert xd[12] == pytest.approx(0.2)
        # attitude rates: R(angles + eps*rates) ~ R (I + eps [w]x)
        eps = 1e-6
        Rp = Rotation.from_euler("ZYX", xi[3:6] + eps * xd[3:6]).as_matrix()
        Rm = Rotation.from_euler("ZYX", xi[3:6] - eps * xd[3:6]).as_matrix()
        W = R.T @ (Rp - Rm) / (2 * eps)
        np.testing.assert_allclose([W[2, 1], W[0, 2], W[1, 0]], w, atol=1e-6)


# ---------------------------------------------------------------------------
# Sec. IV-A suspension on level ground: static equilibrium at chi = 0 (the
# preloads F_s,i = g K_zz,i / 2 carry M g with no pitch moment), and the
# small-signal heave/pitch/roll stiffness of four springs.
def level_state(v, dz=0.0, th=0.0, ph=0.0, vx=0.0):
    xi = np.zeros(13)
    xi[2] = v["hR"] + dz
    xi[4] = th
    xi[5] = ph
    xi[6] = vx
    return xi


def test_level_ground_equilibrium_and_straight_line():
    v = VEH
    t = flat(n=256, cell=0.5, x0=-10.0, y0=-64.0)
    xi = level_state(v, vx=8.0)
    xd, wheel, body = oracle.evaluate(v, no_cost(), t, xi, [0.0, 0.0])
    expect = np.zeros(13)
    expect[0] = 8.0
    np.testing.assert_allclose(xd, expect, atol=1e-11)
    assert np.sum(body[19:23]) == pytest.approx(v["M"] * v["g"], rel=1e-14)
    # 2 s of straight driving: x = x0 + v t exactly, J = w_t T + w_g |goal - p_T|
    c = gen.cost_default(100.0, 0.0)
    ctrl = np.zeros((40, 2), dtype=np.float32)
    st, Jrun, ds = oracle.trajectory(v, c, t, xi, ctrl, 0.05, 10)
    assert ds == -1
    assert st[-1, 0] == pytest.approx(16.0, abs=1e-9)
    np.testing.assert_allclose(st[-1, 1:6], xi[1:6], atol=1e-12)
    r = oracle.rollout(v, c, t, xi.astype(np.float32), ctrl[:, None, :], 0.05, 10)
    assert r["J"][0] == pytest.approx(5.0 * 2.0 + 15.0 * (100.0 - 16.0), abs=1e-8)


@pytest.mark.parametrize("vv", [veh(C=0.0), dict(gen.vehicle_mrzr(), C=0.0)])
def test_small_signal_suspension_stiffness(vv):
    v = vv
    t = flat()
    kf, kr, Lf, Lr, he = v["kf"], v["kr"], v["Lf"], v["Lr"], 0.5 * v["e"]
    eps = 1e-6
    # heave
    xd, _, _ = oracle.evaluate(v, no_cost(), t, level_state(v, dz=eps), [0.0, 0.0])
    assert xd[8] == pytest.approx(-2 * (kf + kr) * eps / v["M"], rel=1e-5)
    assert xd[10] == pytest.approx(2 * (kf * Lf - kr * Lr) * eps / v["Jyy"], abs=1e-9)
    # pitch (positive theta lowers the nose); the rear constraint force that
    # holds v_x against g_Bx = g sin(theta) acts at h+R below the CoM
    xd, _, _ = oracle.evaluate(v, no_cost(), t, level_state(v, th=eps), [0.0, 0.0])
    My = -(2 * kf * Lf ** 2 + 2 * kr * Lr ** 2) * eps + v["M"] * v["g"] * v["hR"] * eps
    assert xd[10] == pytest.approx(My / v["Jyy"], rel=1e-5)
    # kf Lf - kr Lr nearly cancels for the MRZR: compare on the heave scale
    assert xd[8] == pytest.approx(2 * (kf * Lf - kr * Lr) * eps / v["M"], abs=1e-9)
    # roll (positive phi raises the left side)
    xd, _, _ = oracle.evaluate(v, no_cost(), t, level_state(v, ph=eps), [0.0, 0.0])
    assert xd[9] == pytest.approx(-2 * (kf + kr) * he ** 2 * eps / v["Jxx"], rel=1e-5)
    assert xd[7] == pytest.approx(-v["g"] * eps, rel=1e-5)


# ---------------------------------------------------------------------------
# Energy bookkeeping of the suspension (Sec. IV-A): pure heave drop of a
# fore-aft symmetric vehicle (L_f = L_r, so heave does not couple into pitch)
# with the tires inert (C = 0) and no damping.  E = M v^2/2 + M g z + sum V_i with the
# preloaded spring potential V_i = max(F_s,i - k chi, 0)^2 / (2 k) is conserved
# in continuous time; forward Euler drifts by O(h).  With damping E decays.
def heave_energy(v, states):
    Fs_f = 0.5 * v["g"] * v["M"] * v["Lr"] / (v["Lf"] + v["Lr"])
    Fs_r = 0.5 * v["g"] * v["M"] * v["Lf"] / (v["Lf"] + v["Lr"])
    chi = states[:, 2] - v["hR"]
    Vf = np.maximum(Fs_f - v["kf"] * chi, 0.0) ** 2 / (2 * v["kf"])
    Vr = np.maximum(Fs_r - v["kr"] * chi, 0.0) ** 2 / (2 * v["kr"])
    return 0.5 * v["M"] * states[:, 8] ** 2 + v["M"] * v["g"] * states[:, 2] + 2 * Vf + 2 * Vr


@pytest.mark.parametrize("drop", [-0.02, 0.15])   # start compressed / in the air
def test_heave_energy_conserved_to_order_h(drop):
    v = veh(C=0.0, bf=0.0, br=0.0, Lf=1.25, Lr=1.25)
    t = flat()
    xi = level_state(v, dz=drop)
    errs = []
    for n_sub in (50, 100, 200):
        ctrl = np.zeros((20, 2), dtype=np.float32)        # 1 s
        st, _, _ = oracle.trajectory(v, no_cost(), t, xi, ctrl, 0.05, n_sub)
        E = heave_energy(v, st)
        errs.append(np.max(np.abs(E - E[0])) / (v["M"] * v["g"] * v["hR"]))
        # the motion stays pure heave
        assert np.max(np.abs(st[:, [0, 1, 3, 4, 5, 6, 7, 9, 10, 11]])) < 1e-12
    assert errs[0] < 0.05
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_heave_energy_decays_with_damping():
    v = veh(C=0.0, Lf=1.25, Lr=1.25)
    t = flat()
    st, _, _ = oracle.trajectory(v, no_cost(), t, level_state(v, dz=0.1),
                                 np.zeros((40, 2), np.float32), 0.05, 100)
    E = heave_energy(v, st)
    E_eq = heave_energy(v, level_state(v)[None, :])[0]
    assert E[-1] - E_eq < 0.05 * (E[0] - E_eq)


# ---------------------------------------------------------------------------
# Mirror symmetry about y = y_c (the frames are right-handed, App. A): mirror
# the terrain, negate the steering rates and the y-odd state components; the
# trajectories mirror and every cost is identical.
def test_mirror_symmetry_of_rollout():
    w = gen.workload_plain(3, N=64, H=20)
    ter = w.terrain
    ny = ter.ny
    yc = ter.y0 + 0.5 * (ny - 1) * ter.cell
    Hm = ter.heights[::-1, :].copy()
    t1 = oracle.Terrain.of(ter)
    t2 = oracle.Terrain(Hm, ter.cell, ter.x0, ter.y0)
    odd = [3, 5, 7, 9, 11, 12]
    x0 = w.x0.astype(np.float64).copy()
    x0m = x0.copy()
    x0m[1] = 2 * yc - x0[1]
    x0m[odd] = -x0m[odd]
    ctrl_m = w.ctrl.copy()
    ctrl_m[..., 0] = -ctrl_m[..., 0]
    c2 = dict(w.cost, goal_y=2 * yc - w.cost["goal_y"])
    r1 = oracle.rollout(w.vehicle, w.cost, t1, x0.astype(np.float32), w.ctrl, w.dt, w.n_sub)
    r2 = oracle.rollout(w.vehicle, c2, t2, x0m.astype(np.float32), ctrl_m, w.dt, w.n_sub)
    # float32 inputs: the mirrored y0 must be exactly representable
    assert float(np.float32(x0m[1])) == x0m[1]
    np.testing.assert_allclose(r2["J"], r1["J"], rtol=1e-9)
    np.testing.assert_allclose(r2["margin"], r1["margin"], rtol=1e-9, atol=1e-6)
    xf1, xf2 = r1["xf"], r2["xf"]
    np.testing.assert_allclose(xf2[:, 1], 2 * yc - xf1[:, 1], atol=1e-7)
    np.testing.assert_allclose(xf2[:, odd], -xf1[:, odd], atol=1e-7)
    even = [0, 2, 4, 6, 8, 10]
    np.testing.assert_allclose(xf2[:, even], xf1[:, even], atol=1e-7)
    assert oracle.select(r1["J"], r1["flags"]) == oracle.select(r2["J"], r2["flags"])


# ---------------------------------------------------------------------------
# Planar reduction: load-proportional axle cornering stiffness (C F_z with
# F_z ~ L_r / L front, L_f / L rear) makes the linear bicycle neutral-steer,
# so on level ground a small held steering angle settles to yaw rate
# v_x delta / L and lateral acceleration v_x^2 delta / L.
@pytest.mark.parametrize("delta0,vx", [(0.01, 10.0), (-0.02, 6.0)])
def test_neutral_steer_steady_state(delta0, vx):
    v = VEH
    L = v["Lf"] + v["Lr"]
    t = flat(n=400, cell=0.5, x0=-100.0, y0=-100.0)
    xi = level_state(v, vx=vx)
    xi[12] = delta0
    xi[0], xi[1] = 0.0, 0.0
    st, _, _ = oracle.trajectory(v, no_cost(), t, xi, np.zeros((60, 2), np.float32), 0.1, 40)
    r = st[-1, 11]
    assert r == pytest.approx(vx * delta0 / L, rel=0.02)
    assert np.sign(r) == np.sign(delta0)       # positive steer turns left


# ---------------------------------------------------------------------------
# Sec. IV-C cost by hand on a one-step case: the ESM soft term is active
# (rolled chassis, U below 10 % of level ground), goal distance from the
# library rotation.
def test_one_step_cost_by_hand():
    v = veh(C=0.0)
    t = flat()
    Rb, pb = Rbar_phibar(v)
    phi = 0.5 * math.pi - pb - 0.05          # near tipping, U small and positive
    xi = np.zeros(13)
    xi[2] = 3.0                              # in the air: no contact forces
    xi[5] = phi
    xi[6] = 4.0
    xi[3] = 0.4
    c = gen.cost_default(20.0, 5.0)
    U = esm_bruteforce(v, phi, 0.0)
    U0 = esm_bruteforce(v, 0.0, 0.0)
    eps = 0.1 * U0
    assert 0 < U < eps
    h = 0.005
    zeta = np.array([[0.7, 0.0]], np.float32)
    st, Jrun, _ = oracle.trajectory(v, c, t, xi, zeta, h, 1)
    L = c["wt"] + c["wc"] * float(np.float32(0.7)) ** 2 + c["sigma"] * (1 - U / eps) ** 2
    assert Jrun[1] == pytest.approx(h * L, rel=1e-12)
    R = Rotation.from_euler("ZYX", xi[3:6]).as_matrix()
    p1 = xi[0:2] + h * (R @ xi[6:9])[0:2]
    np.testing.assert_allclose(st[1, 0:2], p1, atol=1e-14)
    r = oracle.rollout(v, c, t, xi.astype(np.float32), zeta[:, None, :], h, 1)
    xi32 = xi.astype(np.float32).astype(np.float64)
    U32 = esm_bruteforce(v, xi32[5], 0.0)
    R32 = Rotation.from_euler("ZYX", xi32[3:6]).as_matrix()
    p1 = xi32[0:2] + h * (R32 @ xi32[6:9])[0:2]
    J = h * (c["wt"] + c["wc"] * float(np.float32(0.7)) ** 2 + c["sigma"] * (1 - U32 / eps) ** 2) \
        + c["wg"] * math.hypot(p1[0] - 20.0, p1[1] - 5.0)
    assert r["J"][0] == pytest.approx(J, rel=1e-6)


# Reading Q6: the margin covers the final state too.
def test_margin_includes_final_state():
    v = veh(C=0.0)
    t = flat()
    xi = np.zeros(13)
    xi[2] = 3.0
    xi[5] = 0.2
    xi[9] = 2.0                               # rolling right away from level
    ctrl = np.zeros((1, 1, 2), np.float32)
    r = oracle.rollout(v, no_cost(), t, xi.astype(np.float32), ctrl, 0.01, 1,
                       want_step_margin=True)
    phi1 = float(np.float32(0.2)) + 0.01 * 2.0
    assert r["margin"][0] == pytest.approx(esm_bruteforce(v, phi1, 0.0), rel=1e-12)
    assert r["step_margin"][0, 0] == r["margin"][0]


# Reading Q4: goal truncation; state and cost freeze at the first Euler step
# that starts within r_g of the goal; Phi at the frozen state.
def test_goal_truncation_by_hand():
    v = VEH
    t = flat(n=256, cell=0.5, x0=-10.0, y0=-64.0)
    c = gen.cost_default(12.0, 0.0)
    xi = level_state(v, vx=8.0)
    h = 0.005
    ctrl = np.zeros((40, 1, 2), np.float32)
    r = oracle.rollout(v, c, t, xi.astype(np.float32), ctrl, 0.05, 10)
    # x_s = 8 h s; first s with 12 - x_s <= 2.5  ->  s = ceil(9.5 / 0.04)
    s = math.ceil(9.5 / (8 * h))
    x_done = 8 * h * s
    assert r["flags"][0] & oracle.DONE
    assert r["xf"][0, 0] == pytest.approx(x_done, abs=1e-9)
    assert r["J"][0] == pytest.approx(c["wt"] * h * s + c["wg"] * (12.0 - x_done), abs=1e-8)
    st, _, ds = oracle.trajectory(v, c, t, xi, ctrl[:, 0], 0.05, 10)
    assert ds == s


# Reading Q5 and the admissible control set: steering rate clamped to 1 rad/s
# before use (the cost sees the clamped rate), steering angle to delta_max.
def test_steering_clamps():
    v = VEH
    t = flat(n=256, cell=0.5, x0=-10.0, y0=-64.0)
    c = gen.cost_default(1e4, 0.0)
    c["goal_r"] = 0.0
    xi = level_state(v, vx=5.0)
    ctrl = np.zeros((20, 1, 2), np.float32)
    ctrl[:, 0, 0] = 5.0
    st, Jrun, _ = oracle.trajectory(v, c, t, xi, ctrl[:, 0], 0.05, 10)
    assert st[10, 12] == pytest.approx(0.05, abs=1e-12)        # rate 1 rad/s
    assert np.max(st[:, 12]) == v["delta_max"]
    assert Jrun[1] == pytest.approx(0.005 * (c["wt"] + c["wc"] * 1.0), rel=1e-12)


# ---------------------------------------------------------------------------
# Empirical argmin (Sec. IV-D, reading Q7) against an exhaustive sort.
def test_argmin_bruteforce_enumeration():
    w = gen.workload_plain(0)
    t = oracle.Terrain.of(w.terrain)
    seqs = np.array(np.meshgrid(*[[-1.0, 0.0, 1.0]] * 4, indexing="ij")).reshape(4, -1).T
    N = seqs.shape[0]
    ctrl = np.zeros((4, N, 2), np.float32)
    ctrl[:, :, 0] = seqs.T
    x0 = np.repeat(w.x0[None, :], N, axis=0)
    x0[::3, 5] = 1.2                          # rolled past tipping: infeasible
    r = oracle.rollout(w.vehicle, w.cost, t, x0, ctrl, 0.25, 50)
    keys = sorted((0 if r["flags"][j] & oracle.FEASIBLE else 1, r["J"][j], j) for j in range(N))
    assert oracle.select(r["J"], r["flags"]) == keys[0][2]
    assert not (r["flags"][0] & oracle.FEASIBLE) and (r["flags"][1] & oracle.FEASIBLE)


def test_argmin_ties_take_lowest_index_and_all_infeasible():
    J = np.array([3.0, 1.0, 1.0, 0.5, 1.0])
    F = np.array([1, 1, 1, 0, 1], np.uint8)
    assert oracle.select(J, F) == 1
    F0 = np.zeros(5, np.uint8)
    assert oracle.select(J, F0) == 3
    rng = np.random.default_rng(7)
    for n in (8, 17, 64):
        J = rng.integers(0, 4, n).astype(float)
        F = rng.integers(0, 2, n).astype(np.uint8)
        keys = sorted((1 - F[j], J[j], j) for j in range(n))
        assert oracle.select(J, F) == keys[0][2]


# ---------------------------------------------------------------------------
# Sec. IV-A suspension: forces only in contact and never attractive.  Over a
# grid of extensions and rates, F_z >= 0; F_z = 0 beyond the free length
# chi >= F_s / k; while the linear spring-damper force F_s - k chi - b chi_dot
# is positive in contact, F_z equals it.
def test_suspension_force_contact_and_never_attractive():
    v = veh(C=0.0, Lf=1.25, Lr=1.25)
    t = flat()
    Fs = 0.5 * v["g"] * 0.5 * v["M"]
    iz = oracle.WHEEL_FIELDS.index("Fz")
    for chi in np.linspace(-0.1, 0.12, 23):
        for vz in np.linspace(-3.0, 3.0, 25):
            xi = level_state(v, dz=chi)
            xi[8] = vz
            _, wheel, _ = oracle.evaluate(v, no_cost(), t, xi, [0.0, 0.0])
            Fz = wheel[0, iz]
            assert Fz >= 0.0
            lin = Fs - v["kf"] * chi - v["bf"] * vz
            if chi >= Fs / v["kf"]:
                assert Fz == 0.0
            elif lin > 0:
                assert Fz == pytest.approx(lin, rel=1e-12, abs=1e-9)
            else:
                assert Fz == 0.0


# Sec. IV-A summed forces and moments of a steered vehicle: the body-y force
# is the y component of each tire's lateral force turned by its steering
# angle, and the moment is the cross product of the contact offsets with the
# per-wheel forces (built here with a library rotation and numpy's cross).
def test_steered_force_and_moment_assembly():
    v = VEH
    t = flat()
    for delta in (0.0, 0.35, -0.6):
        xi = level_state(v, dz=-0.01, vx=6.0)
        xi[7] = 0.8                     # side slip so every tire carries force
        xi[12] = delta
        xd, wheel, body = oracle.evaluate(v, no_cost(), t, xi, [0.0, 0.0])
        F = np.zeros(3)
        Mom = np.zeros(3)
        rho = [(v["Lf"], 0.5 * v["e"]), (v["Lf"], -0.5 * v["e"]),
               (-v["Lr"], 0.5 * v["e"]), (-v["Lr"], -0.5 * v["e"])]
        for i in range(4):
            d = delta if i < 2 else 0.0
            lat = Rotation.from_euler("z", d).apply([0.0, wheel[i, oracle.WHEEL_FIELDS.index("Fy")], 0.0])
            Fi = np.array([wheel[i, oracle.WHEEL_FIELDS.index("Fx")], lat[1],
                           wheel[i, oracle.WHEEL_FIELDS.index("Fz")]])
            F += Fi
            Mom += np.cross([rho[i][0], rho[i][1], -v["hR"]], Fi)
        assert body[oracle.BODY_FIELDS.index("Fy")] == pytest.approx(F[1], rel=1e-12, abs=1e-9)
        np.testing.assert_allclose(xd[9:12] * [v["Jxx"], v["Jyy"], v["Jzz"]], Mom,
                                   rtol=1e-10, atol=1e-6)
        if delta != 0.0:
            assert abs(wheel[0, oracle.WHEEL_FIELDS.index("Fy")]) > 100.0


# Sec. IV-A extension rate: chi_dot is the exact time derivative of chi along
# a rigid motion that both translates and rotates (central differences of chi
# with the attitude advanced by the library's exponential map), on tilted
# planes with the chassis tilted against the plane and off its rest offset.
@pytest.mark.parametrize("b,c,psi", [(0.25, 0.0, 0.3), (0.125, -0.25, 2.0)])
def test_chi_rate_is_time_derivative_under_rotation(b, c, psi):
    g = gen.terrain_plane(81, 81, 0.25, 0.5, b, c, x0=-10.0, y0=-10.0)
    t = oracle.Terrain.of(g)
    v = VEH
    xi, R, n = chassis_on_plane(v, b, c, psi, 0.04)
    xi[4] += 0.1                       # tilt the chassis off the plane so that
    xi[5] -= 0.15                      # tau has body x and y components
    R = Rotation.from_euler("ZYX", xi[3:6]).as_matrix()
    rng = np.random.default_rng(11)
    ichi = oracle.WHEEL_FIELDS.index("chi")
    for _ in range(5):
        vb = rng.uniform(-2, 2, 3)
        w = rng.uniform(-1.5, 1.5, 3)
        xi[6:9] = vb
        xi[9:12] = w
        _, wheel, _ = oracle.evaluate(v, no_cost(), t, xi, [0.0, 0.0])
        chis = []
        for sgn in (+1.0, -1.0):
            e = sgn * 1e-6
            Rt = Rotation.from_euler("ZYX", xi[3:6]) * Rotation.from_rotvec(e * w)
            x2 = xi.copy()
            x2[0:3] = xi[0:3] + e * (R @ vb) + 0.5 * e * e * (R @ np.cross(w, vb))
            x2[3:6] = Rt.as_euler("ZYX")
            _, wh, _ = oracle.evaluate(v, no_cost(), t, x2, [0.0, 0.0])
            chis.append(wh[:, ichi])
        fd = (chis[0] - chis[1]) / 2e-6
        np.testing.assert_allclose(wheel[:, oracle.WHEEL_FIELDS.index("chidot")], fd, atol=2e-7)


# Sec. IV-C goal condition |p - goal| <= r_g, inclusive: with dyadic step
# sizes the distance hits r_g exactly, and that step is already the goal.
def test_goal_condition_is_inclusive():
    v = VEH
    t = flat(n=256, cell=0.5, x0=-10.0, y0=-64.0)
    c = gen.cost_default(12.0, 0.0)
    xi = level_state(v, vx=8.0)
    ctrl = np.zeros((40, 2), np.float32)
    st, _, ds = oracle.trajectory(v, c, t, xi, ctrl, 1.0 / 32.0, 8)   # h = 1/256 s
    assert ds == 304                  # x = 304 / 32 = 9.5 = 12 - 2.5 exactly
    assert st[ds, 0] == 9.5
