"""Pins of the FP64 oracle of the extended single-track (EST) planar model
(App. "Extended Single-Track Vehicle Dynamics Model", Sec. IV-C lateral-
acceleration constraint) against facts from outside the oracle: an
independent rotation library, the geometry of a plane's normal, textbook
static and longitudinal axle loads, the neutral-steer linear bicycle, the
static rollover threshold, exact bilinear interpolation of a linear costmap,
mirror symmetry, and the SRB oracle itself on level ground (the planar
reduction)."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import gen
import oracle

VEH = gen.vehicle_baseline()


def plane(a=0.0, b=0.0, n=200, cell=0.5, x0=-50.0, y0=-50.0, costmap=None):
    xs = x0 + cell * np.arange(n)
    ys = y0 + cell * np.arange(n)
    X, Y = np.meshgrid(xs, ys)
    return oracle.Terrain((a * X + b * Y).astype(np.float32), cell, x0, y0, costmap=costmap)


def no_goal():
    c = gen.cost_default(1e6, 0.0)
    c["goal_r"] = 0.0
    return c


def est_state(x=0.0, y=0.0, psi=0.0, vy=0.0, wz=0.0, delta=0.0, vx=8.0):
    return np.array([x, y, psi, vy, wz, delta, vx], dtype=np.float64)


# The 1-2-3 convention: roll about w_x, then pitch about the new y, then yaw
# about b_z, i.e. the intrinsic X-Y-Z composition.
def test_rotation_is_intrinsic_xyz():
    rng = np.random.default_rng(2)
    for _ in range(50):
        ph, th, ps = rng.uniform(-1.2, 1.2), rng.uniform(-1.2, 1.2), rng.uniform(-3, 3)
        R = oracle.est_rotation(ph, th, ps)
        Rs = Rotation.from_euler("XYZ", [ph, th, ps]).as_matrix()
        assert np.max(np.abs(R - Rs)) < 1e-14


# Pitch and roll come from the normal under the CoM: on any plane the body's
# vertical axis (third column of R) is the plane's unit normal, for any yaw,
# and the nose points up an uphill (reading Q1).
# (dyadic slopes: the FP32 heights of the plane are exact)
@pytest.mark.parametrize("a,b,psi", [(0.25, 0.0, 0.0), (0.0, -0.375, 1.0), (0.25, 0.125, -2.5)])
def test_body_vertical_is_plane_normal(a, b, psi):
    t = plane(a, b)
    _, d = oracle.est_evaluate(VEH, no_goal(), t, est_state(psi=psi), [0.0, 0.0])
    R = oracle.est_rotation(d["phi"], d["theta"], psi)
    n = np.array([-a, -b, 1.0]) / math.sqrt(a * a + b * b + 1)
    np.testing.assert_allclose(R[:, 2], n, rtol=0, atol=1e-12)
    # body x axis: its slope along the heading equals the plane's slope there
    bx = R[:, 0]
    assert bx[2] == pytest.approx(a * bx[0] + b * bx[1], abs=1e-12)
    # gravity in B is R^T (0, 0, -g) with the plane's geometry: |g_B| = g
    gB = np.array([d["gBx"], d["gBy"], d["gBz"]])
    assert np.linalg.norm(gB) == pytest.approx(VEH["g"], rel=1e-12)
    assert gB[2] == pytest.approx(-VEH["g"] / math.sqrt(a * a + b * b + 1), rel=1e-12)


def test_side_slope_gravity_points_downhill():
    beta = math.atan(0.25)                   # a dyadic slope: exact FP32 heights
    t = plane(0.0, 0.25)                     # rises towards +y
    _, d = oracle.est_evaluate(VEH, no_goal(), t, est_state(), [0.0, 0.0])
    assert d["phi"] == pytest.approx(beta, abs=1e-12)
    assert d["gBy"] == pytest.approx(-VEH["g"] * math.sin(beta), rel=1e-12)


# Virtual-tire normal forces: static axle loads M g L_r / L and M g L_f / L on
# level ground, and the longitudinal transfer M (h+R) a / L under acceleration.
@pytest.mark.parametrize("acc", [0.0, 2.0, -3.0])
def test_axle_loads_static_and_transfer(acc):
    v = VEH
    L = v["Lf"] + v["Lr"]
    _, d = oracle.est_evaluate(v, no_goal(), plane(), est_state(), [0.0, acc])
    assert d["Fzf"] == pytest.approx(v["M"] * v["g"] * v["Lr"] / L - v["M"] * v["hR"] * acc / L, rel=1e-12)
    assert d["Fzr"] == pytest.approx(v["M"] * v["g"] * v["Lf"] / L + v["M"] * v["hR"] * acc / L, rel=1e-12)
    assert d["Fzf"] + d["Fzr"] == pytest.approx(v["M"] * v["g"], rel=1e-12)


# Straight running on level ground: no slip, no lateral force, no yaw, and the
# position follows the heading.
def test_straight_line_level_ground():
    v = VEH
    psi = 0.7
    xd, d = oracle.est_evaluate(v, no_goal(), plane(), est_state(psi=psi, vx=9.0), [0.0, 0.5])
    np.testing.assert_allclose(xd, [9.0 * math.cos(psi), 9.0 * math.sin(psi), 0.0, 0.0, 0.0, 0.0, 0.5],
                               atol=1e-12)
    assert d["Fyf"] == 0.0 and d["Fyr"] == 0.0


# Neutral steer: load-proportional cornering stiffness makes the linear bicycle
# neutral, so a small held steering angle settles to yaw rate v_x delta / L,
# and the lateral acceleration that the constraint measures to v_x^2 delta / L.
@pytest.mark.parametrize("delta0,vx", [(0.01, 10.0), (-0.02, 6.0)])
def test_neutral_steer_and_lateral_acceleration(delta0, vx):
    v = VEH
    L = v["Lf"] + v["Lr"]
    t = plane(n=400, cell=0.5, x0=-100.0, y0=-100.0)
    st = oracle.est_trajectory(v, no_goal(), t, est_state(delta=delta0, vx=vx),
                               np.zeros((60, 2), np.float32), 0.1, 40)
    r = st[-1, 4]
    assert r == pytest.approx(vx * delta0 / L, rel=0.01)
    _, d = oracle.est_evaluate(v, no_goal(), t, st[-1], [0.0, 0.0])
    assert d["aBy"] == pytest.approx(vx * vx * delta0 / L, rel=0.01)
    # the static rollover threshold g e / (2 (h + R)) is the constraint's bound
    abar = v["g"] * v["e"] / (2 * v["hR"])
    assert d["margin"] == pytest.approx(abar - abs(d["aBy"]), rel=1e-12)


# Soft constraint onset at 10 % of the bound (reading Q2): zero cost at
# margin = 0.1 abar, sigma at margin 0, 4 sigma at margin -0.1 abar.  With
# mu < abar / g the lateral acceleration cannot reach the bound on level
# ground (the paper's traction argument), so this uses a high-traction tire.
def test_lateral_soft_constraint_values():
    v = dict(VEH, mu=1.6)
    abar = v["g"] * v["e"] / (2 * v["hR"])
    assert v["mu"] * v["g"] > abar
    c = no_goal()
    t = plane(n=400, cell=0.5, x0=-100.0, y0=-100.0)
    # level ground, pure side slip (w_z = 0, delta = 0): both tires push the
    # same way and |a_By - g_By| grows with v_By; bisect for the margin wanted
    for target, expect in ((0.1 * abar, 0.0), (0.0, c["sigma"]), (-0.1 * abar, 4 * c["sigma"])):
        lo, hi = 0.0, 10.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            _, d = oracle.est_evaluate(v, c, t, est_state(vy=mid, vx=10.0), [0.0, 0.0])
            if d["margin"] > target:
                lo = mid
            else:
                hi = mid
        _, d = oracle.est_evaluate(v, c, t, est_state(vy=lo, vx=10.0), [0.0, 0.0])
        assert d["margin"] == pytest.approx(target, abs=1e-9)
        assert d["L"] - c["wt"] == pytest.approx(expect, rel=1e-6, abs=1e-3)
    # with the paper's traction the bound is out of reach on level ground
    _, d = oracle.est_evaluate(VEH, c, t, est_state(vy=50.0, vx=10.0), [0.0, 0.0])
    assert abs(d["aBy"]) <= VEH["mu"] * VEH["g"] * (1 + 1e-12) < 0.9 * abar


# Distance constraints: the costmap is read at the four wheel contact points
# p + R rho_i.  A linear costmap is interpolated exactly, so the sum is
# 4 c(p) + (gradient) . R (2 (L_f - L_r), 0, -4 (h+R)).
@pytest.mark.parametrize("a,b,psi", [(0.0, 0.0, 0.4), (0.125, -0.0625, -1.1)])
def test_costmap_read_at_wheel_contact_points(a, b, psi):
    v = VEH
    n, cell, x0, y0 = 200, 0.5, -50.0, -50.0
    xs = x0 + cell * np.arange(n)
    X, Y = np.meshgrid(xs, xs)
    c0, cx, cy = 50.0, 3.0, -2.0            # exact in FP32 on this grid
    cm = (c0 + cx * X + cy * Y).astype(np.float32)
    t = plane(a, b, costmap=cm)
    c = no_goal()
    p = (1.3, -2.1)
    _, d = oracle.est_evaluate(v, c, t, est_state(x=p[0], y=p[1], psi=psi), [0.0, 0.0])
    R = oracle.est_rotation(d["phi"], d["theta"], psi)
    srho = np.array([2 * (v["Lf"] - v["Lr"]), 0.0, -4 * v["hR"]])
    off = R @ srho
    expect = 4 * (c0 + cx * p[0] + cy * p[1]) + cx * off[0] + cy * off[1]
    got = d["cm_fl"] + d["cm_fr"] + d["cm_rl"] + d["cm_rr"]
    assert got == pytest.approx(expect, rel=1e-12)
    assert d["L"] == pytest.approx(c["wt"] + got, rel=1e-12)


def test_mirror_symmetry_of_est_rollout():
    w = gen.workload_plain(5, N=48, H=20)
    ter = w.terrain
    yc = ter.y0 + 0.5 * (ter.ny - 1) * ter.cell
    t1 = oracle.Terrain.of(ter)
    t2 = oracle.Terrain(ter.heights[::-1, :].copy(), ter.cell, ter.x0, ter.y0)
    x0 = oracle.est_state_of(w.x0).astype(np.float64)
    x0m = x0.copy()
    x0m[1] = 2 * yc - x0[1]
    odd = [2, 3, 4, 5]
    x0m[odd] = -x0m[odd]
    assert float(np.float32(x0m[1])) == x0m[1]
    ctrl_m = w.ctrl.copy()
    ctrl_m[..., 0] = -ctrl_m[..., 0]
    c2 = dict(w.cost, goal_y=2 * yc - w.cost["goal_y"])
    r1 = oracle.est_rollout(w.vehicle, w.cost, t1, x0.astype(np.float32), w.ctrl, w.dt, w.n_sub)
    r2 = oracle.est_rollout(w.vehicle, c2, t2, x0m.astype(np.float32), ctrl_m, w.dt, w.n_sub)
    np.testing.assert_allclose(r2["J"], r1["J"], rtol=1e-9)
    np.testing.assert_allclose(r2["margin"], r1["margin"], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(r2["xf"][:, 1], 2 * yc - r1["xf"][:, 1], atol=1e-7)
    np.testing.assert_allclose(r2["xf"][:, odd], -r1["xf"][:, odd], atol=1e-7)
    np.testing.assert_allclose(r2["xf"][:, [0, 6]], r1["xf"][:, [0, 6]], atol=1e-7)


# Planar reduction: on level ground at low lateral acceleration the SRB
# model's planar motion is the EST model's: both reduce to the same linear
# bicycle with the same tire and axle loads.  What the planar model lacks is
# the roll of the chassis on its suspension, which moves the CoM sideways in
# proportion to the lateral acceleration, and the cos(delta) of the front
# force in the EST's lateral force sum.  So headings agree to third order in
# the steering, positions to first order with a small constant (under 0.1 %
# of the distance travelled here), each halving the steering shrinks them
# accordingly.
def test_planar_reduction_srb_vs_est():
    v = VEH
    t = plane(n=400, cell=0.5, x0=-100.0, y0=-100.0)
    tg = gen.Terrain(t.heights, 0.5, -100.0, -100.0, None, "flat")
    x13 = gen.settled_state(tg, v, -80.0, 0.0, 0.2, 8.0).astype(np.float64)

    def run(amp):
        ctrl = np.zeros((40, 2), np.float32)
        ctrl[:, 0] = (amp * np.sin(np.arange(40) / 6.0 + 1.0)).astype(np.float32)
        srb, _, _ = oracle.trajectory(v, no_goal(), t, x13, ctrl, 0.1, 20)
        est = oracle.est_trajectory(v, no_goal(), t, oracle.est_state_of(x13), ctrl, 0.1, 20)
        dpos = np.hypot(srb[:, 0] - est[:, 0], srb[:, 1] - est[:, 1]).max()
        dpsi = np.abs(srb[:, 3] - est[:, 2]).max()
        return dpos, dpsi, est

    d1, p1, est = run(0.05)
    d2, p2, _ = run(0.025)
    travel = 8.0 * 4.0
    assert d1 < 1e-3 * travel and p1 < 5e-4
    assert d2 == pytest.approx(d1 / 2, rel=0.1)        # first order: the roll offset
    assert p2 < p1 / 6                                 # third order in the steering
    # lateral acceleration stays low: |a_y| < 15 % of the rollover bound
    assert np.abs(est[:, 4] * est[:, 6]).max() < 0.15 * v["g"] * v["e"] / (2 * v["hR"])


def test_goal_truncation_and_feasibility_flags():
    w = gen.workload_plain(6, N=64, H=40)
    t = oracle.Terrain.of(w.terrain)
    x0 = oracle.est_state_of(w.x0).astype(np.float32)
    c = dict(w.cost, goal_x=12.0)
    r = oracle.est_rollout(w.vehicle, c, t, x0, w.ctrl, w.dt, w.n_sub, want_step_margin=True)
    done = (r["flags"] & oracle.DONE) != 0
    assert done.sum() > 10
    # feasible <=> min margin > 0 and finite; margin is the min over steps
    feas = (r["flags"] & oracle.FEASIBLE) != 0
    assert np.array_equal(feas, (r["margin"] > 0) & np.isfinite(r["J"]))
    np.testing.assert_array_equal(np.min(r["step_margin"], axis=0), r["margin"])
    # a candidate that starts inside the goal circle is frozen at once: J = w_g |p - goal|
    c2 = dict(w.cost, goal_x=float(x0[0]), goal_y=float(x0[1]))
    r2 = oracle.est_rollout(w.vehicle, c2, t, x0, w.ctrl[:, :4], w.dt, w.n_sub)
    assert np.all(r2["J"] == 0.0) and np.all(r2["flags"] & oracle.DONE)


# The longitudinal acceleration of the CoM in B includes the transport term
# a_Bx = v_x' - w_z v_y, which moves load between the axles in a turn.
def test_axle_load_transfer_uses_body_acceleration():
    v = VEH
    L = v["Lf"] + v["Lr"]
    vy, wz, acc = 0.7, 0.4, 1.5
    _, d = oracle.est_evaluate(v, no_goal(), plane(), est_state(vy=vy, wz=wz), [0.0, acc])
    a = acc - wz * vy
    assert d["aBx"] == pytest.approx(a, rel=1e-12)
    assert d["Fzf"] == pytest.approx(v["M"] * v["g"] * v["Lr"] / L - v["M"] * v["hR"] * a / L, rel=1e-12)


# On a side slope with no slip yet the tires carry no lateral force: the body
# accelerates downhill at g sin(beta), and the lateral-acceleration margin,
# which measures only what the tires transmit (a_By - g_By), is the full abar.
def test_side_slope_without_slip_slides_and_keeps_full_margin():
    v = VEH
    beta = math.atan(0.25)
    t = plane(0.0, 0.25)
    xd, d = oracle.est_evaluate(v, no_goal(), t, est_state(vx=6.0), [0.0, 0.0])
    assert d["Fyf"] == 0.0 and d["Fyr"] == 0.0
    assert xd[3] == pytest.approx(-v["g"] * math.sin(beta), rel=1e-12)
    assert d["margin"] == pytest.approx(v["g"] * v["e"] / (2 * v["hR"]), rel=1e-12)


# Planar velocity: on level ground v_W is v_B turned by the yaw, whatever the
# side slip.
def test_world_velocity_is_body_velocity_turned_by_yaw():
    psi, vx, vy = 0.9, 7.0, -1.3
    xd, _ = oracle.est_evaluate(VEH, no_goal(), plane(), est_state(psi=psi, vx=vx, vy=vy), [0.0, 0.0])
    Rz = Rotation.from_euler("z", psi).as_matrix()
    np.testing.assert_allclose(xd[:2], (Rz @ [vx, vy, 0.0])[:2], rtol=0, atol=1e-12)


# Yaw moment of the steered front tire: its force acts along the wheel's own
# lateral axis, turned by delta; the moment about the CoM is the cross
# product of the axle position with that force (numpy.cross, scipy rotation).
@pytest.mark.parametrize("delta", [0.3, -0.55])
def test_steered_front_force_yaw_moment(delta):
    v = VEH
    vx = 6.0
    _, d = oracle.est_evaluate(v, no_goal(), plane(), est_state(delta=delta, vx=vx), [0.0, 0.0])
    xd, _ = oracle.est_evaluate(v, no_goal(), plane(), est_state(delta=delta, vx=vx), [0.0, 0.0])
    f_wheel = Rotation.from_euler("z", delta).apply([0.0, d["Fyf"], 0.0])
    Mz = np.cross([v["Lf"], 0.0, 0.0], f_wheel)[2] + np.cross([-v["Lr"], 0.0, 0.0], [0.0, d["Fyr"], 0.0])[2]
    assert xd[4] == pytest.approx(Mz / v["Jzz"], rel=1e-12)


# Goal circle inclusive, steering rate and angle clamps, and the feasibility
# threshold, by hand on level ground.
def test_goal_inclusive_and_clamps_and_feasibility():
    v = VEH
    t = plane(n=400, cell=0.5, x0=-100.0, y0=-100.0)
    # goal exactly 1 m ahead, reached after 64 dyadic Euler steps of 1/64 m
    c = dict(gen.cost_default(1.0, 0.0), goal_r=0.0)
    ctrl = np.zeros((4, 1, 2), np.float32)
    r = oracle.est_rollout(v, c, t, est_state(vx=4.0).astype(np.float32), ctrl, 0.125, 32)
    assert r["flags"][0] & oracle.DONE and r["xf"][0][0] == pytest.approx(1.0, abs=1e-12)
    # a steering rate beyond the limit is clamped; the angle stops at delta_max
    ctrl = np.zeros((20, 1, 2), np.float32)
    ctrl[:, 0, 0] = 5.0
    st = oracle.est_trajectory(v, no_goal(), t, est_state(vx=1.0), ctrl[:, 0, :], 0.1, 20)
    assert st[20, 5] == pytest.approx(0.1 * v["delta_rate_max"], rel=1e-9)
    assert st[-1, 5] == pytest.approx(v["delta_max"], rel=1e-15)
    # feasibility: margin > 0 strictly
    vh = dict(v, mu=2.5)
    ctrl = np.zeros((40, 2, 2), np.float32)
    ctrl[:, 0, 0] = 0.25                    # stays inside the bound
    ctrl[:, 1, 0] = 0.3                     # just crosses it (margin between -1 and 0)
    r = oracle.est_rollout(vh, no_goal(), t, est_state(vx=8.0).astype(np.float32), ctrl, 0.05, 10)
    assert r["margin"][0] > 0 and r["flags"][0] & oracle.FEASIBLE
    assert -1.0 < r["margin"][1] < 0 and not r["flags"][1] & oracle.FEASIBLE
