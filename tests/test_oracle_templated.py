"""The templated restatement of the model (oracle/model.hpp) and its two
test-side instantiations: in FP64 it must be the oracle itself, bit for bit;
in FP32 arithmetic it is the reference the parity protocol measures each
candidate's FP32 conditioning with; with the counting scalar it gives the
algorithmic work per Euler step.  These run on the CPU only."""
import math

import numpy as np
import pytest

import gen
import oracle

FIELDS = ("J", "margin", "flags", "xf")


def same_bits(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return bool(np.all((a == b) | (np.isnan(a) & np.isnan(b))))


def variants():
    w = gen.workload_plain(0)
    yield "plain", w
    # goal reached mid-horizon (reading Q4)
    yield "goal", gen.Workload(w.name, w.terrain, w.vehicle, dict(w.cost, goal_x=12.0), w.x0, w.ctrl, w.dt,
                               w.n_sub)
    # leaving the map near its corner (reading Q10)
    x0 = gen.settled_state(w.terrain, w.vehicle, 2.0, 2.0, math.pi * 1.25, 8.0)
    yield "offmap", gen.Workload(w.name, w.terrain, w.vehicle, w.cost, x0, w.ctrl, w.dt, w.n_sub)
    s = gen.workload_scaled(0, N=2048, H=60)
    yield "scaled", s
    # the goal circle around the start: every candidate is frozen at its first
    # state, so every control step ties for the smallest margin (the first wins)
    yield "frozen", gen.Workload(w.name, w.terrain, w.vehicle, dict(w.cost, goal_x=5.0, goal_y=25.6),
                                 w.x0, w.ctrl, w.dt, w.n_sub)


@pytest.mark.parametrize("name,w", list(variants()))
def test_templated_model_in_fp64_is_the_oracle(name, w):
    t = oracle.Terrain.of(w.terrain)
    r = oracle.rollout(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub, want_step_margin=True)
    q = oracle.rollout_templated(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    for k in FIELDS:
        assert same_bits(r[k], q[k]), (name, k)
    # the control step of the smallest per-step margin (first on ties)
    assert np.array_equal(q["min_step"], np.argmin(r["step_margin"], axis=0))
    if name == "frozen":
        assert np.all(r["step_margin"] == r["step_margin"][0]) and np.all(q["min_step"] == 0)


def test_templated_planar_model_matches_the_planar_oracle():
    w = gen.workload_est(0, N=256)
    t = oracle.Terrain.of(w.terrain)
    r = oracle.est_rollout(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub, want_step_margin=True)
    q = oracle.rollout_templated(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub, model="est")
    assert np.array_equal(r["flags"], q["flags"])
    np.testing.assert_allclose(q["J"], r["J"], rtol=1e-12)
    np.testing.assert_allclose(q["margin"], r["margin"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(q["xf"], r["xf"], rtol=1e-12, atol=1e-12)
    assert np.array_equal(q["min_step"], np.argmin(r["step_margin"], axis=0))


def test_fp32_reference_rounds_like_fp32_and_stays_near_the_oracle():
    """Its results differ from the FP64 oracle by FP32 rounding: not zero,
    and within 1e-4 relative for nearly every candidate of the plain plan."""
    from tests import parity
    w = gen.workload_plain(0)
    t = oracle.Terrain.of(w.terrain)
    r = oracle.rollout(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    f = oracle.rollout_f32(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    e = parity.compare(dict(cost=f["J"], margin=f["margin"], xf=f["xf"]), r, w.vehicle)["err"]
    assert np.array_equal(f["flags"], r["flags"])
    assert np.median(e) > 1e-7              # FP32 rounding is there
    assert np.mean(e <= 1e-4) >= 0.99        # and small
    # every result is an FP32 value except the exactly accumulated components
    assert np.array_equal(f["J"], f["J"].astype(np.float32).astype(np.float64))
    wide = [0, 1, 2, 3, 6, 7, 8]
    narrow = [q for q in range(13) if q not in wide]
    assert np.array_equal(f["xf"][:, narrow], f["xf"][:, narrow].astype(np.float32).astype(np.float64))


def test_fp32_reference_accumulates_position_exactly():
    """Straight driving on level ground for 2 s (800 Euler steps of 2.5 ms):
    x = x0 + v t.  The FP32 reference accumulates the position exactly, so
    only the FP32 rounding of each increment remains (~1e-6 m in total); a
    plain FP32 running sum near x = 30 m (ulp 1.9e-6 m) would lose ~1e-4 m."""
    v = gen.vehicle_baseline()
    t = oracle.Terrain(np.zeros((256, 256), np.float32), 0.5, -10.0, -64.0)
    xi = np.zeros(13, np.float32)
    xi[0] = 14.0
    xi[2] = v["hR"]
    xi[6] = 8.0
    c = gen.cost_default(1000.0, 0.0)
    ctrl = np.zeros((80, 1, 2), np.float32)
    f = oracle.rollout_f32(v, c, t, xi, ctrl, 0.025, 10)
    assert abs(f["xf"][0, 0] - (14.0 + 16.0)) < 4e-6
    np.testing.assert_allclose(f["xf"][0, 6], 8.0, atol=0)


def test_fp32_reference_of_the_planar_model():
    from tests import parity
    w = gen.workload_est(1)
    t = oracle.Terrain.of(w.terrain)
    r = oracle.est_rollout(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub)
    f = oracle.rollout_f32(w.vehicle, w.cost, t, w.x0, w.ctrl, w.dt, w.n_sub, model="est")
    e = parity.compare(dict(cost=f["J"], margin=f["margin"], xf=f["xf"]), r, w.vehicle, model="est")["err"]
    assert np.array_equal(f["flags"], r["flags"])
    assert 1e-8 < np.median(e) < 1e-5
    assert np.mean(e <= 1e-4) >= 0.99
