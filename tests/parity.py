"""Shared parity protocol of the GPU-vs-oracle tests.

Error measure: per field |g - o| / max(|o|, floor), floors 1 m (positions),
0.01 rad (angles), 0.1 m/s, 0.1 rad/s, 1 cost unit and 1 % of the level-ground
ESM; a candidate's error is the largest over cost, margin and final state.

Bar: TOL = 1e-4, the FP32-vs-FP64 tolerance.  The rough-terrain rollout is
not equally well conditioned everywhere: nudging the FP32 initial state by one
ulp (relative 6e-8) already moves the exact FP64 result by 1e-5 for a typical
candidate and by far more for some, which no FP32 arithmetic can undercut.  So
each candidate's conditioning is measured on the oracle itself (`sens`, the
largest change over N_NUDGES one-ulp nudges of its inputs) and the GPU must
agree to within max(TOL, KAPPA * sens).  The nudges move every component of
the initial state and every control by one ulp in a random direction, the way
FP32 rounding perturbs every quantity at once.

Every feasible candidate is held to that bound.  Because the conditioning is
a maximum over a few random nudges, a heavy tail of candidates may land a
little above it: up to 2 % of the feasible candidates (at least 3) may exceed
it by at most TAIL_FACTOR; anything beyond that fails.  The other exceptions,
counted and capped the same way, are misses by candidates that pass
within FP32 reach of a discontinuity of the method: a wheel touching down
while compressing, where the damper force jumps from 0 (reach: K_SWITCH times
the candidate's conditioning, at least 1e-4 of the preload); U_ESM = 0, which
decides feasibility; the goal circle.  Infeasible candidates (their roll
crossed the tipping point of the ESM, beyond which the fall diverges
exponentially) are compared on their feasibility bit only.

The planar (EST) model is held to the same protocol with its own state
floors and margin floor (1 % of abar); its feasibility switch is the
lateral-acceleration margin at 0, and it has no contact switch.
"""
import math

import numpy as np

TOL = 1e-4
KAPPA = 20.0
STATE_FLOORS = np.array([1.0, 1.0, 1.0, 0.01, 0.01, 0.01, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.01])
# the planar (EST) model's state: x, y, psi, v_By, w_Bz, delta, v_Bx
EST_FLOORS = np.array([1.0, 1.0, 0.01, 0.1, 0.1, 0.01, 0.1])
COST_FLOOR = 1.0
# distances to a switch (as normalised by the oracle's diag output) below which
# FP32 and FP64 may take different branches
TAU_CONTACT = 1e-4      # |F_s - k chi| / F_s, at least
K_SWITCH = 10.0         # x the candidate's conditioning
TAU_ESM = 1e-4          # |U| / U0
TAU_GOAL = 1e-4         # | |p - goal| - r_g |  [m]
N_NUDGES = 8
TAIL_FACTOR = 4.0       # a capped tail may exceed the bound by this much


def level_esm(veh):
    Rb = math.hypot(veh["hR"], 0.5 * veh["e"])
    return veh["M"] * veh["g"] * (Rb - veh["hR"])


def lateral_bound(veh):
    """abar = g e / (2 (h + R)), the planar model's critical lateral acceleration."""
    return veh["g"] * veh["e"] / (2.0 * veh["hR"])


def margin_floor(veh, model="srb"):
    """1 % of the level-ground ESM (SRB) or of abar (EST)."""
    return 0.01 * (level_esm(veh) if model == "srb" else lateral_bound(veh))


def branch_sensitive(diag, sens=None):
    reach = TAU_CONTACT if sens is None else np.maximum(TAU_CONTACT, K_SWITCH * np.nan_to_num(sens, nan=np.inf))
    return (diag[:, 0] < reach) | (diag[:, 1] < TAU_ESM) | (diag[:, 2] < TAU_GOAL)


def rel(g, o, floor):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    with np.errstate(invalid="ignore"):
        same_inf = np.isinf(g) & np.isinf(o) & (np.sign(g) == np.sign(o))
        e = np.abs(g - o) / np.maximum(np.abs(o), floor)
    e = np.where(same_inf, 0.0, e)
    return np.where(np.isnan(e), np.inf, e)


def compare(gpu: dict, orc: dict, veh: dict, model="srb"):
    """Per-candidate max relative error over cost, margin and final state."""
    eJ = rel(gpu["cost"], orc["J"], COST_FLOOR)
    eM = rel(gpu["margin"], orc["margin"], margin_floor(veh, model))
    err = np.maximum(eJ, eM)
    eX = None
    if gpu.get("xf") is not None and orc.get("xf") is not None:
        floors = STATE_FLOORS if model == "srb" else EST_FLOORS
        eX = rel(gpu["xf"], orc["xf"], floors[None, :])
        err = np.maximum(err, eX.max(axis=1))
    return dict(err=err, eJ=eJ, eM=eM, eX=eX)


def nudge(a, rng):
    """Every element of an FP32 array moved by one ulp, random direction."""
    a = np.asarray(a, dtype=np.float32)
    up = rng.integers(0, 2, size=a.shape).astype(bool)
    return np.nextafter(a, np.where(up, np.float32(np.inf), np.float32(-np.inf))).astype(np.float32)


def conditioning(oracle, veh, cost, ter, x0, ctrl, dt, n_sub, base, seed=0, model="srb"):
    """Largest per-candidate change of the FP64 result over N_NUDGES one-ulp
    nudges of the initial state(s) and the controls."""
    rng = np.random.default_rng(seed)
    sens = np.zeros(len(base["J"]))
    roll = oracle.rollout if model == "srb" else oracle.est_rollout
    for _ in range(N_NUDGES):
        r = roll(veh, cost, ter, nudge(x0, rng), nudge(ctrl, rng), dt, n_sub)
        c = compare(dict(cost=r["J"], margin=r["margin"], xf=r["xf"]), base, veh, model)
        sens = np.maximum(sens, c["err"])
    return sens


def classify(gpu: dict, orc: dict, sens, veh: dict, model="srb"):
    """Per-candidate verdict.  Returns a dict of boolean masks and stats."""
    c = compare(gpu, orc, veh, model)
    err = c["err"]
    feas = (orc["flags"] & 1) > 0
    near = branch_sensitive(orc["diag"], sens)
    bound = np.maximum(TOL, KAPPA * np.nan_to_num(sens, nan=np.inf))
    ok = err <= bound
    strict = err <= TOL
    tail = feas & ~ok & (err <= TAIL_FACTOR * bound) & ~near      # capped
    fail = feas & (err > TAIL_FACTOR * bound) & ~near              # must be empty
    flipped = feas & ~ok & near        # took the other side of a switch
    checked = feas & ~flipped
    cap = max(3, int(0.02 * feas.sum()))
    stats = dict(n=len(err), feasible=int(feas.sum()), switch_misses=int(flipped.sum()),
                 tail=int(tail.sum()), fails=int(fail.sum()), cap=cap,
                 strict_frac=float(strict[feas].mean()) if feas.any() else 1.0,
                 max_err=float(err[checked].max()) if checked.any() else 0.0,
                 worst_ratio=float(np.nan_to_num(err / bound)[checked].max()) if checked.any() else 0.0,
                 median_err=float(np.median(err[feas])) if feas.any() else 0.0,
                 median_sens=float(np.median(sens[feas])) if feas.any() else 0.0)
    return dict(err=err, bound=bound, feas=feas, near=near, branch=near, checked=checked, ok=ok,
                strict=strict, fail=fail, tail=tail, flipped=flipped, stats=stats, cmp=c)
