"""Shared parity protocol of the GPU-vs-oracle tests.

Error measure: per field |g - o| / max(|o|, floor), floors 1 m (positions),
0.01 rad (angles), 0.1 m/s, 0.1 rad/s, 1 cost unit and 1 % of the level-ground
ESM; a candidate's error is the largest over cost, margin and final state.

Bar: TOL = 1e-4, the FP32-vs-FP64 tolerance, for every feasible candidate.
The rough-terrain rollout is not equally well conditioned everywhere, and on
a few candidates no FP32 arithmetic reaches 1e-4.  Which ones, and by how
much, is measured rather than assumed: the FP32 arithmetic reference of the
oracle package (every model quantity rounded to FP32, the state accumulated
exactly, C library elementary functions) is run on the same inputs and on
the inputs moved by one ulp, and the larger of its two errors against the
FP64 oracle is the candidate's FP32 conditioning `cond`.  A candidate then
agrees within max(TOL, KAPPA * cond).  The GPU
path and the reference are two independent FP32 computations, so besides
the per-candidate bound the GPU must be as accurate as the reference over the
whole workload: at 1e-4, 1e-3 and 1e-2 at least as large a fraction of the
candidates within the level as the reference on the same inputs (up to
STRICT_SLACK, or two standard errors of that fraction), and a median error
within LEVEL_FACTOR of the reference's (`assert_fp32_level`).

Exceptions, each counted and capped at max(3, 2 %) of the feasible
candidates:
  * a tail a little above the per-candidate bound (at most TAIL_FACTOR times
    it), since two FP32 runs sample the rounding only twice;
  * candidates that pass within FP32 reach of a discontinuity of the method,
    where FP32 and FP64 may take different branches: a wheel touching down
    while compressing, where the damper force jumps from 0 (reach: K_SWITCH
    times the candidate's conditioning, at least 1e-4 of the preload); U_ESM
    = 0, which decides feasibility; the goal circle;
  * candidates whose FP32 reference itself left the range of the bound
    (KAPPA * cond above CEIL, or a non-finite reference where the oracle is
    finite): they are held to CEIL, and one that misses it counts here; the
    cap of this class grows by the number of candidates on which the FP32
    reference itself misses CEIL.
Anything else above the bound fails.  Infeasible candidates (their roll
crossed the tipping point of the ESM, beyond which the fall diverges
exponentially) are compared on their feasibility bit only.

The planar (EST) model is held to the same protocol with its own state
floors and margin floor (1 % of abar); its feasibility switch is the
lateral-acceleration margin at 0, and it has no contact switch.
"""
import math

import numpy as np

TOL = 1e-4
KAPPA = 10.0            # x the FP32 conditioning
CEIL = 1e-2             # the largest per-candidate bound
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
TAIL_FACTOR = 4.0       # a capped tail may exceed the bound by this much
STRICT_SLACK = 0.005    # the GPU's fraction within TOL may trail the reference's by this
LEVEL_FACTOR = 2.0      # median error at most this times the reference's
LEVELS = (TOL, 10 * TOL, 100 * TOL)   # error levels at which the GPU must keep up with FP32


def level_esm(veh):
    Rb = math.hypot(veh["hR"], 0.5 * veh["e"])
    return veh["M"] * veh["g"] * (Rb - veh["hR"])


def lateral_bound(veh):
    """abar = g e / (2 (h + R)), the planar model's critical lateral acceleration."""
    return veh["g"] * veh["e"] / (2.0 * veh["hR"])


def margin_floor(veh, model="srb"):
    """1 % of the level-ground ESM (SRB) or of abar (EST)."""
    return 0.01 * (level_esm(veh) if model == "srb" else lateral_bound(veh))


def branch_sensitive(diag, cond=None):
    reach = TAU_CONTACT
    if cond is not None:
        reach = np.maximum(TAU_CONTACT, K_SWITCH * np.where(np.isfinite(cond), cond, 0.0))
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


def conditioning(oracle, veh, cost, ter, x0, ctrl, dt, n_sub, base, model="srb", seed=0):
    """Each candidate's FP32 conditioning, measured with the oracle package's
    FP32 arithmetic reference against the FP64 result `base`: `ref`, the
    reference's error on the same inputs, and `cond`, the larger of that and
    its error with every initial-state component and control moved by one
    ulp (a second sample of FP32 perturbation, the smallest the inputs
    admit).  Both are non-finite where the reference is non-finite and the
    oracle is not."""
    def err(x, u):
        r = oracle.rollout_f32(veh, cost, ter, x, u, dt, n_sub, model=model)
        return compare(dict(cost=r["J"], margin=r["margin"], xf=r["xf"]), base, veh, model)["err"]
    rng = np.random.default_rng(seed)
    ref = err(x0, ctrl)
    moved = err(nudge(x0, rng), nudge(ctrl, rng))
    return dict(ref=ref, cond=np.maximum(ref, moved))


def classify(gpu: dict, orc: dict, cond, veh: dict, model="srb"):
    """Per-candidate verdict (cond: what conditioning() returns).  Returns a
    dict of boolean masks and stats."""
    c = compare(gpu, orc, veh, model)
    err = c["err"]
    ref = np.asarray(cond["ref"], np.float64)
    cond = np.asarray(cond["cond"], np.float64)
    feas = (orc["flags"] & 1) > 0
    wild = ~np.isfinite(cond) | (KAPPA * np.where(np.isfinite(cond), cond, 0.0) > CEIL)
    bound = np.where(wild, CEIL, np.maximum(TOL, KAPPA * np.where(wild, 0.0, cond)))
    near = branch_sensitive(orc["diag"], cond)
    ok = err <= bound
    strict = err <= TOL
    excused = near | wild
    tail = feas & ~ok & (err <= TAIL_FACTOR * bound) & ~excused     # capped
    fail = feas & (err > TAIL_FACTOR * bound) & ~excused             # must be empty
    flipped = feas & ~ok & excused       # took the other side of a switch
    checked = feas & ~flipped
    cf = np.where(np.isfinite(ref), ref, np.inf)
    # candidates on which FP32 arithmetic itself (the reference, same inputs)
    # misses the largest bound: the GPU may miss it there too
    ref_miss = int((feas & (cf > CEIL)).sum())
    cap = max(3, int(0.02 * feas.sum()))
    stats = dict(n=len(err), feasible=int(feas.sum()), switch_misses=int(flipped.sum()),
                 wild=int((wild & feas).sum()), ref_misses=ref_miss, tail=int(tail.sum()),
                 fails=int(fail.sum()), cap=cap, switch_cap=cap + ref_miss,
                 strict_frac=float(strict[feas].mean()) if feas.any() else 1.0,
                 strict_frac_f32=float((cf[feas] <= TOL).mean()) if feas.any() else 1.0,
                 max_err=float(err[checked].max()) if checked.any() else 0.0,
                 worst_ratio=float((err / bound)[checked].max()) if checked.any() else 0.0,
                 median_err=float(np.median(err[feas])) if feas.any() else 0.0,
                 median_f32=float(np.median(cf[feas])) if feas.any() else 0.0,
                 p99_err=float(np.percentile(err[feas], 99)) if feas.any() else 0.0,
                 p99_f32=float(np.percentile(cf[feas], 99)) if feas.any() else 0.0,
                 within=[float((err[feas] <= t).mean()) if feas.any() else 1.0 for t in LEVELS],
                 within_f32=[float((cf[feas] <= t).mean()) if feas.any() else 1.0 for t in LEVELS])
    return dict(err=err, bound=bound, feas=feas, near=near, branch=near, wild=wild, checked=checked,
                ok=ok, strict=strict, fail=fail, tail=tail, flipped=flipped, stats=stats, cmp=c)


def assert_fp32_level(stats, slack=STRICT_SLACK, factor=LEVEL_FACTOR, floor=1e-7):
    """The GPU is as accurate as FP32 arithmetic: at each of the error levels
    LEVELS (TOL, 10 TOL, 100 TOL) as large a fraction of the feasible
    candidates within it as the FP32 reference on the same inputs (up to
    `slack`, or two standard errors of that fraction where that is larger),
    and a median error within `factor` of the reference's (or below
    `floor`)."""
    s = stats
    n = max(s["feasible"], 1)
    for got, p in zip(s["within"], s["within_f32"]):
        assert got >= p - max(slack, 2.0 * math.sqrt(p * (1.0 - p) / n)), s
    assert s["median_err"] <= max(factor * s["median_f32"], floor), s
