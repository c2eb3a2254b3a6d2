"""The values the paper prints (tests/golden/paper_values.txt, each line with
where it is printed) against what the tests and the benchmark feed the
oracle: the MRZR parameters of App. B, the real-time configuration of
Sec. IV-C/IV-D, and the energy stability margin of Sec. IV-B evaluated by
the oracle at the paper's own vehicle, checked against the closed forms the
paper defines (R-bar, phi-bar)."""
import math
import os

import numpy as np
import pytest

import gen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (x.strip() for x in line.split("=", 1))
                out[k] = float(v)
    return out


def test_mrzr_parameters_are_the_papers():
    g = golden()
    v = gen.vehicle_mrzr()
    for k in ("M", "Jxx", "Jyy", "Jzz", "Lf", "Lr", "e", "kf", "kr", "bf", "br", "delta_max",
              "delta_rate_max"):
        assert v[k] == g[k], k
    assert v["hR"] == g["h"] + g["R"]
    assert (v["C"], v["mu"]) == (g["C_sim"], g["mu_sim"])     # the simulated trials' tire


def test_real_time_configuration_is_the_papers():
    g = golden()
    assert g["N_resident_max"] == 7 * g["cores"]
    assert g["N"] == g["k"] * g["N_resident_max"]
    w = gen.workload_paper(0, N=64)                   # the configuration at a small N
    assert w.ctrl.shape[0] == g["n_t"]
    assert w.dt == g["dt"]
    assert w.dt / w.n_sub == g["h_euler"]
    assert w.vehicle == gen.vehicle_mrzr()
    import inspect
    assert inspect.signature(gen.workload_paper).parameters["N"].default == g["N"]


def test_esm_at_the_papers_vehicle():
    """U = M g R-bar (1 - sin(|phi| + phi-bar)) cos(theta) with
    R-bar = sqrt((h+R)^2 + (e/2)^2) and phi-bar = atan(2(h+R)/e) (Sec. IV-B):
    level ground, the tip-over roll angle pi/2 - phi-bar where U changes
    sign, and the cos(theta) scaling."""
    g = golden()
    v = gen.vehicle_mrzr()
    hR, e = g["h"] + g["R"], g["e"]
    rbar = math.sqrt(hR ** 2 + (e / 2) ** 2)
    phibar = math.atan(2 * hR / e)
    Mg = g["M"] * v["g"]
    u0 = oracle.esm(v, 0.0, 0.0)
    assert u0 == pytest.approx(Mg * (rbar - hR), rel=1e-12)
    tip = math.pi / 2 - phibar
    assert math.degrees(tip) == pytest.approx(43.65, abs=0.01)
    assert oracle.esm(v, tip - 1e-6, 0.0) > 0 > oracle.esm(v, tip + 1e-6, 0.0)
    assert oracle.esm(v, -(tip - 1e-6), 0.0) > 0 > oracle.esm(v, -(tip + 1e-6), 0.0)
    for th in (0.1, 0.3, -0.2):
        assert oracle.esm(v, 0.2, th) == pytest.approx(oracle.esm(v, 0.2, 0.0) * math.cos(th), rel=1e-12)
