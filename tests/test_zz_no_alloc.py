"""atp_plan_noalloc, the plan entry point for callers that cannot allocate
device memory once running (a planner in a hard real-time control loop whose
latency budget or certification forbids cudaMalloc after start-up, or a plugin
host that gives its plugins no allocator).  Called through the C-ABI, its
results must match atp_plan's on the same inputs, on two calls in a row,
since every call reuses the one static scratch array.  This file is collected
last so that a failure here comes after every other test has run."""
import ctypes as C

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4          # the relative tolerance the parity tests use


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _outputs(H, N):
    return dict(out=torch.zeros(6, dtype=torch.int32, device="cuda"),
                best_ctrl=torch.empty((H, 2), dtype=torch.float32, device="cuda"),
                best_margin=torch.empty(H, dtype=torch.float32, device="cuda"),
                cost=torch.empty(N, dtype=torch.float32, device="cuda"),
                margin=torch.empty(N, dtype=torch.float32, device="cuda"),
                flags=torch.empty(N, dtype=torch.uint8, device="cuda"))


def _noalloc(lib, w, ter, x0_dev, ctrl, o, with_candidates=True):
    from paper_2603_20525_gb300 import atp
    xs = None if x0_dev is not None else atp.state(w.x0)
    rc = lib.atp_plan_noalloc(C.byref(atp.vehicle(w.vehicle)), C.byref(atp.cost(w.cost)),
                              C.byref(ter.c), C.byref(xs) if xs is not None else None,
                              _ptr(x0_dev), _ptr(ctrl), w.N, w.H, float(w.dt), int(w.n_sub),
                              _ptr(o["out"]), _ptr(o["best_ctrl"]), _ptr(o["best_margin"]),
                              _ptr(o["cost"]) if with_candidates else None,
                              _ptr(o["margin"]) if with_candidates else None,
                              _ptr(o["flags"]) if with_candidates else None, None,
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def _same(a, b):
    from paper_2603_20525_gb300 import atp
    da, db = atp.decode_out(a["out"]), atp.decode_out(b["out"])
    assert da["best_idx"] == db["best_idx"] and da["n_feasible"] == db["n_feasible"]
    assert da["best_min_step"] == db["best_min_step"]
    for k in ("best_cost", "best_min_margin"):
        assert abs(da[k] - db[k]) <= TOL * max(abs(db[k]), 1.0), k
    for k in ("best_ctrl", "best_margin", "cost", "margin"):
        x, y = a[k].double(), b[k].double()
        close = (x == y) | ((x - y).abs() <= TOL * torch.clamp(y.abs(), min=1.0))   # inf == inf
        assert torch.all(close), k
    assert torch.equal(a["flags"], b["flags"])


@pytest.mark.parametrize("which", ["plain", "scaled"])
def test_noalloc_matches_plan_on_two_calls(which):
    from paper_2603_20525_gb300 import atp
    w = gen.workload_plain(0) if which == "plain" else gen.workload_scaled(0)
    ctx = atp.Context(0)
    lib = atp.load()
    heights = torch.as_tensor(w.terrain.heights).cuda()
    ter = ctx.terrain_prepare(heights, w.terrain.cell, w.terrain.x0, w.terrain.y0)
    ctrl = torch.as_tensor(w.ctrl).cuda()
    per = w.x0.ndim == 2
    x0_dev = torch.as_tensor(np.ascontiguousarray(w.x0.T)).cuda() if per else None
    ref = ctx.plan(w.vehicle, w.cost, ter, x0_dev if per else [float(v) for v in w.x0], ctrl,
                   w.dt, w.n_sub)
    first, second = _outputs(w.H, w.N), _outputs(w.H, w.N)
    assert _noalloc(lib, w, ter, x0_dev, ctrl, first) == atp.ATP_OK
    assert _noalloc(lib, w, ter, x0_dev, ctrl, second) == atp.ATP_OK
    torch.cuda.synchronize()
    _same(first, ref)
    _same(second, ref)
    # without caller candidate buffers the static array holds them as well
    third = _outputs(w.H, w.N)
    assert _noalloc(lib, w, ter, x0_dev, ctrl, third, with_candidates=False) == atp.ATP_OK
    torch.cuda.synchronize()
    d3, dr = atp.decode_out(third["out"]), atp.decode_out(ref["out"])
    assert d3["best_idx"] == dr["best_idx"] and d3["n_feasible"] == dr["n_feasible"]
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2603_20525_gb300 import atp
    w = gen.workload_plain(0, N=16384, H=126)    # 4 N H bytes alone exceed 8 MiB
    ctx = atp.Context(0)
    lib = atp.load()
    ter = ctx.terrain_prepare(torch.as_tensor(w.terrain.heights).cuda(), w.terrain.cell)
    ctrl = torch.as_tensor(w.ctrl).cuda()
    o = _outputs(w.H, w.N)
    assert _noalloc(lib, w, ter, None, ctrl, o) == -2          # ATP_ERR_UNSUPPORTED
    ctx.close()
