"""atp_plan_noalloc, the plan entry point for callers that cannot allocate
device memory once running (a planner in a hard real-time control loop whose
latency budget or certification forbids cudaMalloc after start-up, or a plugin
host that gives its plugins no allocator).  Called through the C-ABI, its
results must be those of atp_plan on the same inputs (the same kernel, the
same default options, so the same bits), on two calls in a row, since every
call reuses the one static scratch array; and the calls after the first must
leave the device's free memory unchanged.  This file is collected last so
that a failure here comes after every other test has run."""
import ctypes as C

import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ATP_ERR_UNSUPPORTED = -2


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _outputs(H, N, best_margin=True):
    return dict(out=torch.zeros(6, dtype=torch.int32, device="cuda"),
                best_ctrl=torch.empty((H, 2), dtype=torch.float32, device="cuda"),
                best_margin=torch.empty(H, dtype=torch.float32, device="cuda") if best_margin else None,
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


def _same(a, b, keys=("out", "best_ctrl", "best_margin", "cost", "margin", "flags")):
    for k in keys:
        if a.get(k) is None and b.get(k) is None:
            continue
        assert torch.equal(a[k], b[k]), k


def _problem(which, N=None, H=None):
    from paper_2603_20525_gb300 import atp
    if which == "plain":
        w = gen.workload_plain(0)
    elif which == "scaled":
        w = gen.workload_scaled(0)
    else:
        w = gen.workload_scaled(1, N=N, H=H)
    ctx = atp.Context(0)
    heights = torch.as_tensor(w.terrain.heights).cuda()
    ter = ctx.terrain_prepare(heights, w.terrain.cell, w.terrain.x0, w.terrain.y0)
    ctrl = torch.as_tensor(w.ctrl).cuda()
    x0_dev = torch.as_tensor(np.ascontiguousarray(w.x0.T)).cuda() if w.x0.ndim == 2 else None
    return w, ctx, ter, ctrl, x0_dev


@pytest.mark.parametrize("which", ["plain", "scaled"])
def test_noalloc_matches_plan_on_two_calls(which):
    from paper_2603_20525_gb300 import atp
    w, ctx, ter, ctrl, x0_dev = _problem(which)
    lib = atp.load()
    ref = ctx.plan(w.vehicle, w.cost, ter, x0_dev if x0_dev is not None else [float(v) for v in w.x0],
                   ctrl, w.dt, w.n_sub)
    setup = _outputs(w.H, w.N)
    # the first call on a device looks up the static array's address
    assert _noalloc(lib, w, ter, x0_dev, ctrl, setup) == atp.ATP_OK
    torch.cuda.synchronize()
    first, second = _outputs(w.H, w.N), _outputs(w.H, w.N)
    free_before = torch.cuda.mem_get_info()[0]
    assert _noalloc(lib, w, ter, x0_dev, ctrl, first) == atp.ATP_OK
    assert _noalloc(lib, w, ter, x0_dev, ctrl, second) == atp.ATP_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before      # nothing allocated
    _same(setup, ref)
    _same(first, ref)
    _same(second, ref)
    # without caller candidate buffers the static array holds them as well
    third = _outputs(w.H, w.N)
    assert _noalloc(lib, w, ter, x0_dev, ctrl, third, with_candidates=False) == atp.ATP_OK
    torch.cuda.synchronize()
    _same(third, ref, keys=("out", "best_ctrl", "best_margin"))
    ctx.close()


def test_noalloc_without_per_step_margins_takes_larger_plans():
    """Without best_margin_dev no per-step margins are kept, so a plan of
    65536 candidates and 100 steps (26 MB of per-step margins) fits."""
    from paper_2603_20525_gb300 import atp
    w, ctx, ter, ctrl, x0_dev = _problem("big", N=65536, H=100)
    lib = atp.load()
    ref = ctx.plan(w.vehicle, w.cost, ter, x0_dev, ctrl, w.dt, w.n_sub, want_best_margin=False)
    o = _outputs(w.H, w.N, best_margin=False)
    assert _noalloc(lib, w, ter, x0_dev, ctrl, o) == atp.ATP_OK
    torch.cuda.synchronize()
    _same(o, ref)
    o2 = _outputs(w.H, w.N)                     # with per-step margins it does not fit
    assert _noalloc(lib, w, ter, x0_dev, ctrl, o2) == ATP_ERR_UNSUPPORTED
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2603_20525_gb300 import atp
    # the whole layout (256 + 13 N + 4 N H bytes, each of its five parts
    # rounded up to 256 B) is 8,470,784 bytes for N = 16384, H = 126: over 8 MiB
    w = gen.workload_plain(0, N=16384, H=126)
    ctx = atp.Context(0)
    lib = atp.load()
    ter = ctx.terrain_prepare(torch.as_tensor(w.terrain.heights).cuda(), w.terrain.cell)
    ctrl = torch.as_tensor(w.ctrl).cuda()
    o = _outputs(w.H, w.N)
    assert _noalloc(lib, w, ter, None, ctrl, o) == ATP_ERR_UNSUPPORTED
    ctx.close()
