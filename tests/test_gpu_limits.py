"""Size limits of the C-ABI: a candidate count above what keeps every
kernel's 32-bit thread index in range is refused with ATP_ERR_UNSUPPORTED
before anything is launched or allocated, and the context stays usable.
Each refused call gets small, valid buffers; the count alone is too large,
and the check runs before any buffer is touched."""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu

MAX_N = 2 ** 31 - 1025
UNSUPPORTED = -2                        # ATP_ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def setup():
    from paper_2603_20525_gb300 import atp
    ctx = atp.Context(0)
    w = gen.workload_plain(0, N=256, H=10)
    t = w.terrain
    ter = ctx.terrain_prepare(torch.as_tensor(t.heights).cuda(), t.cell, t.x0, t.y0)
    vc, cc, xc = atp.vehicle(w.vehicle), atp.cost(w.cost), atp.state([float(v) for v in w.x0])
    ctrl = torch.as_tensor(w.ctrl).cuda()
    yield dict(atp=atp, ctx=ctx, w=w, ter=ter, vc=vc, cc=cc, xc=xc, ctrl=ctrl)
    ctx.close()


def still_plans(s):
    """A plan after a refused call gives its usual result."""
    w = s["w"]
    o = s["ctx"].plan(w.vehicle, w.cost, s["ter"], [float(v) for v in w.x0], s["ctrl"], w.dt, w.n_sub)
    torch.cuda.synchronize()
    r = s["atp"].decode_out(o["out"])
    assert 0 <= r["best_idx"] < w.N


def test_plan_above_the_limit(setup):
    s = setup
    atp, w = s["atp"], s["w"]
    out = torch.zeros(6, dtype=torch.int32, device="cuda")
    C = atp.C
    for N in (MAX_N + 1, 2 ** 31 - 1):
        with pytest.raises(atp.AtpError, match="UNSUPPORTED"):
            s["ctx"].plan_raw(C.pointer(s["vc"]), C.pointer(s["cc"]), C.pointer(s["ter"].c), C.pointer(s["xc"]),
                              s["ctrl"].data_ptr(), N, w.H, w.dt, w.n_sub, out.data_ptr(), None, None)
    still_plans(s)


def test_sampler_and_refinement_above_the_limit(setup):
    s = setup
    atp, ctx = s["atp"], s["ctx"]
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(atp.AtpError, match="UNSUPPORTED"):
        ctx.sample_raw(MAX_N + 1, 4, 0.2, 0.3, (1, 2), 0, None, 0, 0, buf.data_ptr(), None)
    rc = ctx.lib.atp_refine_init(ctx.h, atp.C.c_void_p(buf.data_ptr()), MAX_N + 1, 1, 1.0,
                                 atp.C.c_void_p(buf.data_ptr()), None)
    assert rc == UNSUPPORTED
    still_plans(s)


def test_adjoint_above_its_limit(setup):
    s = setup
    atp, ctx, w = s["atp"], s["ctx"], s["w"]
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    C = atp.C
    rc = ctx.lib.atp_grad(ctx.h, C.byref(s["vc"]), C.byref(s["cc"]), C.byref(s["ter"].c), C.byref(s["xc"]),
                          None, C.c_void_p(s["ctrl"].data_ptr()), 2 ** 28 + 1, w.H, float(w.dt), int(w.n_sub),
                          10, C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), None)
    assert rc == UNSUPPORTED
    assert "2^28" in ctx.lib.atp_last_error(ctx.h).decode()
    still_plans(s)
    J, G = ctx.grad(w.vehicle, w.cost, s["ter"], [float(v) for v in w.x0], s["ctrl"][:, :16].contiguous(),
                    w.dt, w.n_sub)
    torch.cuda.synchronize()
    assert np.isfinite(J.cpu().numpy()).any()
