"""Precision report over 64 seeds of the plain plan (1024 candidates, H = 40,
dt = 0.05 s): GPU variants against the FP64 oracle.

  f32        FP32 terrain, FP32 arithmetic and cost accumulation
  f32+acc64  the same with the running cost accumulated in FP64
  bf16       BF16 terrain against the oracle on the original FP32 terrain
             (arithmetic plus quantisation error)
  bf16/dec   BF16 terrain against the oracle on the same BF16-decoded terrain
             (arithmetic error only)

Per variant: per-field maximum and median relative error over the feasible
candidates of all seeds (floors as in tests/parity.py), the fraction of
candidates whose feasibility flag agrees, and the number of seeds whose chosen
candidate agrees.  Usage (GPU): python tests/precision_report.py [seeds]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
import oracle  # noqa: E402
from tests import parity  # noqa: E402

FIELDS = ("x", "y", "z", "psi", "theta", "phi", "vx", "vy", "vz", "wx", "wy", "wz", "delta")


def main(n_seeds=64):
    import torch
    from paper_2603_20525_gb300 import atp
    ctx = atp.Context(0)
    acc = {k: dict(err=[], feas_agree=0, feas_n=0, argmin=0, seeds=0)
           for k in ("f32", "f32+acc64", "bf16", "bf16/dec")}
    for seed in range(n_seeds):
        w = gen.workload_plain(seed)
        t = w.terrain
        o32 = oracle.plan(w.vehicle, w.cost, oracle.Terrain.of(t), w.x0, w.ctrl, w.dt, w.n_sub)
        h_dec, gx, gy, _, _ = oracle.bf16_terrain(t.heights, t.cell)
        odec = oracle.plan(w.vehicle, w.cost, oracle.Terrain(h_dec, t.cell, t.x0, t.y0, gx=gx, gy=gy),
                           w.x0, w.ctrl, w.dt, w.n_sub)
        hd = torch.as_tensor(t.heights).cuda()
        ctrl = torch.as_tensor(w.ctrl).cuda()
        x0 = [float(v) for v in w.x0]
        runs = {}
        for fmt, opt in ((atp.F32X4, 0), (atp.F32X4, 1), (atp.BF16X4, 0)):
            ter = ctx.terrain_prepare(hd, t.cell, t.x0, t.y0, fmt=fmt)
            ctx.set_option(atp.OPT_COST_FP64, opt)
            o = ctx.plan(w.vehicle, w.cost, ter, x0, ctrl, w.dt, w.n_sub, want_xf=True)
            torch.cuda.synchronize()
            g = {k: v.cpu().numpy() for k, v in o.items() if k != "out"}
            g.update(atp.decode_out(o["out"]))
            g["xf"] = g["xf"].T.copy()
            runs[(fmt, opt)] = g
        ctx.set_option(atp.OPT_COST_FP64, 0)
        for name, g, ref in (("f32", runs[(atp.F32X4, 0)], o32), ("f32+acc64", runs[(atp.F32X4, 1)], o32),
                             ("bf16", runs[(atp.BF16X4, 0)], o32), ("bf16/dec", runs[(atp.BF16X4, 0)], odec)):
            c = parity.compare(g, ref, w.vehicle)
            feas = (ref["flags"] & 1) > 0
            a = acc[name]
            a["err"].append(np.concatenate([c["eX"], c["eJ"][:, None], c["eM"][:, None]], 1)[feas])
            a["feas_agree"] += int(np.sum((g["flags"] & 1) == (ref["flags"] & 1)))
            a["feas_n"] += len(feas)
            a["argmin"] += int(g["best_idx"] == ref["best"])
            a["seeds"] += 1
    out = {}
    for name, a in acc.items():
        e = np.concatenate(a["err"], 0)
        names = FIELDS + ("J", "margin")
        out[name] = dict(max_rel={n: float(v) for n, v in zip(names, e.max(0))},
                         median_rel={n: float(v) for n, v in zip(names, np.median(e, 0))},
                         feasibility_agreement=a["feas_agree"] / a["feas_n"],
                         argmin_agreement=f"{a['argmin']}/{a['seeds']}")
    print(json.dumps(out, indent=1))
    ctx.close()


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 64)
