"""Thin ctypes binding of libatp.so (include/atp.h).

Argument marshalling only: device memory comes from PyTorch tensors, whose
raw pointers and the current CUDA stream handle are passed to the C-ABI.
Every step of the planner runs in the library's CUDA kernels; if the library
cannot be loaded the binding raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

ATP_OK = 0
ERRORS = {-1: "ATP_ERR_INVALID", -2: "ATP_ERR_UNSUPPORTED", -3: "ATP_ERR_NOMEM",
          -4: "ATP_ERR_CUDA", -5: "ATP_ERR_TIMEOUT"}
F32X4, BF16X4 = 0, 1
OPT_COST_FP64 = 1
OPT_LANES = 2
OPT_STAGE_TERRAIN = 3
FEASIBLE, DONE, OFFMAP, NONFINITE = 1, 2, 4, 8
TERRAIN_HAS_COSTMAP = 1

# every symbol include/atp.h declares
EXPORTS = ("atp_version", "atp_create", "atp_destroy", "atp_last_error", "atp_reserve",
           "atp_terrain_bytes", "atp_terrain_prepare", "atp_plan", "atp_rollout",
           "atp_plan_noalloc", "atp_math_check", "atp_sample", "atp_plan_batch",
           "atp_set_option", "atp_grad", "atp_grad_margin", "atp_plan_est", "atp_lod_smooth",
           "atp_costmap", "atp_plan_lanes", "atp_refine_init", "atp_refine_trial",
           "atp_refine_accept")


class Vehicle(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("M", "Jxx", "Jyy", "Jzz", "Lf", "Lr", "e", "hR",
                                          "kf", "kr", "bf", "br", "C", "mu", "delta_max",
                                          "delta_rate_max", "g")]


class Cost(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("wt", "wc", "wg", "sigma", "eps_esm",
                                          "goal_x", "goal_y", "goal_r")]


class State(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("x", "y", "z", "psi", "theta", "phi", "vx", "vy",
                                         "vz", "wx", "wy", "wz", "delta")]


class TerrainC(C.Structure):
    _fields_ = [("texels", C.c_void_p), ("nx", C.c_int), ("ny", C.c_int),
                ("cell", C.c_double), ("x0", C.c_double), ("y0", C.c_double),
                ("format", C.c_int), ("flags", C.c_int)]


class EstState(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("x", "y", "psi", "vy", "wz", "delta", "vx")]


class PlanRequest(C.Structure):
    _fields_ = [("veh", C.POINTER(Vehicle)), ("cost", C.POINTER(Cost)),
                ("terrain", C.POINTER(TerrainC)), ("x0", C.POINTER(State)),
                ("x0_dev", C.c_void_p), ("ctrl_dev", C.c_void_p), ("N", C.c_int), ("H", C.c_int),
                ("dt", C.c_float), ("n_sub", C.c_int), ("out_dev", C.c_void_p),
                ("best_ctrl_dev", C.c_void_p), ("best_margin_dev", C.c_void_p),
                ("cand_cost_dev", C.c_void_p), ("cand_margin_dev", C.c_void_p),
                ("cand_flags_dev", C.c_void_p), ("cand_xf_dev", C.c_void_p)]


class PlanOut(C.Structure):
    _fields_ = [("best_idx", C.c_uint32), ("n_feasible", C.c_uint32),
                ("best_cost", C.c_float), ("best_min_margin", C.c_float),
                ("best_min_step", C.c_int32), ("reserved", C.c_uint32)]


_vp = C.c_void_p


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libatp.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libatp.so not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        L.atp_version.restype = C.c_int
        L.atp_create.argtypes = [C.POINTER(_vp), C.c_int]
        L.atp_destroy.argtypes = [_vp]
        L.atp_last_error.argtypes = [_vp]
        L.atp_last_error.restype = C.c_char_p
        L.atp_reserve.argtypes = [_vp, C.c_int, C.c_int]
        L.atp_terrain_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
        L.atp_terrain_bytes.restype = C.c_size_t
        L.atp_terrain_prepare.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.c_double, C.c_int, _vp, C.POINTER(TerrainC), _vp]
        L.atp_plan.argtypes = [_vp, C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(TerrainC),
                               C.POINTER(State), _vp, _vp, C.c_int, C.c_int, C.c_float, C.c_int,
                               _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.atp_rollout.argtypes = [_vp, C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(TerrainC),
                                  C.POINTER(State), _vp, _vp, C.c_int, C.c_int, C.c_float, C.c_int,
                                  _vp, _vp, _vp, _vp, _vp, _vp]
        L.atp_plan_noalloc.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(TerrainC),
                                       C.POINTER(State), _vp, _vp, C.c_int, C.c_int, C.c_float,
                                       C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.atp_math_check.argtypes = [_vp, _vp, C.c_int, _vp, _vp]
        L.atp_plan_batch.argtypes = [_vp, C.POINTER(PlanRequest), C.c_int, _vp]
        L.atp_set_option.argtypes = [_vp, C.c_int, C.c_int]
        L.atp_grad.argtypes = [_vp, C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(TerrainC),
                               C.POINTER(State), _vp, _vp, C.c_int, C.c_int, C.c_float, C.c_int,
                               C.c_int, _vp, _vp, _vp]
        L.atp_grad_margin.argtypes = L.atp_grad.argtypes
        L.atp_refine_init.argtypes = [_vp, _vp, C.c_int, C.c_int, C.c_float, _vp, _vp]
        L.atp_refine_trial.argtypes = [_vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _vp, _vp]
        L.atp_refine_accept.argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.atp_sample.argtypes = [_vp, _vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64,
                                 C.c_uint64, C.c_uint64, C.c_int, C.c_int, _vp, _vp]
        L.atp_plan_lanes.argtypes = [_vp, C.c_int]
        L.atp_plan_lanes.restype = C.c_int
        L.atp_plan_est.argtypes = [_vp, C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(TerrainC),
                                   C.POINTER(EstState), _vp, _vp, C.c_int, C.c_int, C.c_float, C.c_int,
                                   _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.atp_lod_smooth.argtypes = [_vp, _vp, C.c_int, C.c_int, C.c_double, C.c_double, _vp, _vp, _vp]
        L.atp_costmap.argtypes = [_vp, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int, C.c_int,
                                  C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                  _vp, _vp, _vp]
        for n in ("atp_create", "atp_destroy", "atp_reserve", "atp_terrain_prepare",
                  "atp_plan", "atp_rollout", "atp_plan_noalloc", "atp_math_check", "atp_sample",
                  "atp_plan_batch", "atp_set_option", "atp_grad", "atp_plan_est", "atp_lod_smooth",
                  "atp_costmap"):
            getattr(L, n).restype = C.c_int
        _lib = L
        return L


def vehicle(d: dict) -> Vehicle:
    return Vehicle(**{k: float(d[k]) for k, _ in Vehicle._fields_})


def cost(d: dict) -> Cost:
    return Cost(**{k: float(d[k]) for k, _ in Cost._fields_})


def state(x) -> State:
    return State(*[float(v) for v in x])


class AtpError(RuntimeError):
    pass


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Terrain:
    """A prepared terrain: the texel tensor (kept alive here) and its handle."""

    def __init__(self, texels, handle: TerrainC):
        self.texels = texels
        self.c = handle


class Context:
    """One atp_ctx on one device (not thread-safe; one per stream)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        rc = self.lib.atp_create(C.byref(self.h), int(device))
        if rc != ATP_OK:
            raise AtpError(f"atp_create failed: {ERRORS.get(rc, rc)}")
        self.device = device

    def close(self):
        if self.h:
            self.lib.atp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != ATP_OK:
            msg = self.lib.atp_last_error(self.h).decode()
            raise AtpError(f"{what}: {ERRORS.get(rc, rc)}: {msg}")

    def set_option(self, option: int, value: int):
        self._check(self.lib.atp_set_option(self.h, int(option), int(value)), "atp_set_option")

    def plan_lanes(self, N: int) -> int:
        """Threads per candidate a plan of N candidates runs with."""
        rc = self.lib.atp_plan_lanes(self.h, int(N))
        self._check(rc if rc < 0 else ATP_OK, "atp_plan_lanes")
        return rc

    def reserve(self, N: int, H: int):
        self._check(self.lib.atp_reserve(self.h, int(N), int(H)), "atp_reserve")

    def terrain_prepare(self, heights, cell, x0=0.0, y0=0.0, costmap=None, fmt=F32X4, stream=None):
        """heights: float32 CUDA tensor [ny, nx]; returns a Terrain."""
        import torch
        ny, nx = heights.shape
        nbytes = self.lib.atp_terrain_bytes(nx, ny, fmt)
        tex = torch.empty((nbytes + 3) // 4, dtype=torch.float32, device=heights.device)
        h = TerrainC()
        rc = self.lib.atp_terrain_prepare(self.h, _ptr(heights), _ptr(costmap), nx, ny,
                                          float(cell), float(x0), float(y0), int(fmt),
                                          _ptr(tex), C.byref(h), _stream(stream))
        self._check(rc, "atp_terrain_prepare")
        return Terrain(tex, h)

    def plan(self, veh: dict, cst: dict, terrain: Terrain, x0, ctrl, dt, n_sub=0, out=None,
             stream=None, want_candidates=True, want_xf=False, want_best_margin=True):
        """Plan over ctrl (float32 CUDA [H, N, 2]).  x0: 13 floats (host) or a
        float32 CUDA tensor [13, N] of per-candidate states.  Returns a dict of
        CUDA tensors; nothing is synchronized.  Without want_best_margin the
        best candidate's per-step margins are not produced (and no candidate's
        per-step margins are kept)."""
        import torch
        H, N, _ = ctrl.shape
        dev = ctrl.device
        o = out if out is not None else {}
        if "out" not in o:
            o["out"] = torch.zeros(6, dtype=torch.int32, device=dev)
            o["best_ctrl"] = torch.empty((H, 2), dtype=torch.float32, device=dev)
            if want_best_margin:
                o["best_margin"] = torch.empty(H, dtype=torch.float32, device=dev)
            if want_candidates:
                o["cost"] = torch.empty(N, dtype=torch.float32, device=dev)
                o["margin"] = torch.empty(N, dtype=torch.float32, device=dev)
                o["flags"] = torch.empty(N, dtype=torch.uint8, device=dev)
            if want_xf:
                o["xf"] = torch.empty((13, N), dtype=torch.float32, device=dev)
        xs, xdev = (None, x0) if isinstance(x0, torch.Tensor) else (state(x0), None)
        rc = self.lib.atp_plan(self.h, C.byref(vehicle(veh)), C.byref(cost(cst)),
                               C.byref(terrain.c), C.byref(xs) if xs is not None else None,
                               _ptr(xdev), _ptr(ctrl), int(N), int(H), float(dt), int(n_sub),
                               _ptr(o["out"]), _ptr(o.get("best_ctrl")), _ptr(o.get("best_margin")),
                               _ptr(o.get("cost")), _ptr(o.get("margin")), _ptr(o.get("flags")),
                               _ptr(o.get("xf")), _stream(stream))
        self._check(rc, "atp_plan")
        return o

    def plan_est(self, veh: dict, cst: dict, terrain: Terrain, x0, ctrl, dt, n_sub=0, out=None,
                 stream=None, want_candidates=True, want_xf=False):
        """Plan with the planar EST model (atp_plan_est).  x0: 7 floats (x, y,
        psi, v_By, w_Bz, delta, v_Bx) or a float32 CUDA tensor [7, N]."""
        import torch
        H, N, _ = ctrl.shape
        dev = ctrl.device
        o = out if out is not None else {}
        if "out" not in o:
            o.update(plan_outputs(N, H, device=dev, candidates=want_candidates))
            if want_xf:
                o["xf"] = torch.empty((7, N), dtype=torch.float32, device=dev)
        if isinstance(x0, torch.Tensor):
            xs, xdev = None, x0
        else:
            xs, xdev = EstState(*[float(v) for v in x0]), None
        rc = self.lib.atp_plan_est(self.h, C.byref(vehicle(veh)), C.byref(cost(cst)),
                                   C.byref(terrain.c), C.byref(xs) if xs is not None else None,
                                   _ptr(xdev), _ptr(ctrl), int(N), int(H), float(dt), int(n_sub),
                                   _ptr(o["out"]), _ptr(o.get("best_ctrl")), _ptr(o.get("best_margin")),
                                   _ptr(o.get("cost")), _ptr(o.get("margin")), _ptr(o.get("flags")),
                                   _ptr(o.get("xf")), _stream(stream))
        self._check(rc, "atp_plan_est")
        return o

    def lod_smooth(self, heights, cell, sigma, out=None, stream=None):
        """Gaussian level of detail of a float32 CUDA heightmap [ny, nx]."""
        import torch
        ny, nx = heights.shape
        tmp = torch.empty_like(heights)
        o = out if out is not None else torch.empty_like(heights)
        rc = self.lib.atp_lod_smooth(self.h, _ptr(heights), int(nx), int(ny), float(cell), float(sigma),
                                     _ptr(tmp), _ptr(o), _stream(stream))
        self._check(rc, "atp_lod_smooth")
        if stream is not None:          # the allocator frees tmp in the stream's order
            tmp.record_stream(stream)
        return o

    def costmap(self, polys, nx, ny, cell, x0=0.0, y0=0.0, eps=0.25, sigma=1e6, want_sdist=False,
                device="cuda", stream=None):
        """Distance-constraint costmap float32 CUDA [ny, nx] (and the smallest
        signed distance) of perimeters given as a list of (vertices [n, 2],
        kind) with kind 0 obstacle, 1 path boundary."""
        import numpy as np
        import torch
        xy = np.concatenate([np.asarray(p, np.float64).reshape(-1, 2) for p, _ in polys])
        start = (C.c_int * (len(polys) + 1))(0, *np.cumsum([len(np.asarray(p).reshape(-1, 2))
                                                            for p, _ in polys]).tolist())
        kind = (C.c_int * len(polys))(*[int(k) for _, k in polys])
        xy_d = torch.as_tensor(xy, device=device)
        cm = torch.empty((ny, nx), dtype=torch.float32, device=device)
        sd = torch.empty((ny, nx), dtype=torch.float32, device=device) if want_sdist else None
        rc = self.lib.atp_costmap(self.h, _ptr(xy_d), start, kind, len(polys), int(nx), int(ny),
                                  float(cell), float(x0), float(y0), float(eps), float(sigma),
                                  _ptr(cm), _ptr(sd), _stream(stream))
        self._check(rc, "atp_costmap")
        if stream is not None:
            xy_d.record_stream(stream)
        return (cm, sd) if want_sdist else cm

    def plan_batch(self, requests, stream=None):
        """One launch over a ragged batch of plans.  Each request is a dict
        with veh, cost, terrain (Terrain), x0 (13 floats or CUDA [13, N]),
        ctrl (CUDA [H, N, 2]), dt, n_sub and an `out` dict of output tensors
        as returned by plan_outputs()."""
        import torch
        n = len(requests)
        arr = (PlanRequest * n)()
        keep = []
        for i, q in enumerate(requests):
            H, N, _ = q["ctrl"].shape
            veh, cst = vehicle(q["veh"]), cost(q["cost"])
            x0 = q["x0"]
            xs, xdev = (None, x0) if isinstance(x0, torch.Tensor) else (state(x0), None)
            keep += [veh, cst, xs]
            o = q["out"]
            arr[i] = PlanRequest(C.pointer(veh), C.pointer(cst), C.pointer(q["terrain"].c),
                                 C.pointer(xs) if xs is not None else None,
                                 None if xdev is None else xdev.data_ptr(), q["ctrl"].data_ptr(),
                                 int(N), int(H), float(q["dt"]), int(q.get("n_sub", 0)),
                                 o["out"].data_ptr(),
                                 *[None if o.get(k) is None else o[k].data_ptr()
                                   for k in ("best_ctrl", "best_margin", "cost", "margin",
                                             "flags", "xf")])
        rc = self.lib.atp_plan_batch(self.h, arr, n, _stream(stream))
        self._check(rc, "atp_plan_batch")
        return [q["out"] for q in requests]

    # -- raw-pointer forms for a caller that keeps its own buffers and
    # -- marshalled structs (the serving loop); the same C calls as above
    def sample_raw(self, N, H, sigma_rate, sigma_acc, key, nonce, prev_ptr, prev_H, shift, out_ptr,
                   stream_ptr):
        """atp_sample with device pointers (ints) and a stream handle (int)."""
        rc = self.lib.atp_sample(self.h, prev_ptr or None, int(prev_H), int(shift), float(sigma_rate),
                                 float(sigma_acc), int(key[0]), int(key[1]), int(nonce), int(N), int(H),
                                 out_ptr, stream_ptr)
        self._check(rc, "atp_sample")

    def plan_raw(self, veh_p, cost_p, ter_p, x0_p, ctrl_ptr, N, H, dt, n_sub, out_ptr, best_ctrl_ptr,
                 stream_ptr):
        """atp_plan with marshalled structs (ctypes pointers), device pointers
        (ints) and a stream handle; no per-candidate outputs."""
        rc = self.lib.atp_plan(self.h, veh_p, cost_p, ter_p, x0_p, None, ctrl_ptr, int(N), int(H),
                               float(dt), int(n_sub), out_ptr, best_ctrl_ptr, None, None, None, None,
                               None, stream_ptr)
        self._check(rc, "atp_plan")

    def plan_batch_raw(self, arr, n, stream_ptr):
        """atp_plan_batch over a prepared PlanRequest array."""
        self._check(self.lib.atp_plan_batch(self.h, arr, int(n), stream_ptr), "atp_plan_batch")

    def grad(self, veh: dict, cst: dict, terrain: Terrain, x0, ctrl, dt, n_sub=0, ckpt=10,
             stream=None, objective="cost"):
        """J [K] and dJ/dctrl [H, K, 2] of K candidates (atp_grad), or with
        objective="margin" each candidate's ESM margin and its gradient
        (atp_grad_margin)."""
        import torch
        H, K, _ = ctrl.shape
        J = torch.empty(K, dtype=torch.float32, device=ctrl.device)
        G = torch.empty((H, K, 2), dtype=torch.float32, device=ctrl.device)
        xs, xdev = (None, x0) if isinstance(x0, torch.Tensor) else (state(x0), None)
        fn = {"cost": self.lib.atp_grad, "margin": self.lib.atp_grad_margin}[objective]
        rc = fn(self.h, C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(terrain.c),
                C.byref(xs) if xs is not None else None, _ptr(xdev), _ptr(ctrl),
                int(K), int(H), float(dt), int(n_sub), int(ckpt), _ptr(J), _ptr(G), _stream(stream))
        self._check(rc, "atp_grad" if objective == "cost" else "atp_grad_margin")
        return J, G

    def refine_init(self, grad, step, eta, stream=None):
        H, K, _ = grad.shape
        self._check(self.lib.atp_refine_init(self.h, _ptr(grad), int(K), int(H), float(step), _ptr(eta),
                                             _stream(stream)), "atp_refine_init")

    def refine_trial(self, ctrl, grad, eta, rate_max, trial, stream=None):
        H, K, _ = ctrl.shape
        self._check(self.lib.atp_refine_trial(self.h, _ptr(ctrl), _ptr(grad), _ptr(eta), int(K), int(H),
                                              float(rate_max), _ptr(trial), _stream(stream)), "atp_refine_trial")

    def refine_accept(self, trial, trial_cost, trial_grad, ctrl, cost, grad, eta, stream=None):
        H, K, _ = ctrl.shape
        self._check(self.lib.atp_refine_accept(self.h, int(K), int(H), _ptr(trial), _ptr(trial_cost),
                                               _ptr(trial_grad), _ptr(ctrl), _ptr(cost), _ptr(grad), _ptr(eta),
                                               _stream(stream)), "atp_refine_accept")

    def sample(self, N, H, sigma_rate, sigma_acc, key, nonce, prev=None, shift=1, out=None,
               stream=None):
        """Warm-started Gaussian candidates float32 CUDA [H, N, 2] (atp_sample)."""
        import torch
        ctrl = out if out is not None else torch.empty((H, N, 2), dtype=torch.float32, device="cuda")
        Hp = 0 if prev is None else int(prev.shape[0])
        rc = self.lib.atp_sample(self.h, _ptr(prev), Hp, int(shift), float(sigma_rate),
                                 float(sigma_acc), int(key[0]), int(key[1]), int(nonce), int(N),
                                 int(H), _ptr(ctrl), _stream(stream))
        self._check(rc, "atp_sample")
        return ctrl

    def rollout(self, veh: dict, cst: dict, terrain: Terrain, x0, ctrl, dt, n_sub=0,
                want_xf=True, want_step_margin=False, stream=None):
        import torch
        H, N, _ = ctrl.shape
        dev = ctrl.device
        o = dict(cost=torch.empty(N, dtype=torch.float32, device=dev),
                 margin=torch.empty(N, dtype=torch.float32, device=dev),
                 flags=torch.empty(N, dtype=torch.uint8, device=dev))
        if want_xf:
            o["xf"] = torch.empty((13, N), dtype=torch.float32, device=dev)
        if want_step_margin:
            o["step_margin"] = torch.empty((H, N), dtype=torch.float32, device=dev)
        xs, xdev = (None, x0) if isinstance(x0, torch.Tensor) else (state(x0), None)
        rc = self.lib.atp_rollout(self.h, C.byref(vehicle(veh)), C.byref(cost(cst)),
                                  C.byref(terrain.c), C.byref(xs) if xs is not None else None,
                                  _ptr(xdev), _ptr(ctrl), int(N), int(H), float(dt), int(n_sub),
                                  _ptr(o["cost"]), _ptr(o["margin"]), _ptr(o["flags"]),
                                  _ptr(o.get("xf")), _ptr(o.get("step_margin")), _stream(stream))
        self._check(rc, "atp_rollout")
        return o


def plan_outputs(N, H, device="cuda", candidates=True, xf=False):
    """Output tensors of one plan (for Context.plan(out=...) and plan_batch)."""
    import torch
    o = dict(out=torch.zeros(6, dtype=torch.int32, device=device),
             best_ctrl=torch.empty((H, 2), dtype=torch.float32, device=device),
             best_margin=torch.empty(H, dtype=torch.float32, device=device))
    if candidates:
        o["cost"] = torch.empty(N, dtype=torch.float32, device=device)
        o["margin"] = torch.empty(N, dtype=torch.float32, device=device)
        o["flags"] = torch.empty(N, dtype=torch.uint8, device=device)
    if xf:
        o["xf"] = torch.empty((13, N), dtype=torch.float32, device=device)
    return o


def decode_out(t) -> dict:
    """The 24-byte atp_plan_out tensor (int32 [6]) as a dict (host copy)."""
    import numpy as np
    a = t.detach().cpu().numpy().astype(np.int32)
    return dict(best_idx=int(np.uint32(a[0])), n_feasible=int(np.uint32(a[1])),
                best_cost=float(a[2:3].view(np.float32)[0]),
                best_min_margin=float(a[3:4].view(np.float32)[0]),
                best_min_step=int(a[4]))
