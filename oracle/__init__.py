"""FP64 CPU oracle of the SRB rollout planner (arxiv 2603.20525, Sec. IV).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is an
independent restatement of the paper in plain C (``srb.c``), built with gcc
into ``oracle/_build/liboracle.so`` and called through ctypes; ``sampler.c``
restates the candidate sampler (Philox4x64-10 and Box-Muller).  It shares no
code with the CUDA path, and the product never falls back to it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, n) for n in ("srb.c", "sampler.c", "est.c", "terrain_tools.c")]
_SRC_CXX = [os.path.join(_HERE, n) for n in ("adjoint.cpp", "emul32.cpp")]
_HDR = [os.path.join(_HERE, n) for n in ("oracle.h", "model.hpp")]
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

FEASIBLE, DONE, OFFMAP, NONFINITE = 1, 2, 4, 8
WHEEL_FIELDS = ("Px", "Py", "Pz", "vix", "viy", "viz", "f", "fx", "fy", "cmap",
                "taux", "tauy", "tauz", "chi", "chidot", "Fk", "Fb", "Fz", "alpha",
                "Fy", "Fx", "offmap")
BODY_FIELDS = tuple(f"R{i}" for i in range(9)) + ("gBx", "gBy", "gBz", "Fy", "Fz",
                                                 "Mx", "My", "Mz", "U", "L",
                                                 "Fs_fl", "Fs_fr", "Fs_rl", "Fs_rr")


def build(force: bool = False) -> str:
    """Compile liboracle.so (FP64, no FMA contraction, OpenMP): the C model
    and sampler with gcc, the C++ adjoint with g++."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + _SRC_CXX + _HDR)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= newest:
        return _OUT
    tag = f".{os.getpid()}"
    objs = []
    common = ["-O2", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
              "-fopenmp", "-Wall", "-Wno-unknown-pragmas", "-c"]
    for src in _SRC:
        o = os.path.join(os.path.dirname(_OUT), os.path.basename(src) + tag + ".o")
        subprocess.run(["gcc", "-std=c11", *common, src, "-o", o], check=True, capture_output=True, text=True)
        objs.append(o)
    for src in _SRC_CXX:
        o = os.path.join(os.path.dirname(_OUT), os.path.basename(src) + tag + ".o")
        subprocess.run(["g++", "-std=c++17", *common, src, "-o", o], check=True, capture_output=True,
                       text=True)
        objs.append(o)
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-shared", "-fopenmp", *objs, "-o", tmp, "-lm"], check=True,
                   capture_output=True, text=True)
    os.replace(tmp, _OUT)
    for o in objs:
        os.remove(o)
    return _OUT


class Vehicle(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("M", "Jxx", "Jyy", "Jzz", "Lf", "Lr", "e", "hR",
                                          "kf", "kr", "bf", "br", "C", "mu", "delta_max",
                                          "delta_rate_max", "g")]


class Cost(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("wt", "wc", "wg", "sigma", "eps_esm",
                                          "goal_x", "goal_y", "goal_r")]


class _Terrain(C.Structure):
    _fields_ = [("heights", C.POINTER(C.c_float)), ("gx", C.POINTER(C.c_double)),
                ("gy", C.POINTER(C.c_double)), ("costmap", C.POINTER(C.c_float)),
                ("nx", C.c_int), ("ny", C.c_int), ("cell", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double)]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_up = C.POINTER(C.c_ubyte)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_terrain_gradients.argtypes = [_fp, C.c_int, C.c_int, C.c_double, _dp, _dp]
            L.orc_terrain_sample.argtypes = [C.POINTER(_Terrain), C.c_double, C.c_double, _dp]
            L.orc_terrain_sample.restype = C.c_int
            L.orc_tire.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_tire.restype = C.c_double
            L.orc_esm.argtypes = [C.POINTER(Vehicle), C.c_double, C.c_double]
            L.orc_esm.restype = C.c_double
            L.orc_rotation.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
            L.orc_eval.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                   _dp, _dp, _dp, _dp, _dp]
            L.orc_rollout.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                      _fp, C.c_int, _fp, C.c_int, C.c_int, C.c_double, C.c_int,
                                      _dp, _dp, _up, _dp, _dp, _dp, C.c_int]
            L.orc_rollout.restype = C.c_int
            L.orc_trajectory.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                         _dp, _fp, C.c_int, C.c_double, C.c_int, _dp, _dp]
            L.orc_trajectory.restype = C.c_int
            L.orc_select.argtypes = [_dp, _up, C.c_int]
            L.orc_select.restype = C.c_int
            _u64p = C.POINTER(C.c_uint64)
            L.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
            L.orc_sample.argtypes = [_fp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_uint64,
                                     C.c_uint64, C.c_uint64, C.c_int, C.c_int, _dp]
            L.orc_cost_templated.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                             _dp, _fp, C.c_int, C.c_double, C.c_int]
            L.orc_cost_templated.restype = C.c_double
            L.orc_cost_f64.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                       _dp, _dp, C.c_int, C.c_double, C.c_int]
            L.orc_cost_f64.restype = C.c_double
            L.orc_grad_batch.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                         _fp, C.c_int, _fp, C.c_int, C.c_int, C.c_double, C.c_int,
                                         _dp, _dp]
            L.orc_grad_batch.restype = C.c_int
            L.orc_grad_margin_batch.argtypes = L.orc_grad_batch.argtypes
            L.orc_grad_margin_batch.restype = C.c_int
            L.orc_margin_f64.argtypes = L.orc_cost_f64.argtypes
            L.orc_margin_f64.restype = C.c_double
            L.orc_est_rotation.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
            L.orc_est_eval.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                       _dp, _dp, _dp, _dp]
            L.orc_est_rollout.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                          _fp, C.c_int, _fp, C.c_int, C.c_int, C.c_double, C.c_int,
                                          _dp, _dp, _up, _dp, _dp, _dp, C.c_int]
            L.orc_est_rollout.restype = C.c_int
            L.orc_est_trajectory.argtypes = [C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                             _dp, _fp, C.c_int, C.c_double, C.c_int, _dp]
            L.orc_est_trajectory.restype = C.c_int
            L.orc_lod_weights.argtypes = [C.c_double, C.c_double, C.c_int, _dp]
            L.orc_lod_weights.restype = C.c_int
            L.orc_lod_smooth.argtypes = [_fp, C.c_int, C.c_int, C.c_double, C.c_double, _dp]
            L.orc_lod_smooth.restype = C.c_int
            _ip = C.POINTER(C.c_int)
            _roll = [C.c_int, C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain), _fp, C.c_int,
                     _fp, C.c_int, C.c_int, C.c_double, C.c_int, _dp, _dp, _up, _dp, _ip]
            L.orc_rollout_f32.argtypes = _roll
            L.orc_rollout_f32.restype = C.c_int
            L.orc_rollout_templated.argtypes = _roll
            L.orc_rollout_templated.restype = C.c_int
            L.orc_count_ops.argtypes = [C.c_int, C.POINTER(Vehicle), C.POINTER(Cost), C.POINTER(_Terrain),
                                        _fp, C.c_int, _fp, C.c_int, C.c_int, C.c_double, C.c_int,
                                        C.POINTER(C.c_long)]
            L.orc_count_ops.restype = C.c_int
            L.orc_sdist.argtypes = [_dp, C.c_int, C.c_int, C.c_double, C.c_double]
            L.orc_sdist.restype = C.c_double
            L.orc_costmap.argtypes = [_dp, _ip, _ip, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, _dp, _dp]
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def vehicle(d: dict) -> Vehicle:
    return Vehicle(**{k: float(d[k]) for k, _ in Vehicle._fields_})


def cost(d: dict) -> Cost:
    return Cost(**{k: float(d[k]) for k, _ in Cost._fields_})


class Terrain:
    """Oracle view of a heightmap: FP32 heights (the same bytes the GPU gets),
    FP64 node gradients computed here, optional FP32 costmap."""

    def __init__(self, heights, cell, x0=0.0, y0=0.0, costmap=None, gx=None, gy=None):
        self.heights = np.ascontiguousarray(heights, dtype=np.float32)
        ny, nx = self.heights.shape
        if gx is None:
            self.gx = np.empty((ny, nx), dtype=np.float64)
            self.gy = np.empty((ny, nx), dtype=np.float64)
            lib().orc_terrain_gradients(_ptr(self.heights, _fp), nx, ny, float(cell),
                                        _ptr(self.gx, _dp), _ptr(self.gy, _dp))
        else:                       # given node slopes (a stored terrain format)
            self.gx = np.ascontiguousarray(gx, dtype=np.float64)
            self.gy = np.ascontiguousarray(gy, dtype=np.float64)
        self.costmap = None if costmap is None else np.ascontiguousarray(costmap, np.float32)
        self.c = _Terrain(_ptr(self.heights, _fp), _ptr(self.gx, _dp), _ptr(self.gy, _dp),
                          _ptr(self.costmap, _fp), nx, ny, float(cell), float(x0), float(y0))

    @classmethod
    def of(cls, t):
        """From a gen.Terrain-like object (heights, cell, x0, y0, costmap)."""
        return cls(t.heights, t.cell, t.x0, t.y0, getattr(t, "costmap", None))

    def sample(self, x, y):
        out = np.empty(4)
        off = lib().orc_terrain_sample(C.byref(self.c), float(x), float(y), _ptr(out, _dp))
        return out, bool(off)


def tire(Cc, mu, alpha):
    return lib().orc_tire(float(Cc), float(mu), float(alpha))


def esm(veh: dict, phi, theta):
    return lib().orc_esm(C.byref(vehicle(veh)), float(phi), float(theta))


def rotation(psi, theta, phi):
    R = np.empty(9)
    lib().orc_rotation(float(psi), float(theta), float(phi), _ptr(R, _dp))
    return R.reshape(3, 3)


def evaluate(veh: dict, cst: dict, ter: Terrain, xi, zeta):
    """xi_dot, per-wheel diagnostics [4, 22] and body diagnostics [23]."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    xd = np.empty(13)
    wheel = np.empty((4, len(WHEEL_FIELDS)))
    body = np.empty(len(BODY_FIELDS))
    lib().orc_eval(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                   _ptr(xi, _dp), _ptr(zeta, _dp), _ptr(xd, _dp), _ptr(wheel, _dp),
                   _ptr(body, _dp))
    return xd, wheel, body


def rollout(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int,
            want_xf=True, want_step_margin=False, want_diag=True, nthreads=0):
    """Roll out every candidate.  x0 float32 [13] or [N, 13]; ctrl float32 [H, N, 2]."""
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
    H, N, _ = ctrl.shape
    per = 1 if x0.ndim == 2 else 0
    if per:
        assert x0.shape == (N, 13)
    J = np.empty(N)
    margin = np.empty(N)
    flags = np.empty(N, dtype=np.uint8)
    xf = np.empty((N, 13)) if want_xf else None
    sm = np.empty((H, N)) if want_step_margin else None
    diag = np.empty((N, 3)) if want_diag else None
    rc = lib().orc_rollout(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                           _ptr(x0, _fp), per, _ptr(ctrl, _fp), N, H, float(dt), int(n_sub),
                           _ptr(J, _dp), _ptr(margin, _dp), _ptr(flags, _up),
                           _ptr(xf, _dp), _ptr(sm, _dp), _ptr(diag, _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rollout rejected its arguments")
    return dict(J=J, margin=margin, flags=flags, xf=xf, step_margin=sm, diag=diag)


def select(J, flags) -> int:
    J = np.ascontiguousarray(J, dtype=np.float64)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    return int(lib().orc_select(_ptr(J, _dp), _ptr(flags, _up), len(J)))


def plan(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int, nthreads=0):
    """Rollout, empirical argmin and the best candidate's outputs."""
    r = rollout(veh, cst, ter, x0, ctrl, dt, n_sub, want_step_margin=True, nthreads=nthreads)
    b = select(r["J"], r["flags"])
    ctrl = np.asarray(ctrl, dtype=np.float32)
    best_ctrl = ctrl[:, b, :].astype(np.float64)
    best_ctrl[:, 0] = np.clip(best_ctrl[:, 0], -veh["delta_rate_max"], veh["delta_rate_max"])
    r.update(best=b, n_feasible=int(np.count_nonzero(r["flags"] & FEASIBLE)),
             best_cost=float(r["J"][b]), best_margin=float(r["margin"][b]),
             best_ctrl=best_ctrl, best_step_margin=r["step_margin"][:, b].copy())
    return r


def trajectory(veh: dict, cst: dict, ter: Terrain, x0, ctrl_h2, dt: float, n_sub: int):
    """One candidate with every Euler state: states [S+1, 13], running cost
    [S+1], Euler-step index of goal arrival (or -1)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    ctrl_h2 = np.ascontiguousarray(ctrl_h2, dtype=np.float32)
    H = ctrl_h2.shape[0]
    S = H * n_sub
    states = np.empty((S + 1, 13))
    Jrun = np.empty(S + 1)
    ds = lib().orc_trajectory(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                              _ptr(x0, _dp), _ptr(ctrl_h2, _fp), H, float(dt), int(n_sub),
                              _ptr(states, _dp), _ptr(Jrun, _dp))
    return states, Jrun, int(ds)


def philox4x64_10(ctr, key):
    """The four 64-bit Philox words at counter `ctr` (4 ints) under `key` (2)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    p = C.POINTER(C.c_uint64)
    lib().orc_philox4x64_10(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def sample(prev, shift, sigma_rate, sigma_acc, key, nonce, N, H):
    """Warm-started Gaussian candidates, FP64 [H, N, 2] (see sampler.c)."""
    if prev is None:
        prev = np.zeros((0, 2), np.float32)
    prev = np.ascontiguousarray(prev, dtype=np.float32)
    out = np.empty((H, N, 2))
    lib().orc_sample(_ptr(prev, _fp), int(prev.shape[0]), int(shift), float(sigma_rate),
                     float(sigma_acc), int(key[0]), int(key[1]), int(nonce), int(N), int(H),
                     _ptr(out, _dp))
    return out


def bf16_round(x):
    """float32 -> bf16 bits (uint16), round to nearest even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32)


def bf16_terrain(heights, cell):
    """The BF16 terrain storage format restated on the host.  Per 8 x 8 block
    the FP32 plane c0 + cx (i mod 8) + cy (j mod 8) through the block's first
    node with the slopes of its first row and first column, every operation
    rounded to FP32 on its own; per node the bf16 (round to nearest even) of
    the height's residual from the plane and of the node slopes' (central
    differences, one-sided on the border, in FP64, rounded to FP32) residuals
    from the plane's slopes.  Returns
    (decoded FP32 heights, decoded slopes gx, gy as FP64, the bf16 words
    (res, gx, gy), the block planes [nby, nbx, 3])."""
    f32 = np.float32
    H = np.ascontiguousarray(heights, dtype=np.float32)
    ny, nx = H.shape
    nbx, nby = (nx + 7) // 8, (ny + 7) // 8
    plane = np.zeros((nby, nbx, 3), np.float32)
    for bj in range(nby):
        for bi in range(nbx):
            i0, j0 = 8 * bi, 8 * bj
            ni, nj = min(8, nx - i0), min(8, ny - j0)
            c0 = H[j0, i0]
            cx = f32(f32(H[j0, i0 + ni - 1] - c0) * f32(f32(1.0) / f32(ni - 1))) if ni > 1 else f32(0)
            cy = f32(f32(H[j0 + nj - 1, i0] - c0) * f32(f32(1.0) / f32(nj - 1))) if nj > 1 else f32(0)
            plane[bj, bi] = (c0, cx, cy)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    P = plane[jj // 8, ii // 8]
    base = (P[..., 0] + P[..., 1] * (ii & 7).astype(np.float32)).astype(np.float32)
    base = (base + (P[..., 2] * (jj & 7).astype(np.float32)).astype(np.float32)).astype(np.float32)
    res = (H - base).astype(np.float32)
    g = Terrain(H, cell)
    inv = np.float32(1.0 / cell)
    px = (P[..., 1] * inv).astype(np.float32)          # the plane's slopes
    py = (P[..., 2] * inv).astype(np.float32)
    w_res = bf16_round(res)
    w_gx = bf16_round((g.gx.astype(np.float32) - px).astype(np.float32))
    w_gy = bf16_round((g.gy.astype(np.float32) - py).astype(np.float32))
    h_dec = (base + bf16_value(w_res)).astype(np.float32)
    gx_dec = (px + bf16_value(w_gx)).astype(np.float32)
    gy_dec = (py + bf16_value(w_gy)).astype(np.float32)
    return (h_dec, gx_dec.astype(np.float64), gy_dec.astype(np.float64), (w_res, w_gx, w_gy), plane)


def cost_templated(veh: dict, cst: dict, ter: Terrain, x0, ctrl_h2, dt: float, n_sub: int):
    """J of one candidate through the adjoint's templated model (FP64)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    ctrl_h2 = np.ascontiguousarray(ctrl_h2, dtype=np.float32)
    return lib().orc_cost_templated(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                                    _ptr(x0, _dp), _ptr(ctrl_h2, _fp), ctrl_h2.shape[0], float(dt),
                                    int(n_sub))


def grad(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int):
    """J [N] and dJ/du [H, N, 2] by FP64 reverse-mode AD (adjoint.cpp)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
    H, N, _ = ctrl.shape
    J = np.empty(N)
    G = np.empty((H, N, 2))
    rc = lib().orc_grad_batch(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                              _ptr(x0, _fp), 1 if x0.ndim == 2 else 0, _ptr(ctrl, _fp), N, H,
                              float(dt), int(n_sub), _ptr(J, _dp), _ptr(G, _dp))
    if rc != 0:
        raise ValueError("oracle grad rejected its arguments")
    return J, G


def grad_margin(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int):
    """ESM margin [N] (min U_ESM over each trajectory) and d(margin)/du
    [H, N, 2] by FP64 reverse-mode AD (adjoint.cpp)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
    H, N, _ = ctrl.shape
    M = np.empty(N)
    G = np.empty((H, N, 2))
    rc = lib().orc_grad_margin_batch(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                                     _ptr(x0, _fp), 1 if x0.ndim == 2 else 0, _ptr(ctrl, _fp), N, H,
                                     float(dt), int(n_sub), _ptr(M, _dp), _ptr(G, _dp))
    if rc != 0:
        raise ValueError("oracle margin gradient rejected its arguments")
    return M, G


def margin_f64(veh: dict, cst: dict, ter: Terrain, x0, u, dt: float, n_sub: int):
    """The ESM margin of one candidate with FP64 controls u [H, 2]."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_margin_f64(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                                _ptr(x0, _dp), _ptr(u, _dp), u.shape[0], float(dt), int(n_sub))


def cost_f64(veh: dict, cst: dict, ter: Terrain, x0, u, dt: float, n_sub: int):
    """J of one candidate with FP64 controls u [H, 2] (for finite differences)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_cost_f64(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                              _ptr(x0, _dp), _ptr(u, _dp), u.shape[0], float(dt), int(n_sub))


# ---- The templated model (model.hpp): FP32 reference, restatement check, operation count
def _templated(fn, model, veh, cst, ter, x0, ctrl, dt, n_sub):
    n = 13 if model == "srb" else 7
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
    H, N, _ = ctrl.shape
    per = 1 if x0.ndim == 2 else 0
    J = np.empty(N)
    margin = np.empty(N)
    flags = np.empty(N, dtype=np.uint8)
    xf = np.empty((N, n))
    ms = np.empty(N, dtype=np.int32)
    rc = fn(0 if model == "srb" else 1, C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
            _ptr(x0, _fp), per, _ptr(ctrl, _fp), N, H, float(dt), int(n_sub), _ptr(J, _dp),
            _ptr(margin, _dp), _ptr(flags, _up), _ptr(xf, _dp), _ptr(ms, C.POINTER(C.c_int)))
    if rc != 0:
        raise ValueError("templated rollout rejected its arguments")
    return dict(J=J, margin=margin, flags=flags, xf=xf, min_step=ms)


def rollout_f32(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int, model="srb"):
    """The FP32 arithmetic reference (emul32.cpp): every model quantity rounded
    to FP32, position, heading and linear velocity accumulated exactly, the
    other state components rounded to FP32 each Euler step; node slopes
    stored in FP32.  Same outputs as rollout() (diag aside) plus the control step of the
    smallest per-step margin."""
    return _templated(lib().orc_rollout_f32, model, veh, cst, ter, x0, ctrl, dt, n_sub)


def rollout_templated(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int, model="srb"):
    """The templated restatement (model.hpp) in plain FP64."""
    return _templated(lib().orc_rollout_templated, model, veh, cst, ter, x0, ctrl, dt, n_sub)


OP_FIELDS = ("euler_steps", "add", "mul", "div", "sqrt", "sin", "cos", "atan2", "asin")


def count_ops(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int, model="srb"):
    """Operations of the templated model's rollout of every candidate, summed
    (additions count subtractions too), with the number of Euler steps run."""
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
    H, N, _ = ctrl.shape
    out = (C.c_long * 9)()
    rc = lib().orc_count_ops(0 if model == "srb" else 1, C.byref(vehicle(veh)), C.byref(cost(cst)),
                             C.byref(ter.c), _ptr(x0, _fp), 1 if x0.ndim == 2 else 0, _ptr(ctrl, _fp), N, H,
                             float(dt), int(n_sub), out)
    if rc != 0:
        raise ValueError("operation count rejected its arguments")
    return dict(zip(OP_FIELDS, [int(v) for v in out]))


# ---- Extended single-track (EST) planar model --------------------------------
EST_FIELDS = ("theta", "phi", "gBx", "gBy", "gBz", "aBx", "Fzf", "Fzr", "alpha_f", "alpha_r",
              "Fyf", "Fyr", "aBy", "margin", "L", "cm_fl", "cm_fr", "cm_rl", "cm_rr")


def est_rotation(phi, theta, psi):
    R = np.empty(9)
    lib().orc_est_rotation(float(phi), float(theta), float(psi), _ptr(R, _dp))
    return R.reshape(3, 3)


def est_evaluate(veh: dict, cst: dict, ter: Terrain, xi, zeta):
    """EST xi_dot [7] and the diagnostics named by EST_FIELDS."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    zeta = np.ascontiguousarray(zeta, dtype=np.float64)
    xd = np.empty(7)
    d = np.empty(len(EST_FIELDS))
    lib().orc_est_eval(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c), _ptr(xi, _dp),
                       _ptr(zeta, _dp), _ptr(xd, _dp), _ptr(d, _dp))
    return xd, dict(zip(EST_FIELDS, d))


def est_rollout(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int,
                want_xf=True, want_step_margin=False, want_diag=True, nthreads=0):
    """EST rollout of every candidate.  x0 float32 [7] or [N, 7]; ctrl float32 [H, N, 2]."""
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float32)
    H, N, _ = ctrl.shape
    per = 1 if x0.ndim == 2 else 0
    if per:
        assert x0.shape == (N, 7)
    J = np.empty(N)
    margin = np.empty(N)
    flags = np.empty(N, dtype=np.uint8)
    xf = np.empty((N, 7)) if want_xf else None
    sm = np.empty((H, N)) if want_step_margin else None
    diag = np.empty((N, 3)) if want_diag else None
    rc = lib().orc_est_rollout(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                               _ptr(x0, _fp), per, _ptr(ctrl, _fp), N, H, float(dt), int(n_sub),
                               _ptr(J, _dp), _ptr(margin, _dp), _ptr(flags, _up),
                               _ptr(xf, _dp), _ptr(sm, _dp), _ptr(diag, _dp), int(nthreads))
    if rc != 0:
        raise ValueError("oracle EST rollout rejected its arguments")
    return dict(J=J, margin=margin, flags=flags, xf=xf, step_margin=sm, diag=diag)


def est_plan(veh: dict, cst: dict, ter: Terrain, x0, ctrl, dt: float, n_sub: int, nthreads=0):
    """EST rollout, empirical argmin and the best candidate's outputs."""
    r = est_rollout(veh, cst, ter, x0, ctrl, dt, n_sub, want_step_margin=True, nthreads=nthreads)
    b = select(r["J"], r["flags"])
    ctrl = np.asarray(ctrl, dtype=np.float32)
    best_ctrl = ctrl[:, b, :].astype(np.float64)
    best_ctrl[:, 0] = np.clip(best_ctrl[:, 0], -veh["delta_rate_max"], veh["delta_rate_max"])
    r.update(best=b, n_feasible=int(np.count_nonzero(r["flags"] & FEASIBLE)),
             best_cost=float(r["J"][b]), best_margin=float(r["margin"][b]),
             best_ctrl=best_ctrl, best_step_margin=r["step_margin"][:, b].copy())
    return r


def est_trajectory(veh: dict, cst: dict, ter: Terrain, x0, ctrl_h2, dt: float, n_sub: int):
    """One EST candidate with every Euler state: [H n_sub + 1, 7]."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    ctrl_h2 = np.ascontiguousarray(ctrl_h2, dtype=np.float32)
    H = ctrl_h2.shape[0]
    states = np.empty((H * n_sub + 1, 7))
    lib().orc_est_trajectory(C.byref(vehicle(veh)), C.byref(cost(cst)), C.byref(ter.c),
                             _ptr(x0, _dp), _ptr(ctrl_h2, _fp), H, float(dt), int(n_sub),
                             _ptr(states, _dp))
    return states


def est_state_of(x13):
    """EST state (x, y, psi, v_By, w_Bz, delta, v_Bx) of an SRB state."""
    x13 = np.asarray(x13)
    return x13[..., [0, 1, 3, 7, 11, 12, 6]]


# ---- Terrain preprocessing ----------------------------------------------------
def lod_weights(cell: float, sigma: float):
    w = np.empty(2 * 4096 + 1)
    r = lib().orc_lod_weights(float(cell), float(sigma), 4096, _ptr(w, _dp))
    if r < 0:
        raise ValueError("kernel radius above 4096 cells")
    return w[: 2 * r + 1].copy()


def lod_smooth(heights, cell: float, sigma: float):
    """Gaussian level of detail of a heightmap, FP64 [ny, nx]."""
    f = np.ascontiguousarray(heights, dtype=np.float32)
    out = np.empty(f.shape)
    if lib().orc_lod_smooth(_ptr(f, _fp), f.shape[1], f.shape[0], float(cell), float(sigma),
                            _ptr(out, _dp)) != 0:
        raise ValueError("kernel radius above 4096 cells")
    return out


def _perimeters(polys):
    xy = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).reshape(-1, 2) for p, _ in polys]))
    start = np.zeros(len(polys) + 1, dtype=np.int32)
    start[1:] = np.cumsum([len(np.asarray(p).reshape(-1, 2)) for p, _ in polys])
    kind = np.ascontiguousarray([k for _, k in polys], dtype=np.int32)
    return xy, start, kind


def sdist(poly, kind: int, px: float, py: float) -> float:
    """Signed distance to one closed perimeter: kind 0 obstacle (negative
    inside), kind 1 path boundary (negative outside)."""
    xy = np.ascontiguousarray(np.asarray(poly, np.float64).reshape(-1, 2))
    return lib().orc_sdist(_ptr(xy, _dp), len(xy), int(kind), float(px), float(py))


def costmap(polys, nx: int, ny: int, cell: float, x0: float, y0: float, eps: float = 0.25,
            sigma: float = 1e6):
    """Summed distance-constraint cost rate at every node and the smallest
    signed distance; polys is a list of (vertices [n, 2], kind)."""
    xy, start, kind = _perimeters(polys)
    c = np.empty((ny, nx))
    s = np.empty((ny, nx))
    _ip = C.POINTER(C.c_int)
    lib().orc_costmap(_ptr(xy, _dp), _ptr(start, _ip), _ptr(kind, _ip), len(polys), int(nx), int(ny),
                      float(cell), float(x0), float(y0), float(eps), float(sigma), _ptr(c, _dp),
                      _ptr(s, _dp))
    return c, s
