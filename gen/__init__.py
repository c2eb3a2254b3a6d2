"""Seeded synthetic inputs for the rollout planner: terrain heightmaps, vehicles,
initial states and candidate control sequences.

This module produces input data only.  It holds none of the planner's
arithmetic (no vehicle dynamics, no terrain lookup, no constraint or cost), so
the FP64 oracle and the CUDA path can both consume its output without sharing
any code of the method.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) turned into uniforms on (0, 1)
and normals by the Box-Muller transform, all in FP64 numpy, so the same seed
gives the same bytes on any host.

The terrain shapes stand in for the paper's private photogrammetric scan of a
hilly off-road park (Sec. V-A: rough trails with bumps, ruts, berms and
banked turns).  The paper's scan, obstacle polygons and plant are not
available, so every workload here is synthetic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.ndimage import gaussian_filter

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n SplitMix64 outputs of the generator seeded by (seed, stream)."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF],
                             dtype=np.uint64))[0]
        ctr = np.arange(1, n + 1, dtype=np.uint64) * _GOLDEN + base
        return _mix(ctr)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniforms on the open interval (0, 1), FP64."""
    bits = splitmix64(seed, stream, n) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller, FP64."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[:m]))
    t = 2.0 * math.pi * u[m:]
    return np.concatenate([r * np.cos(t), r * np.sin(t)])[:n]


# ----------------------------------------------------------------------------
# Vehicles (SI units).  Keys follow the paper's notation table (App. A):
# M, J, L_f, L_r, e (track), h+R (CoM height over the contact patch), k, b,
# tire C and mu, delta_max, delta_rate_max, g.
# ----------------------------------------------------------------------------

def vehicle_mrzr() -> dict:
    """Polaris MRZR D4 of the paper's model and simulation-tire parameter tables (App. B)."""
    return dict(M=969.0, Jxx=280.9, Jyy=692.1, Jzz=810.7, Lf=1.565, Lr=1.148,
                e=1.280, hR=0.380 + 0.291, kf=4.2e4, kr=5.8e4, bf=3.1e3, br=4.3e3,
                C=6.1, mu=0.6, delta_max=0.639, delta_rate_max=1.0, g=9.81)


def vehicle_baseline() -> dict:
    """The 1000 kg benchmark vehicle: wheelbase 2.5 m, track 1.5 m, CoM height
    0.6 m, 40 kN/m spring and 3 kN s/m damper at every corner.  What the
    benchmark leaves open is filled from App. B: the front/rear split of the
    wheelbase in the MRZR's ratio, the MRZR inertias, the simulation tire
    (C = 6.1 /rad, mu = 0.6), delta_max = 0.639 rad, |delta_dot| <= 1 rad/s."""
    L = 2.5
    return dict(M=1000.0, Jxx=280.9, Jyy=692.1, Jzz=810.7,
                Lf=L * 1.565 / (1.565 + 1.148), Lr=L * 1.148 / (1.565 + 1.148),
                e=1.5, hR=0.6, kf=4.0e4, kr=4.0e4, bf=3.0e3, br=3.0e3,
                C=6.1, mu=0.6, delta_max=0.639, delta_rate_max=1.0, g=9.81)


def cost_default(goal_x: float, goal_y: float) -> dict:
    """Cost weights of Sec. IV-C: w_t = 5 /s, w_c = 8 /s per (rad/s)^2,
    w_g = 15 /m, sigma = 1e6 /s, goal radius 2.5 m.  eps_esm = 0 asks each
    side for its default, 10 % of the level-ground energy stability margin."""
    return dict(wt=5.0, wc=8.0, wg=15.0, sigma=1.0e6, eps_esm=0.0,
                goal_x=float(goal_x), goal_y=float(goal_y), goal_r=2.5)


# ----------------------------------------------------------------------------
# Terrain
# ----------------------------------------------------------------------------

@dataclass
class Terrain:
    """Row-major heightmap: heights[j, i] = f(x0 + i*cell, y0 + j*cell)."""
    heights: np.ndarray            # float32 [ny, nx]
    cell: float
    x0: float = 0.0
    y0: float = 0.0
    costmap: np.ndarray | None = None   # float32 [ny, nx] or None
    name: str = ""

    @property
    def nx(self) -> int:
        return int(self.heights.shape[1])

    @property
    def ny(self) -> int:
        return int(self.heights.shape[0])

    def grid(self):
        xs = self.x0 + self.cell * np.arange(self.nx, dtype=np.float64)
        ys = self.y0 + self.cell * np.arange(self.ny, dtype=np.float64)
        return np.meshgrid(xs, ys)


def _smoothstep(t):
    t = np.clip(t, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def fbm(n: int, cell: float, amplitude: float, seed: int, stream: int = 1,
        octaves: int = 5, dirs: int = 8, lambda0: float = 12.8) -> np.ndarray:
    """Spectral fractional-Brownian-motion-like field on an n x n grid (FP64).

    Octave o sums `dirs` plane waves with random directions and phases,
    wavelength lambda0 / 2**o and gain 0.5**o; the field is then scaled so
    that max |f| = amplitude."""
    u = uniform(seed, stream, octaves * dirs * 2)
    ang = 2.0 * math.pi * u[: octaves * dirs]
    phs = 2.0 * math.pi * u[octaves * dirs:]
    c = cell * np.arange(n, dtype=np.float64)
    # cos(kx x + ky y + p) = cos(kx x) cos(ky y + p) - sin(kx x) sin(ky y + p):
    # every wave is a rank-2 outer product, so the sum is one matrix product
    A = np.empty((n, 2 * octaves * dirs))
    B = np.empty((2 * octaves * dirs, n))
    for o in range(octaves):
        lam = lambda0 / 2.0 ** o
        g = 0.5 ** o
        for d in range(dirs):
            w = o * dirs + d
            a, p = ang[w], phs[w]
            kx = (2.0 * math.pi / lam) * math.cos(a)
            ky = (2.0 * math.pi / lam) * math.sin(a)
            A[:, 2 * w] = g * np.cos(ky * c + p)
            A[:, 2 * w + 1] = -g * np.sin(ky * c + p)
            B[2 * w] = np.cos(kx * c)
            B[2 * w + 1] = np.sin(kx * c)
    f = A @ B
    return f * (amplitude / np.max(np.abs(f)))


def srb_lod(f: np.ndarray, cell: float, sigma_m: float = 0.3) -> np.ndarray:
    """The single-rigid-body level of detail of Sec. V-B: the raw terrain
    smoothed by a Gaussian of 0.3 m standard deviation, so that it is planar
    at the length scale of a wheel as the model assumes."""
    if sigma_m <= 0:
        return f
    return gaussian_filter(f, sigma=sigma_m / cell, mode="nearest")


def _raised_cosine(s, height, base):
    half = 0.5 * base
    return np.where(np.abs(s) < half, height * 0.5 * (1.0 + np.cos(math.pi * s / half)), 0.0)


def terrain_plain(seed: int = 0, lod_sigma: float = 0.3) -> Terrain:
    """256 x 256 at 0.2 m: fBm (5 octaves, 0.5 m), two 0.4 m berms crossing
    the path obliquely at x = 9 m and 13 m, one 15 degree side slope over
    x in [15, 23] m blended in over 2 m; then the SRB level of detail."""
    n, cell = 256, 0.2
    f = fbm(n, cell, 0.5, seed, stream=11)
    X, Y = np.meshgrid(cell * np.arange(n), cell * np.arange(n))
    yc = 25.6
    for xc, deg in ((9.0, 30.0), (13.0, -30.0)):
        a = math.radians(deg)
        s = (X - xc) * math.cos(a) - (Y - yc) * math.sin(a)
        f += _raised_cosine(s, 0.4, 1.5)
    w = _smoothstep((X - 13.0) / 2.0) * _smoothstep((25.0 - X) / 2.0)
    f += w * math.tan(math.radians(15.0)) * (Y - yc)
    return Terrain(srb_lod(f, cell, lod_sigma).astype(np.float32), cell, name="plain-256-0.2m")


def terrain_scaled(seed: int = 0, n: int = 1024, cell: float = 0.1,
                   lod_sigma: float = 0.3) -> Terrain:
    """1024 x 1024 at 0.1 m: fBm (0.8 m), two 0.3 m deep, 0.3 m wide ruts
    1.5 m apart running along x with a 0.5 m sinusoidal wander, and side
    slopes alternating +/-20 degrees in 8 m segments along x, blended over 2 m;
    then the SRB level of detail."""
    f = fbm(n, cell, 0.8, seed, stream=12)
    X, Y = np.meshgrid(cell * np.arange(n), cell * np.arange(n))
    yc = 0.5 * n * cell
    wander = 0.5 * np.sin(2.0 * math.pi * X / 17.0)
    for off in (-0.75, 0.75):
        f -= _raised_cosine(Y - (yc + off + wander), 0.3, 0.3)
    seg = 8.0
    b = np.round(X / seg)                       # nearest segment boundary
    d = X - b * seg                             # signed distance to it, [-4, 4]
    right = np.where((b % 2) == 0, 1.0, -1.0)   # sign of the segment after it
    s = -right + 2.0 * right * _smoothstep((d + 1.0) / 2.0)   # 2 m blend
    f += s * math.tan(math.radians(20.0)) * (Y - yc)
    return Terrain(srb_lod(f, cell, lod_sigma).astype(np.float32), cell,
                   name=f"scaled-{n}-{cell}m")


def terrain_tile(side: int, seed: int, cell: float = 0.1, lod_sigma: float = 0.3) -> Terrain:
    """A serving vehicle's own tile: fBm (0.6 m) plus one 0.4 m berm and a
    12 degree bank, side x side nodes at `cell`; then the SRB level of detail."""
    f = fbm(side, cell, 0.6, seed, stream=13)
    X, Y = np.meshgrid(cell * np.arange(side), cell * np.arange(side))
    ext = side * cell
    u = uniform(seed, 14, 3)
    xc = ext * (0.3 + 0.4 * u[0])
    a = math.radians(60.0 * (u[1] - 0.5))
    s = (X - xc) * math.cos(a) - (Y - 0.5 * ext) * math.sin(a)
    f += _raised_cosine(s, 0.4, 1.5)
    f += math.tan(math.radians(12.0 * (2.0 * u[2] - 1.0))) * (Y - 0.5 * ext) * 0.3
    return Terrain(srb_lod(f, cell, lod_sigma).astype(np.float32), cell,
                   name=f"tile-{side}-{cell}m-s{seed}")


def terrain_plane(nx: int, ny: int, cell: float, a: float, b: float, c: float,
                  x0: float = 0.0, y0: float = 0.0) -> Terrain:
    """f = a + b x + c y sampled on the grid (exact in FP32 when a, b, c, cell
    and the origin are dyadic and the grid is small)."""
    xs = x0 + cell * np.arange(nx)
    ys = y0 + cell * np.arange(ny)
    X, Y = np.meshgrid(xs, ys)
    return Terrain((a + b * X + c * Y).astype(np.float32), cell, x0, y0, name="plane")


# ----------------------------------------------------------------------------
# Initial state and candidates
# ----------------------------------------------------------------------------

STATE = ("x", "y", "z", "psi", "theta", "phi", "vx", "vy", "vz", "wx", "wy", "wz", "delta")


def settled_state(terrain: Terrain, veh: dict, x: float, y: float, psi: float,
                  vx: float) -> np.ndarray:
    """Chassis placed on the least-squares plane through the terrain nodes
    nearest to its four nominal wheel positions: body z along the plane
    normal, heading psi projected into the plane, CoM at h+R above it.
    Rates zero, steering zero.  Returns float32 [13] in the paper's state
    order (x, y, z, psi, theta, phi, vx, vy, vz, wx, wy, wz, delta)."""
    cps, sps = math.cos(psi), math.sin(psi)
    pts = []
    for lx in (veh["Lf"], -veh["Lr"]):
        for ly in (0.5 * veh["e"], -0.5 * veh["e"]):
            px = x + cps * lx - sps * ly
            py = y + sps * lx + cps * ly
            i = int(round((px - terrain.x0) / terrain.cell))
            j = int(round((py - terrain.y0) / terrain.cell))
            i = min(max(i, 0), terrain.nx - 1)
            j = min(max(j, 0), terrain.ny - 1)
            pts.append((terrain.x0 + i * terrain.cell, terrain.y0 + j * terrain.cell,
                        float(terrain.heights[j, i])))
    P = np.array(pts)
    A = np.stack([np.ones(4), P[:, 0], P[:, 1]], axis=1)
    (a, b, c), *_ = np.linalg.lstsq(A, P[:, 2], rcond=None)
    n = np.array([-b, -c, 1.0])
    n /= np.linalg.norm(n)
    hx = np.array([cps, sps, 0.0])
    bx = hx - np.dot(hx, n) * n
    bx /= np.linalg.norm(bx)
    by = np.cross(n, bx)
    Rm = np.stack([bx, by, n], axis=1)           # columns = body axes in world
    theta = -math.asin(max(-1.0, min(1.0, Rm[2, 0])))
    phi = math.atan2(Rm[2, 1], Rm[2, 2])
    yaw = math.atan2(Rm[1, 0], Rm[0, 0])
    # CoM so that the plane point below it, along n, is h+R away
    z = (a + b * (x - veh["hR"] * n[0]) + c * (y - veh["hR"] * n[1])) + veh["hR"] * n[2]
    s = np.zeros(13)
    s[0], s[1], s[2] = x, y, z
    s[3], s[4], s[5] = yaw, theta, phi
    s[6] = vx
    return s.astype(np.float32)


def candidates(N: int, H: int, seed: int, sigma_rate: float = 0.2,
               sigma_acc: float = 0.3, nominal=(0.0, 0.0)) -> np.ndarray:
    """Candidate controls zeta = (steering rate [rad/s], longitudinal
    acceleration [m/s^2]) held per control step, float32 [H, N, 2]
    (time-major).  Candidate 0 is the unperturbed nominal; the others are
    i.i.d. normal perturbations about it."""
    u = np.empty((H, N, 2), dtype=np.float64)
    u[..., 0] = nominal[0] + sigma_rate * normal(seed, 21, H * N).reshape(H, N)
    u[..., 1] = nominal[1] + sigma_acc * normal(seed, 22, H * N).reshape(H, N)
    u[:, 0, 0] = nominal[0]
    u[:, 0, 1] = nominal[1]
    return u.astype(np.float32)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    terrain: Terrain
    vehicle: dict
    cost: dict
    x0: np.ndarray                  # float32 [13] (shared) or [N, 13]
    ctrl: np.ndarray                # float32 [H, N, 2]
    dt: float
    n_sub: int
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.ctrl.shape[1])

    @property
    def H(self) -> int:
        return int(self.ctrl.shape[0])


def workload_plain(seed: int = 0, N: int = 1024, H: int = 40, dt: float = 0.05,
                   goal=(45.0, 25.6)) -> Workload:
    """Plain single plan: 1024 candidates, horizon 40 at dt = 0.05 s (10 Euler
    substeps of 5 ms), 8 m/s straight nominal from (5, 25.6) on the 256^2
    terrain; steering-rate sigma 0.2 rad/s, acceleration sigma 0.3 m/s^2."""
    ter = terrain_plain(seed)
    veh = vehicle_baseline()
    x0 = settled_state(ter, veh, 5.0, 25.6, 0.0, 8.0)
    ctrl = candidates(N, H, seed)
    return Workload("plain-1024x40", ter, veh, cost_default(*goal), x0, ctrl, dt,
                    n_sub=max(1, math.ceil(round(dt / 0.005, 9))),
                    meta=dict(seed=seed))


def workload_scaled(seed: int = 0, N: int = 16384, H: int = 100, dt: float = 0.02,
                    terrain: Terrain | None = None) -> Workload:
    """Scaled rollout: 16384 candidates, horizon 100 at dt = 0.02 s (4
    substeps), per-candidate initial speed uniform in [5, 15] m/s, from
    (10, 51.2) on the 1024^2 terrain at 0.1 m."""
    ter = terrain if terrain is not None else terrain_scaled(seed)
    veh = vehicle_baseline()
    base = settled_state(ter, veh, 10.0, 51.2, 0.0, 10.0)
    x0 = np.repeat(base[None, :], N, axis=0)
    x0[:, 6] = (5.0 + 10.0 * uniform(seed, 31, N)).astype(np.float32)
    ctrl = candidates(N, H, seed)
    return Workload(f"scaled-{N}x{H}", ter, veh, cost_default(95.0, 51.2), x0, ctrl, dt,
                    n_sub=max(1, math.ceil(round(dt / 0.005, 9))),
                    meta=dict(seed=seed))


def n_substeps(dt: float, h_max: float = 0.005) -> int:
    """Euler substeps per control step: ceil(dt / 5 ms)."""
    return max(1, math.ceil(round(dt / h_max, 9)))


@dataclass
class FleetVehicle:
    """One vehicle of a serving fleet: its own terrain tile, parameters,
    goal and settled start."""
    terrain: Terrain
    vehicle: dict
    cost: dict
    x0: np.ndarray
    key: tuple


def fleet(n: int = 32, seed: int = 0, sides=(512, 1024, 2048)):
    """n vehicles, each on its own seeded 0.1 m tile of side drawn from
    `sides`, alternately the benchmark vehicle and the MRZR, started settled
    at the tile centre at 5-10 m/s with the goal 40 m ahead."""
    u = uniform(seed, 41, 4 * n)
    out = []
    for v in range(n):
        side = int(sides[min(int(u[4 * v] * len(sides)), len(sides) - 1)])
        t = terrain_tile(side, seed * 1000 + v)
        veh = vehicle_baseline() if v % 2 == 0 else vehicle_mrzr()
        ext = side * t.cell
        psi = math.pi * (2.0 * u[4 * v + 1] - 1.0)
        x = y = 0.5 * ext
        x0 = settled_state(t, veh, x, y, psi, 5.0 + 5.0 * u[4 * v + 2])
        cost = cost_default(x + 40.0 * math.cos(psi), y + 40.0 * math.sin(psi))
        out.append(FleetVehicle(t, veh, cost, x0, (seed + 1, v + 1)))
    return out


def candidates_uniform(N: int, H: int, seed: int, rate_max: float = 1.0) -> np.ndarray:
    """The paper's sampling (Sec. IV-D, V): i.i.d. uniform steering rates over
    the admissible set |delta_dot| <= rate_max, zero longitudinal
    acceleration; float32 [H, N, 2]."""
    u = np.zeros((H, N, 2), dtype=np.float64)
    u[..., 0] = rate_max * (2.0 * uniform(seed, 23, H * N).reshape(H, N) - 1.0)
    return u.astype(np.float32)


def workload_paper(seed: int = 0, N: int = 204288) -> Workload:
    """The paper's real-time configuration (Sec. IV-D): N = 204,288 candidates
    of 16 zero-order-hold steps of 0.25 s (a 4 s horizon, 800 Euler steps of
    5 ms), steering only, on the scaled 1024^2 terrain, MRZR vehicle at
    7.5 m/s."""
    ter = terrain_scaled(seed)
    veh = vehicle_mrzr()
    x0 = settled_state(ter, veh, 10.0, 51.2, 0.0, 7.5)
    ctrl = candidates_uniform(N, 16, seed)
    return Workload(f"paper-{N}x16", ter, veh, cost_default(95.0, 51.2), x0, ctrl, 0.25,
                    n_sub=50, meta=dict(seed=seed))


def obstacles(terrain: Terrain, seed: int, n: int = 4, path_margin: float = 4.0):
    """Perimeters for the distance constraints (Sec. IV-C): n convex polygonal
    obstacles (5 to 9 vertices on a jittered circle of radius 0.6-1.5 m)
    scattered over the middle of the map, and one path boundary, the map
    shrunk by path_margin metres on every side.  Returns [(vertices [k, 2]
    float64 world metres, kind)] with kind 0 obstacle, 1 path boundary."""
    ext_x = (terrain.nx - 1) * terrain.cell
    ext_y = (terrain.ny - 1) * terrain.cell
    u = uniform(seed, 41, 6 * n)
    out = []
    for q in range(n):
        cx = terrain.x0 + ext_x * (0.2 + 0.6 * u[6 * q])
        cy = terrain.y0 + ext_y * (0.3 + 0.4 * u[6 * q + 1])
        r = 0.6 + 0.9 * u[6 * q + 2]
        k = 5 + int(5 * u[6 * q + 3]) % 5
        a0 = 2 * math.pi * u[6 * q + 4]
        jit = uniform(seed, 42 + q, k)
        ang = a0 + 2 * math.pi * (np.arange(k) + 0.3 * (jit - 0.5)) / k
        out.append((np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], 1), 0))
    m = path_margin
    box = np.array([[terrain.x0 + m, terrain.y0 + m], [terrain.x0 + ext_x - m, terrain.y0 + m],
                    [terrain.x0 + ext_x - m, terrain.y0 + ext_y - m], [terrain.x0 + m, terrain.y0 + ext_y - m]])
    out.append((box, 1))
    return out


def workload_est(seed: int = 0, N: int = 1024, H: int = 40, dt: float = 0.05, scaled: bool = False) -> Workload:
    """The planar model's workloads: the plain (or scaled) configuration on the
    planar model's level of detail (Gaussian of 1.5 m, Sec. V-B), with the
    SRB start state reduced to (x, y, psi, v_By, w_Bz, delta, v_Bx)."""
    if scaled:
        w = workload_scaled(seed, N=N, H=H, dt=dt, terrain=terrain_scaled(seed, lod_sigma=1.5))
    else:
        ter = terrain_plain(seed, lod_sigma=1.5)
        veh = vehicle_baseline()
        x0 = settled_state(ter, veh, 5.0, 25.6, 0.0, 8.0)
        w = Workload("plain", ter, veh, cost_default(45.0, 25.6), x0, candidates(N, H, seed), dt,
                     n_sub=n_substeps(dt), meta=dict(seed=seed))
    x0 = w.x0[..., [0, 1, 3, 7, 11, 12, 6]].astype(np.float32)
    return Workload(f"est-{w.name}", w.terrain, w.vehicle, w.cost, x0, w.ctrl, w.dt, w.n_sub, meta=w.meta)
