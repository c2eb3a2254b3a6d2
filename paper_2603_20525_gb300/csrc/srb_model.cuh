// srb_model.cuh - FP32 device model of the single-rigid-body (SRB) off-road
// vehicle of arxiv 2603.20525, Sec. IV-A, with the sigmoid tire of Sec. III-A,
// the energy stability margin of Sec. IV-B and the running cost of Sec. IV-C.
//
// A candidate's state lives in registers for the whole horizon (in one
// thread, or repeated in the two or four threads that share its wheels), so a
// rollout step reads memory only for the four bilinear terrain lookups (16
// texels).  A wheel is written as its geometry (what depends on position and
// attitude: the lookup, the slope normal, the extension) and its forces
// (what depends on the velocities).
//
// Precision.  The arithmetic is FP32, compiled without implicit FMA
// contraction: every fused multiply-add is written as fmaf (or as fma2, its
// packed two-wide form, which rounds each half the same way), so the rounding
// of each expression is fixed by the source and the same in every kernel that
// inlines it.  The slowly varying, large-magnitude
// state components (position, heading and linear velocity) are accumulated as
// unevaluated sums hi + lo of two floats (Kahan's compensated summation per
// step, Knuth's TwoSum where the start is taken into the terrain frame), and
// positions are
// kept relative to the terrain origin and split into an integer cell and a
// fraction before the lookup.  Without that, the rounding of a 20-100 m
// coordinate (1e-6 m per Euler step) walks the wheels across the terrain by
// ~1e-5 m over a horizon, which the spring turns into force errors far above
// the 1e-4 relative agreement with the FP64 oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fastmath.cuh"

namespace atp {

// Vehicle constants in FP32, derived on the host in FP64 (App. B notation).
struct Veh {
    float M, halfM, invM;
    float dJyz, dJxz, dJxy;          // Jyy-Jzz, Jxx-Jzz, Jxx-Jyy
    float invJxx, invJyy, invJzz;
    float Lf, Lr, he, hR;            // he = e / 2
    float kf, kr, bf, br;
    float Fsf, Fsr;                  // nominal tire loading (g/2) K_zz,i
    float C, mu, mu2;
    float dmax, ddmax, g;
    float MgRbar;                    // M g Rbar
    float cpb, spb;                  // cos(phibar), sin(phibar)
    float tip;                       // pi/2 - phibar: roll at which U_ESM = 0
    // planar (EST) model: load-transfer coefficients and the critical lateral
    // acceleration M g / (2 K_zy)
    float Kzzf, Kzzr, Kzx, abar;
};

struct Cost {
    float wt, wc, wg, sigma, inv_eps;
    float gx_hi, gx_lo, gy_hi, gy_lo;  // goal relative to the terrain origin
    float goal_r2;
};

// Texel formats (ATP_TERRAIN_*): F32 = float4 (f, f_x, f_y, cost) per node;
// BF16 = four bf16 per node (f - plane, f_x - plane_x, f_y - plane_y, cost)
// with the FP32 plane (c0, cx, cy) of the node's 8 x 8 block.  F32W is F32
// with a window of the texels staged in the CTA's shared memory (`atp_win`,
// ww x wh nodes from node (wx0, wy0)): a lookup whose four corners lie in
// the window reads them there, any other from global memory.
enum { TEX_F32 = 0, TEX_BF16 = 1, TEX_F32W = 2 };

// the staged window of TEX_F32W (dynamic shared memory of the staging kernel)
extern __shared__ float4 atp_win[];

struct Terrain {
    const float4 *tex;               // F32 texels, row-major
    const uint2 *tex16;              // BF16 texels, row-major
    const float4 *plane16;           // BF16 block planes [ceil(ny/8)][ceil(nx/8)]
    int nbx;                         // blocks per row
    int nx, ny;
    int has_cm;                      // the texels carry a costmap
    float inv_cell;                  // 1 / cell
    float x0_hi, x0_lo, y0_hi, y0_lo;  // terrain origin
    int wx0, wy0, ww, wh;            // TEX_F32W: the staged window (ww, wh >= 2)
};

// x + y = s + e exactly (Knuth's TwoSum; no ordering precondition).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// hi + lo += d, with the carried low part folded into the increment first
// (Kahan's compensated summation; the new low part by Dekker's Fast2Sum,
// exact while |hi| >= |d + lo|, which holds for a state component and its
// increment over one Euler step except near the component's zero, where
// the plain FP32 sum it reduces to is accurate to the component's own small
// magnitude).  Folding keeps hi the FP32 value nearest the compensated sum,
// so the dynamics, which read hi alone, see the state as exactly
// accumulated; a low part summed on its own instead leaves hi the plain FP32
// running sum, whose error grows with every step (a constant increment
// rounds the same way each time).
__device__ __forceinline__ void acc2(float &hi, float &lo, float d)
{
    const float y = __fadd_rn(d, lo);
    const float s = __fadd_rn(hi, y);
    lo = __fsub_rn(y, __fsub_rn(s, hi));
    hi = s;
}

// Energy stability margin (Sec. IV-B): U = +/- M g Rbar (1 - sin(|phi| +
// phibar)) cos(theta), positive while the CoM is inside the footprint,
// |phi| < pi/2 - phibar.  sin(|phi| + phibar) is expanded with the already
// computed sin(phi), cos(phi), so it costs no extra transcendental.
__device__ __forceinline__ float esm(const Veh &V, float ph, float sph, float cph, float cth)
{
    float sabs = ph < 0.f ? -sph : sph;                  // sin(|phi|)
    float s = fmaf(sabs, V.cpb, cph * V.spb);            // sin(|phi| + phibar)
    float u = V.MgRbar * (1.f - s) * cth;
    return fabsf(ph) < V.tip ? u : -u;
}

// Position of the CoM in cell units split into an integer cell and a
// fraction, from the compensated coordinate hi + lo (metres from the origin).
__device__ __forceinline__ void cell_split(float hi, float lo, float inv_cell, int &ic, float &fc)
{
    const float u = fminf(fmaxf(hi * inv_cell, -4194304.f), 4194304.f);   // NaN -> low edge
    const float fl = floorf(u);
    ic = (int)fl;
    fc = fmaf(lo, inv_cell, fmaf(hi, inv_cell, -fl));
}

// One axis of a wheel lookup: CoM cell (ic, fc) plus the wheel's offset `o`
// metres; returns the clamped cell index in [0, n-2] and the weight in [0, 1]
// (queries clamped to the map, reading Q10).
// Written with selects rather than branches: the four wheels' lookups then
// form one basic block that the compiler can interleave (measured on the
// GB300: 9 % off a full-GPU plan, 3 to 10 % off the smaller ones).  The cell
// comes from one rounding-down conversion, which saturates for a huge or
// infinite offset and gives 0 for NaN; the sum with the CoM cell wraps
// (unsigned) instead of overflowing, and every out-of-range index is clamped
// below, so no lookup leaves the map.
__device__ __forceinline__ int axis(int ic, float fc, float o, float inv_cell, int n, float &a, bool &off)
{
    const float u = fmaf(o, inv_cell, fc);
    const int fi = __float2int_rd(u);
    const int i = (int)((unsigned)ic + (unsigned)fi);
    const float w = u - (float)fi;
    const bool below = i < 0, above = i >= n - 1;
    off = off || below || (above && (i > n - 1 || w > 0.f));
    a = below ? 0.f : (above ? 1.f : w);
    return below ? 0 : (above ? n - 2 : i);
}

// axis() for both axes of one lookup, with the cell coordinate and fraction
// of the two taken as pairs; bit for bit the same as two axis() calls
__device__ __forceinline__ void axis_xy(int icx, int icy, float2 fc, float2 o, float inv_cell, int nx,
                                        int ny, int &i, int &j, float &a, float &b, bool &off)
{
    const float2 u = fma2(o, splat2(inv_cell), fc);
    const int fx = __float2int_rd(u.x), fy = __float2int_rd(u.y);
    const float2 w = sub2(u, make_float2((float)fx, (float)fy));
    const int ix = (int)((unsigned)icx + (unsigned)fx);
    const int iy = (int)((unsigned)icy + (unsigned)fy);
    const bool bx = ix < 0, ex = ix >= nx - 1, by = iy < 0, ey = iy >= ny - 1;
    off = off || bx || (ex && (ix > nx - 1 || w.x > 0.f)) || by || (ey && (iy > ny - 1 || w.y > 0.f));
    a = bx ? 0.f : (ex ? 1.f : w.x);
    b = by ? 0.f : (ey ? 1.f : w.y);
    i = bx ? 0 : (ex ? nx - 2 : ix);
    j = by ? 0 : (ey ? ny - 2 : iy);
}

__device__ __forceinline__ float lerp2d(float t00, float t10, float t01, float t11, float a, float b)
{
    const float lo = fmaf(a, t10 - t00, t00), hi = fmaf(a, t11 - t01, t01);
    return fmaf(b, hi - lo, lo);
}

// lerp2d on two channels at once, bit for bit the same
__device__ __forceinline__ float2 lerp2d2(float2 t00, float2 t10, float2 t01, float2 t11, float2 a,
                                          float2 b)
{
    const float2 lo = fma2(a, sub2(t10, t00), t00), hi = fma2(a, sub2(t11, t01), t01);
    return fma2(b, sub2(hi, lo), lo);
}

// bilinear height, slopes and (when the terrain has a costmap) cost
__device__ __forceinline__ float4 lerp4(float4 t00, float4 t10, float4 t01, float4 t11, float a, float b,
                                        bool cm)
{
    const float2 a2 = splat2(a), b2 = splat2(b);
    const float2 xy = lerp2d2(make_float2(t00.x, t00.y), make_float2(t10.x, t10.y),
                              make_float2(t01.x, t01.y), make_float2(t11.x, t11.y), a2, b2);
    const float2 zw = lerp2d2(make_float2(t00.z, t00.w), make_float2(t10.z, t10.w),
                              make_float2(t01.z, t01.w), make_float2(t11.z, t11.w), a2, b2);
    return make_float4(xy.x, xy.y, zw.x, cm ? zw.y : 0.f);
}

// height of a block's plane (c0, cx, cy) at node (i, j): c0 + cx (i mod 8) +
// cy (j mod 8), every operation rounded on its own
__device__ __forceinline__ float block_plane(float4 P, int i, int j)
{
    return __fadd_rn(__fadd_rn(P.x, __fmul_rn(P.y, (float)(i & 7))), __fmul_rn(P.z, (float)(j & 7)));
}

// one BF16 texel decoded: height = block plane + residual
__device__ __forceinline__ float4 texel16(const Terrain &T, int i, int j)
{
    const uint2 u = __ldg(T.tex16 + (size_t)j * T.nx + i);
    const float4 P = __ldg(T.plane16 + (size_t)(j >> 3) * T.nbx + (i >> 3));
    float4 t;
    t.x = __fadd_rn(block_plane(P, i, j), __uint_as_float(u.x << 16));
    t.y = __fadd_rn(__fmul_rn(P.y, T.inv_cell), __uint_as_float(u.x & 0xffff0000u));
    t.z = __fadd_rn(__fmul_rn(P.z, T.inv_cell), __uint_as_float(u.y << 16));
    t.w = __uint_as_float(u.y & 0xffff0000u);
    return t;
}

template <int TEX>
__device__ __forceinline__ float4 bilerp(const Terrain &T, int i, int j, float a, float b)
{
    const bool cm = T.has_cm != 0;
    if (TEX == TEX_F32) {
        const float4 *r0 = T.tex + (size_t)j * T.nx + i;
        return lerp4(__ldg(r0), __ldg(r0 + 1), __ldg(r0 + T.nx), __ldg(r0 + T.nx + 1), a, b, cm);
    } else if (TEX == TEX_F32W) {
        // one generic pointer into the window or the texel array, so that a
        // warp whose lookups fall on both sides still issues four loads
        const unsigned li = (unsigned)(i - T.wx0), lj = (unsigned)(j - T.wy0);
        const bool in = li < (unsigned)(T.ww - 1) && lj < (unsigned)(T.wh - 1);
        const float4 *r0 = in ? atp_win + (lj * (unsigned)T.ww + li) : T.tex + (size_t)j * T.nx + i;
        const int s = in ? T.ww : T.nx;
        return lerp4(r0[0], r0[1], r0[s], r0[s + 1], a, b, cm);
    } else {
        return lerp4(texel16(T, i, j), texel16(T, i + 1, j), texel16(T, i, j + 1),
                     texel16(T, i + 1, j + 1), a, b, cm);
    }
}

// What the force of one wheel needs from the state's position and attitude
// alone: the local slope-normal tau in B (and 1 / tau_z) and the suspension
// extension chi at the contact point, and the costmap there.
struct WheelGeo {
    float tx, ty, tz, itz, chi, cost;
};

// One wheel's geometry (Sec. IV-A): contact point P = p + R rho, the terrain
// below it, the slope-normal tau ~ (-f_x, -f_y, 1) (reading Q1) resolved in
// B and the extension chi along it.  (icx, fcx), (icy, fcy) is the CoM's cell
// and fraction, z_hi + z_lo its height.  PAIRED takes the lookup's two axes
// as packed pairs: the same bits, measured faster with two lanes per
// candidate and slower with one or four.
template <int TEX, bool PAIRED = false>
__device__ __forceinline__ WheelGeo wheel_geo(const Veh &V, const Terrain &T, const float R[9], int icx,
                                              int icy, float fcx, float fcy, float z_hi, float z_lo,
                                              float rx, float ry, bool &off)
{
    // offset of the contact point from the CoM in W: R (rx, ry, -(h+R))
    const float2 oxy = fma2(splat2(rx), make_float2(R[0], R[3]),
                            fma2(splat2(ry), make_float2(R[1], R[4]),
                                 make_float2(-V.hR * R[2], -V.hR * R[5])));
    const float oz = fmaf(rx, R[6], fmaf(ry, R[7], -V.hR * R[8]));
    // terrain below the contact point
    float a, bb;
    int i, j;
    if constexpr (PAIRED) {
        axis_xy(icx, icy, make_float2(fcx, fcy), oxy, T.inv_cell, T.nx, T.ny, i, j, a, bb, off);
    } else {
        i = axis(icx, fcx, oxy.x, T.inv_cell, T.nx, a, off);
        j = axis(icy, fcy, oxy.y, T.inv_cell, T.ny, bb, off);
    }
    const float4 t = bilerp<TEX>(T, i, j, a, bb);
    // tau in B = R^T (-f_x, -f_y, 1)
    const float2 txy = fma2(make_float2(-R[3], -R[4]), splat2(t.z),
                            fma2(make_float2(-R[0], -R[1]), splat2(t.y), make_float2(R[6], R[7])));
    WheelGeo g;
    g.tx = txy.x;
    g.ty = txy.y;
    g.tz = fmaf(-R[5], t.z, fmaf(-R[2], t.y, R[8]));
    g.itz = rcp(g.tz);
    // P_z - f with the compensated CoM height
    g.chi = ((z_hi - t.x) + (oz + z_lo)) * g.itz;
    g.cost = t.w;
    return g;
}

// What one wheel contributes to the force and moment sums.
struct WheelOut {
    float Fz, Fy, cost;
};

// One wheel's forces (Sec. IV-A) at the body velocity (vx, vy, vz) and rate
// (wx, wy, wz): the contact point's body velocity v + w x rho, the extension
// rate chi_dot, spring and damper with liftoff, slip angle and sigmoid tire
// force.  PAIRED takes the extension rate's inner pair as a packed pair (the
// same bits).
template <bool PAIRED = false>
__device__ __forceinline__ WheelOut wheel_dyn(const Veh &V, const WheelGeo &g, float vx, float vy, float vz,
                                              float wx, float wy, float wz, float rx, float ry, float k,
                                              float b, float Fs, float di)
{
    // body velocity of the contact point: v + w x rho
    const float vix = fmaf(-wz, ry, fmaf(-wy, V.hR, vx));
    const float viy = fmaf(wx, V.hR, fmaf(wz, rx, vy));
    const float viz = fmaf(-wy, rx, fmaf(wx, ry, vz));
    // omega x b_z in B is (w_y, -w_x, 0)
    float chid;
    if constexpr (PAIRED) {
        const float2 rel = fma2(splat2(g.chi), make_float2(wx, -wy), make_float2(viy, vix));
        chid = fmaf(g.tz, viz, fmaf(g.ty, rel.x, g.tx * rel.y)) * g.itz;
    } else {
        chid = fmaf(g.tz, viz, fmaf(g.ty, fmaf(g.chi, wx, viy), g.tx * fmaf(-g.chi, wy, vix))) * g.itz;
    }
    const float Fk = fmaxf(fmaf(-k, g.chi, Fs), 0.f);
    const float Fz = Fk > 0.f ? fmaxf(fmaf(-b, chid, Fk), 0.f) : 0.f;   // = F_k + max(-b chid, -F_k)
    const float alpha = atan2_r(viy, vix) - di;
    const float Ca = V.C * alpha;
    const float Fy = Fz * (-Ca * V.mu) * rsq(fmaf(Ca, Ca, V.mu2));
    WheelOut w;
    w.Fz = Fz;
    w.Fy = Fy;
    w.cost = g.cost;
    return w;
}

// Per-step body quantities the four wheels share.
struct Body {
    float R[9];
    int icx, icy;            // CoM cell
    float fcx, fcy;          // CoM fraction of the cell
    float z_hi, z_lo;        // CoM height
    float vx, vy, vz, wx, wy, wz;
};

// One wheel (Sec. IV-A): its geometry, then its forces at the body's
// velocities.
template <int TEX, bool PAIRED = false>
__device__ __forceinline__ WheelOut wheel(const Veh &V, const Terrain &T, const Body &B, float rx, float ry,
                                          float k, float b, float Fs, float di, bool &off)
{
    const WheelGeo g = wheel_geo<TEX, PAIRED>(V, T, B.R, B.icx, B.icy, B.fcx, B.fcy, B.z_hi, B.z_lo, rx, ry,
                                              off);
    return wheel_dyn<PAIRED>(V, g, B.vx, B.vy, B.vz, B.wx, B.wy, B.wz, rx, ry, k, b, Fs, di);
}

}  // namespace atp
