// adjoint.cu - hand-written reverse-mode adjoint of the discrete rollout
// (arxiv 2603.20525, Sec. IV-A..IV-C): the gradient, with respect to the raw
// control sequence u of each of K candidates, of its cost J = sum over Euler
// steps of h L + Phi, or of its ESM margin, the minimum of U_ESM over every
// state of the trajectory (Sec. IV-B; the constraint the soft cost guards).
// The margin's gradient is that of U_ESM at the state holding the minimum
// (the first one on ties), as a subgradient of the minimum.
//
// Four threads per candidate, one wheel each, as in the plan kernel's
// four-lane layout: every lane repeats the body arithmetic and its adjoint
// bit-identically, runs its own wheel forwards and backwards, and the quad
// exchanges only sums (the force and moment sums forwards; the wheels'
// contributions to the body adjoints backwards).  The forward pass stores the
// state every `ckpt` control steps; the reverse pass recomputes one segment
// at a time into a per-lane buffer and walks its Euler steps backwards (for
// a small grid on separate warps, the next segment recomputed while this one
// is walked).  Each backward step recomputes the step's intermediates from
// the stored state and propagates the state adjoint lambda through the Euler
// update, the state derivative A(xi) + B zeta, the force and moment sums,
// every wheel (contact kinematics, bilinear terrain, suspension with
// liftoff, slip and tire), the rotation and the running cost with its ESM
// soft constraint.  Branches (spring and damper liftoff, steering clamps,
// off-map clamping, the goal test) follow the forward pass's choice, so the
// result is the derivative of the piecewise-smooth discrete map along the
// primal trajectory.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "adjoint.cuh"
#include "atp.h"
#include "srb_model.cuh"

namespace atp {

namespace {

struct St {
    float x, xl, y, yl, z, zl, psi, psil, th, ph;
    float vx, vxl, vy, vyl, vz, vzl, wx, wy, wz, d;
};
constexpr int kStFloats = 20;

__device__ __forceinline__ void st_store(float *dst, size_t stride, const St &s)
{
    const float *v = &s.x;
#pragma unroll
    for (int c = 0; c < kStFloats; ++c) dst[c * stride] = v[c];
}

__device__ __forceinline__ void st_load(const float *src, size_t stride, St &s)
{
    float *v = &s.x;
#pragma unroll
    for (int c = 0; c < kStFloats; ++c) v[c] = src[c * stride];
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

// sum over the four lanes of a candidate (the same bits in every lane)
__device__ __forceinline__ float qsum(float v, unsigned mask)
{
    v += __shfl_xor_sync(mask, v, 1);
    v += __shfl_xor_sync(mask, v, 2);
    return v;
}

// this lane's wheel: fl, fr, rl, rr for q = 0..3
struct Lane {
    int q;
    unsigned mask;
    bool front;
    float rx, ry, k, b, Fs;
};

__device__ __forceinline__ Lane lane_of(const Veh &V, int q, unsigned mask)
{
    Lane l;
    l.q = q;
    l.mask = mask;
    l.front = q < 2;
    l.rx = l.front ? V.Lf : -V.Lr;
    l.ry = (q & 1) ? -V.he : V.he;
    l.k = l.front ? V.kf : V.kr;
    l.b = l.front ? V.bf : V.br;
    l.Fs = l.front ? V.Fsf : V.Fsr;
    return l;
}

// a lookup axis: cell, weight and whether the query was clamped
__device__ __forceinline__ int axis_c(int ic, float fc, float o, float inv_cell, int n, float &a, bool &clamped)
{
    const float u = fmaf(o, inv_cell, fc);
    const float fl = floorf(u);
    const int i = ic + (int)fmaxf(fminf(fl, 4194304.f), -4194304.f);
    const float w = u - fl;
    const bool below = i < 0, above = i >= n - 1;
    clamped = below || above;
    a = below ? 0.f : (above ? 1.f : w);
    return below ? 0 : (above ? n - 2 : i);
}

// every intermediate of one wheel that its adjoint needs
struct WF {
    float ox, oy, oz, vix, viy, viz;
    float a, b;
    bool cx, cy;
    float4 t00, t10, t01, t11, t;
    float tx, ty, tz, itz, Q, chi, A, Bv, N, chid, Fk, Fb0, Fz, alpha, Ca, T, Fy;
};

__device__ __forceinline__ void wheel_fwd(const Veh &V, const Terrain &T, const float R[9], int icx, float fcx,
                                          int icy, float fcy, float z, float zl, float vx, float vy, float vz,
                                          float wx, float wy, float wz, float rx, float ry, float k, float b,
                                          float Fs, float di, WF &w)
{
    w.ox = fmaf(rx, R[0], fmaf(ry, R[1], -V.hR * R[2]));
    w.oy = fmaf(rx, R[3], fmaf(ry, R[4], -V.hR * R[5]));
    w.oz = fmaf(rx, R[6], fmaf(ry, R[7], -V.hR * R[8]));
    w.vix = fmaf(-wz, ry, fmaf(-wy, V.hR, vx));
    w.viy = fmaf(wx, V.hR, fmaf(wz, rx, vy));
    w.viz = fmaf(-wy, rx, fmaf(wx, ry, vz));
    const int i = axis_c(icx, fcx, w.ox, T.inv_cell, T.nx, w.a, w.cx);
    const int j = axis_c(icy, fcy, w.oy, T.inv_cell, T.ny, w.b, w.cy);
    const float4 *r0 = T.tex + (size_t)j * T.nx + i;
    w.t00 = __ldg(r0);
    w.t10 = __ldg(r0 + 1);
    w.t01 = __ldg(r0 + T.nx);
    w.t11 = __ldg(r0 + T.nx + 1);
    w.t = lerp4(w.t00, w.t10, w.t01, w.t11, w.a, w.b, T.has_cm != 0);
    w.tx = fmaf(-R[3], w.t.z, fmaf(-R[0], w.t.y, R[6]));
    w.ty = fmaf(-R[4], w.t.z, fmaf(-R[1], w.t.y, R[7]));
    w.tz = fmaf(-R[5], w.t.z, fmaf(-R[2], w.t.y, R[8]));
    w.itz = rcp(w.tz);
    w.Q = (z - w.t.x) + (w.oz + zl);
    w.chi = w.Q * w.itz;
    w.A = fmaf(-w.chi, wy, w.vix);
    w.Bv = fmaf(w.chi, wx, w.viy);
    w.N = fmaf(w.tz, w.viz, fmaf(w.ty, w.Bv, w.tx * w.A));
    w.chid = w.N * w.itz;
    w.Fk = fmaxf(fmaf(-k, w.chi, Fs), 0.f);
    w.Fb0 = fmaf(-b, w.chid, w.Fk);
    w.Fz = w.Fk > 0.f ? fmaxf(w.Fb0, 0.f) : 0.f;
    w.alpha = atan2_r(w.viy, w.vix) - di;
    w.Ca = V.C * w.alpha;
    const float is = rsq(fmaf(w.Ca, w.Ca, V.mu2));
    w.T = (-w.Ca * V.mu) * is;                    // F_y / F_z
    w.Fy = w.Fz * w.T;
}

// adjoint accumulators of one Euler step
struct Adj {
    float R[9];
    float x, y, z, vx, vy, vz, wx, wy, wz, d;
};

// one wheel backwards: given a_Fz, a_Fy and a_cost of this wheel, accumulate
// the adjoints of R, of the CoM position and of the rates
__device__ __forceinline__ void wheel_adj(const Veh &V, const Terrain &T, const float R[9], float wx, float wy,
                                          float rx, float ry, float k, float b, float di_is_delta, const WF &w,
                                          float aFz, float aFy, float aC, Adj &ad, float &a_d)
{
    // tire: Fy = Fz T(Ca), T = -mu Ca / sqrt(mu^2 + Ca^2), T' = -mu^3 / (mu^2 + Ca^2)^(3/2)
    aFz += aFy * w.T;
    const float den = fmaf(w.Ca, w.Ca, V.mu2);
    const float is = rsq(den);
    const float dT = -V.mu * V.mu2 * is * is * is;
    const float aAlpha = aFy * w.Fz * dT * V.C;
    // alpha = atan2(viy, vix) - di
    const float r2 = fmaf(w.vix, w.vix, w.viy * w.viy);
    float aVix = 0.f, aViy = 0.f;
    if (r2 > 0.f) {
        const float ir2 = rcp(r2);
        aViy += aAlpha * w.vix * ir2;
        aVix -= aAlpha * w.viy * ir2;
    }
    a_d -= aAlpha * di_is_delta;
    // suspension: Fz = max(Fk - b chid, 0) while Fk > 0
    float aFk = 0.f, aChid = 0.f;
    if (w.Fk > 0.f && w.Fb0 > 0.f) {
        aFk = aFz;
        aChid = -b * aFz;
    }
    float aChi = 0.f;
    if (w.Fk > 0.f) aChi -= k * aFk;                 // Fk = Fs - k chi
    // chid = N itz, N = tx A + ty B + tz viz
    const float aN = aChid * w.itz;
    float aItz = aChid * w.N;
    float aTx = aN * w.A, aTy = aN * w.Bv, aTz = aN * w.viz;
    const float aA = aN * w.tx, aB = aN * w.ty;
    float aViz = aN * w.tz;
    aVix += aA;
    aChi -= aA * wy;
    ad.wy -= aA * w.chi;
    aViy += aB;
    aChi += aB * wx;
    ad.wx += aB * w.chi;
    // chi = Q itz, Q = (z - f) + (oz + zl)
    const float aQ = aChi * w.itz;
    aItz += aChi * w.Q;
    ad.z += aQ;
    float aF = -aQ;                                  // interpolated height
    float aOz = aQ;
    // itz = 1 / tz
    aTz -= aItz * w.itz * w.itz;
    // tau = R^T (-f_x, -f_y, 1)
    ad.R[6] += aTx;
    ad.R[0] -= aTx * w.t.y;
    ad.R[3] -= aTx * w.t.z;
    ad.R[7] += aTy;
    ad.R[1] -= aTy * w.t.y;
    ad.R[4] -= aTy * w.t.z;
    ad.R[8] += aTz;
    ad.R[2] -= aTz * w.t.y;
    ad.R[5] -= aTz * w.t.z;
    const float aGx = -(aTx * R[0] + aTy * R[1] + aTz * R[2]);   // interpolated f_x
    const float aGy = -(aTx * R[3] + aTy * R[4] + aTz * R[5]);   // interpolated f_y
    // bilinear: d/da = (1-b)(t10 - t00) + b (t11 - t01), d/db = hi - lo
    const float4 &t00 = w.t00, &t10 = w.t10, &t01 = w.t01, &t11 = w.t11;
    const float ob = 1.f - w.b, oa = 1.f - w.a;
    const float dA_f = ob * (t10.x - t00.x) + w.b * (t11.x - t01.x);
    const float dA_gx = ob * (t10.y - t00.y) + w.b * (t11.y - t01.y);
    const float dA_gy = ob * (t10.z - t00.z) + w.b * (t11.z - t01.z);
    const float dA_c = ob * (t10.w - t00.w) + w.b * (t11.w - t01.w);
    const float dB_f = oa * (t01.x - t00.x) + w.a * (t11.x - t10.x);
    const float dB_gx = oa * (t01.y - t00.y) + w.a * (t11.y - t10.y);
    const float dB_gy = oa * (t01.z - t00.z) + w.a * (t11.z - t10.z);
    const float dB_c = oa * (t01.w - t00.w) + w.a * (t11.w - t10.w);
    const float aWa = aF * dA_f + aGx * dA_gx + aGy * dA_gy + aC * dA_c;
    const float aWb = aF * dB_f + aGx * dB_gx + aGy * dB_gy + aC * dB_c;
    float aOx = 0.f, aOy = 0.f;
    if (!w.cx) {
        ad.x += aWa * T.inv_cell;
        aOx += aWa * T.inv_cell;
    }
    if (!w.cy) {
        ad.y += aWb * T.inv_cell;
        aOy += aWb * T.inv_cell;
    }
    // contact velocity v + w x rho, rho = (rx, ry, -(h+R))
    ad.vx += aVix;
    ad.wy -= aVix * V.hR;
    ad.wz -= aVix * ry;
    ad.vy += aViy;
    ad.wz += aViy * rx;
    ad.wx += aViy * V.hR;
    ad.vz += aViz;
    ad.wx += aViz * ry;
    ad.wy -= aViz * rx;
    // contact offset R rho
    ad.R[0] += aOx * rx;
    ad.R[1] += aOx * ry;
    ad.R[2] -= aOx * V.hR;
    ad.R[3] += aOy * rx;
    ad.R[4] += aOy * ry;
    ad.R[5] -= aOy * V.hR;
    ad.R[6] += aOz * rx;
    ad.R[7] += aOz * ry;
    ad.R[8] -= aOz * V.hR;
}

struct StepOut {
    float L;
    bool stepped;     // false: the goal was reached before this step
};

// One forward Euler step (the four-lane arithmetic of the plan kernel);
// returns the running cost rate.
__device__ __forceinline__ StepOut step_fwd(const GradParams &p, St &s, float dd, float ax, const Lane &ln)
{
    const Veh &V = p.V;
    const Cost &Cc = p.C;
    const Terrain &T = p.T;
    StepOut o;
    o.L = 0.f;
    o.stepped = false;
    const float gdx = (s.x - Cc.gx_hi) + (s.xl - Cc.gx_lo);
    const float gdy = (s.y - Cc.gy_hi) + (s.yl - Cc.gy_lo);
    if (fmaf(gdx, gdx, gdy * gdy) <= Cc.goal_r2) return o;
    o.stepped = true;
    float sps, cps, sth, cth, sph, cph, sd, cd;
    sincos_r(s.psi, sps, cps);
    sincos_r(s.th, sth, cth);
    sincos_r(s.ph, sph, cph);
    sincos_r(s.d, sd, cd);
    const float U = esm(V, s.ph, sph, cph, cth);
    float R[9];
    R[0] = cps * cth;
    R[1] = fmaf(cps * sph, sth, -cph * sps);
    R[2] = fmaf(cph * cps, sth, sph * sps);
    R[3] = cth * sps;
    R[4] = fmaf(sph * sps, sth, cph * cps);
    R[5] = fmaf(cph * sps, sth, -cps * sph);
    R[6] = -sth;
    R[7] = cth * sph;
    R[8] = cph * cth;
    int icx, icy;
    float fcx, fcy;
    cell_split(s.x, s.xl, T.inv_cell, icx, fcx);
    cell_split(s.y, s.yl, T.inv_cell, icy, fcy);
    const float gBx = -V.g * R[6], gBy = -V.g * R[7], gBz = -V.g * R[8];
    WF w;
    wheel_fwd(V, T, R, icx, fcx, icy, fcy, s.z, s.zl, s.vx, s.vy, s.vz, s.wx, s.wy, s.wz, ln.rx, ln.ry, ln.k,
              ln.b, ln.Fs, ln.front ? s.d : 0.f, w);
    const float fy = ln.front ? w.Fy * cd : w.Fy;
    const float FyB = qsum(fy, ln.mask);
    const float FzB = qsum(w.Fz, ln.mask);
    const float Mx = fmaf(V.hR, FyB, qsum(ln.ry * w.Fz, ln.mask));
    float My = qsum(-ln.rx * w.Fz, ln.mask);
    const float Mz = qsum(ln.rx * fy, ln.mask);
    const float csum = T.has_cm ? qsum(w.t.w, ln.mask) : 0.f;
    const float Fx = V.halfM * fmaf(-s.wz, s.vy, fmaf(s.wy, s.vz, ax - gBx));
    My = fmaf(-V.hR, 2.f * Fx, My);
    const float soft = fmaxf(fmaf(-U, Cc.inv_eps, 1.f), 0.f);
    o.L = fmaf(Cc.sigma * soft, soft, fmaf(Cc.wc * dd, dd, Cc.wt)) + csum;
    const float ic = rcp(cth);
    const float wsc = fmaf(sph, s.wy, cph * s.wz);
    const float dx = fmaf(R[2], s.vz, fmaf(R[1], s.vy, R[0] * s.vx));
    const float dy = fmaf(R[5], s.vz, fmaf(R[4], s.vy, R[3] * s.vx));
    const float dz = fmaf(R[8], s.vz, fmaf(R[7], s.vy, R[6] * s.vx));
    const float dpsi = wsc * ic;
    const float dth = fmaf(cph, s.wy, -sph * s.wz);
    const float dph = fmaf(wsc, sth * ic, s.wx);
    const float dvy = fmaf(-s.wz, s.vx, fmaf(s.wx, s.vz, fmaf(FyB, V.invM, gBy)));
    const float dvz = fmaf(s.wy, s.vx, fmaf(-s.wx, s.vy, fmaf(FzB, V.invM, gBz)));
    const float dwx = fmaf(V.dJyz * s.wy, s.wz, Mx) * V.invJxx;
    const float dwy = fmaf(-V.dJxz * s.wx, s.wz, My) * V.invJyy;
    const float dwz = fmaf(V.dJxy * s.wx, s.wy, Mz) * V.invJzz;
    const float h = p.h;
    acc2(s.x, s.xl, h * dx);
    acc2(s.y, s.yl, h * dy);
    acc2(s.z, s.zl, h * dz);
    acc2(s.psi, s.psil, h * dpsi);
    s.th = fmaf(h, dth, s.th);
    s.ph = fmaf(h, dph, s.ph);
    acc2(s.vx, s.vxl, h * ax);
    acc2(s.vy, s.vyl, h * dvy);
    acc2(s.vz, s.vzl, h * dvz);
    s.wx = fmaf(h, dwx, s.wx);
    s.wy = fmaf(h, dwy, s.wy);
    s.wz = fmaf(h, dwz, s.wz);
    s.d = clampf(fmaf(h, dd, s.d), -V.dmax, V.dmax);
    return o;
}

// One Euler step backwards from the state s at its start: lam (13: x, y, z,
// psi, theta, phi, vx, vy, vz, wx, wy, wz, delta) is the adjoint of the state
// after the step on entry and of the state before it on exit; g_dd and g_ax
// receive the step's contributions to dJ/d(steering rate) and dJ/d(accel).
__device__ void step_adj(const GradParams &p, const St &s, float dd, float ax, float lam[13], float &g_dd,
                         float &g_ax, const Lane &ln)
{
    // the running cost enters the cost's adjoint only
    const float cw = p.objective == kGradCost ? 1.f : 0.f;
    const Veh &V = p.V;
    const Cost &Cc = p.C;
    const Terrain &T = p.T;
    const float h = p.h;
    float sps, cps, sth, cth, sph, cph, sd, cd;
    sincos_r(s.psi, sps, cps);
    sincos_r(s.th, sth, cth);
    sincos_r(s.ph, sph, cph);
    sincos_r(s.d, sd, cd);
    const float U = esm(V, s.ph, sph, cph, cth);
    float R[9];
    R[0] = cps * cth;
    R[1] = fmaf(cps * sph, sth, -cph * sps);
    R[2] = fmaf(cph * cps, sth, sph * sps);
    R[3] = cth * sps;
    R[4] = fmaf(sph * sps, sth, cph * cps);
    R[5] = fmaf(cph * sps, sth, -cps * sph);
    R[6] = -sth;
    R[7] = cth * sph;
    R[8] = cph * cth;
    int icx, icy;
    float fcx, fcy;
    cell_split(s.x, s.xl, T.inv_cell, icx, fcx);
    cell_split(s.y, s.yl, T.inv_cell, icy, fcy);
    const float vx = s.vx, vy = s.vy, vz = s.vz, wx = s.wx, wy = s.wy, wz = s.wz;
    WF w;
    wheel_fwd(V, T, R, icx, fcx, icy, fcy, s.z, s.zl, vx, vy, vz, wx, wy, wz, ln.rx, ln.ry, ln.k, ln.b, ln.Fs,
              ln.front ? s.d : 0.f, w);
    const float soft = fmaxf(fmaf(-U, Cc.inv_eps, 1.f), 0.f);
    const float ic = rcp(cth);
    const float wsc = fmaf(sph, wy, cph * wz);
    const float dd_next = fmaf(h, dd, s.d);
    const bool d_clamped = dd_next < -V.dmax || dd_next > V.dmax;

    Adj ad;
#pragma unroll
    for (int c = 0; c < 9; ++c) ad.R[c] = 0.f;
    // Euler update: state' = state + h * rate
    ad.x = lam[0];
    ad.y = lam[1];
    ad.z = lam[2];
    float a_psi = lam[3], a_th = lam[4], a_ph = lam[5];
    ad.vx = lam[6];
    ad.vy = lam[7];
    ad.vz = lam[8];
    ad.wx = lam[9];
    ad.wy = lam[10];
    ad.wz = lam[11];
    float a_d = d_clamped ? 0.f : lam[12];
    const float a_dx = h * lam[0], a_dy = h * lam[1], a_dz = h * lam[2];
    const float a_dpsi = h * lam[3], a_dth = h * lam[4], a_dph = h * lam[5];
    g_ax += h * lam[6];
    const float a_dvy = h * lam[7], a_dvz = h * lam[8];
    const float a_dwx = h * lam[9], a_dwy = h * lam[10], a_dwz = h * lam[11];
    if (!d_clamped) g_dd += h * lam[12];
    // running cost: J += h L, L = wt + wc dd^2 + sigma soft^2 + sum of costmap
    g_dd += cw * (h * 2.f * Cc.wc * dd);
    float a_U = 0.f;
    if (soft > 0.f) a_U = cw * (-h * 2.f * Cc.sigma * soft * Cc.inv_eps);
    const float a_csum = cw * h;
    // positions: d(x,y,z) = R v
    float a_sph = 0.f, a_cph = 0.f, a_sth = 0.f, a_cth = 0.f, a_sps = 0.f, a_cps = 0.f;
    ad.R[0] += a_dx * vx; ad.R[1] += a_dx * vy; ad.R[2] += a_dx * vz;
    ad.R[3] += a_dy * vx; ad.R[4] += a_dy * vy; ad.R[5] += a_dy * vz;
    ad.R[6] += a_dz * vx; ad.R[7] += a_dz * vy; ad.R[8] += a_dz * vz;
    ad.vx += a_dx * R[0] + a_dy * R[3] + a_dz * R[6];
    ad.vy += a_dx * R[1] + a_dy * R[4] + a_dz * R[7];
    ad.vz += a_dx * R[2] + a_dy * R[5] + a_dz * R[8];
    // Euler-angle rates
    const float a_wsc = a_dpsi * ic + a_dph * sth * ic;
    const float a_ic = a_dpsi * wsc + a_dph * wsc * sth;
    a_sth += a_dph * wsc * ic;
    ad.wx += a_dph;
    a_cph += a_dth * wy;
    ad.wy += a_dth * cph;
    a_sph -= a_dth * wz;
    ad.wz -= a_dth * sph;
    a_sph += a_wsc * wy;
    ad.wy += a_wsc * sph;
    a_cph += a_wsc * wz;
    ad.wz += a_wsc * cph;
    a_cth -= a_ic * ic * ic;
    // velocity rates
    const float a_FyB0 = a_dvy * V.invM;
    const float a_gBy = a_dvy;
    ad.wx += a_dvy * vz;
    ad.vz += a_dvy * wx;
    ad.wz -= a_dvy * vx;
    ad.vx -= a_dvy * wz;
    const float a_FzB = a_dvz * V.invM;
    const float a_gBz = a_dvz;
    ad.wx -= a_dvz * vy;
    ad.vy -= a_dvz * wx;
    ad.wy += a_dvz * vx;
    ad.vx += a_dvz * wy;
    // angular rates (Euler's equations)
    const float a_Mx = a_dwx * V.invJxx, a_My = a_dwy * V.invJyy, a_Mz = a_dwz * V.invJzz;
    ad.wy += a_Mx * V.dJyz * wz;
    ad.wz += a_Mx * V.dJyz * wy;
    ad.wx -= a_My * V.dJxz * wz;
    ad.wz -= a_My * V.dJxz * wx;
    ad.wx += a_Mz * V.dJxy * wy;
    ad.wy += a_Mz * V.dJxy * wx;
    // rear longitudinal constraint force, which enters My only
    const float a_Fx = -2.f * V.hR * a_My;
    g_ax += a_Fx * V.halfM;
    float a_gBx = -a_Fx * V.halfM;
    ad.wy += a_Fx * V.halfM * vz;
    ad.vz += a_Fx * V.halfM * wy;
    ad.wz -= a_Fx * V.halfM * vy;
    ad.vy -= a_Fx * V.halfM * wz;
    // sums: FyB = sum fy, Mx = hR FyB + sum ry Fz, My = sum -rx Fz (+ the
    // constraint force), Mz = sum rx fy, with fy = Fy cos(delta) in front
    const float a_FyB = a_FyB0 + V.hR * a_Mx;
    const float a_fy = a_FyB + ln.rx * a_Mz;
    const float aFy = ln.front ? a_fy * cd : a_fy;
    const float aFz = a_FzB + ln.ry * a_Mx - ln.rx * a_My;
    // gravity in B
    ad.R[6] -= V.g * a_gBx;
    ad.R[7] -= V.g * a_gBy;
    ad.R[8] -= V.g * a_gBz;
    // this lane's wheel into its own accumulator, then the quad's sum
    Adj aw;
#pragma unroll
    for (int c = 0; c < 9; ++c) aw.R[c] = 0.f;
    aw.x = aw.y = aw.z = aw.vx = aw.vy = aw.vz = aw.wx = aw.wy = aw.wz = aw.d = 0.f;
    float a_dw = ln.front ? -sd * a_fy * w.Fy : 0.f;                // cos(delta) of the front forces
    wheel_adj(V, T, R, wx, wy, ln.rx, ln.ry, ln.k, ln.b, ln.front ? 1.f : 0.f, w, aFz, aFy, a_csum, aw, a_dw);
#pragma unroll
    for (int c = 0; c < 9; ++c) ad.R[c] += qsum(aw.R[c], ln.mask);
    ad.x += qsum(aw.x, ln.mask);
    ad.y += qsum(aw.y, ln.mask);
    ad.z += qsum(aw.z, ln.mask);
    ad.vx += qsum(aw.vx, ln.mask);
    ad.vy += qsum(aw.vy, ln.mask);
    ad.vz += qsum(aw.vz, ln.mask);
    ad.wx += qsum(aw.wx, ln.mask);
    ad.wy += qsum(aw.wy, ln.mask);
    ad.wz += qsum(aw.wz, ln.mask);
    a_d += qsum(a_dw, ln.mask);
    // ESM: U = +/- M g Rbar (1 - (sin|phi| cos phibar + cos phi sin phibar)) cos theta
    {
        const float sg = fabsf(s.ph) < V.tip ? 1.f : -1.f;
        const float sabs = s.ph < 0.f ? -sph : sph;
        const float sv = fmaf(sabs, V.cpb, cph * V.spb);
        const float a_u = sg * a_U;
        const float a_s = -V.MgRbar * cth * a_u;
        a_cth += V.MgRbar * (1.f - sv) * a_u;
        a_sph += (s.ph < 0.f ? -1.f : 1.f) * a_s * V.cpb;
        a_cph += a_s * V.spb;
    }
    // rotation matrix
    const float *aR = ad.R;
    a_cps += aR[0] * cth + aR[1] * sph * sth + aR[2] * cph * sth + aR[4] * cph - aR[5] * sph;
    a_cth += aR[0] * cps + aR[3] * sps + aR[7] * sph + aR[8] * cph;
    a_sph += aR[1] * cps * sth + aR[2] * sps + aR[4] * sps * sth - aR[5] * cps + aR[7] * cth;
    a_sth += aR[1] * cps * sph + aR[2] * cph * cps + aR[4] * sph * sps + aR[5] * cph * sps - aR[6];
    a_cph += -aR[1] * sps + aR[2] * cps * sth + aR[4] * cps + aR[5] * sps * sth + aR[8] * cth;
    a_sps += -aR[1] * cph + aR[2] * sph + aR[3] * cth + aR[4] * sph * sth + aR[5] * cph * sth;
    // angles
    a_psi += a_sps * cps - a_cps * sps;
    a_th += a_sth * cth - a_cth * sth;
    a_ph += a_sph * cph - a_cph * sph;
    lam[0] = ad.x;
    lam[1] = ad.y;
    lam[2] = ad.z;
    lam[3] = a_psi;
    lam[4] = a_th;
    lam[5] = a_ph;
    lam[6] = ad.vx;
    lam[7] = ad.vy;
    lam[8] = ad.vz;
    lam[9] = ad.wx;
    lam[10] = ad.wy;
    lam[11] = ad.wz;
    lam[12] = a_d;
}

// U_ESM of a state (Sec. IV-B), as the plan kernel evaluates it
__device__ __forceinline__ float state_esm(const Veh &V, const St &s)
{
    float sth, cth, sph, cph;
    sincos_r(s.th, sth, cth);
    sincos_r(s.ph, sph, cph);
    return esm(V, s.ph, sph, cph, cth);
}

// lam += dU_ESM/d(state) at the state s: U = +/- M g Rbar (1 - (sin|phi|
// cos phibar + cos phi sin phibar)) cos theta depends on theta and phi only
__device__ __forceinline__ void esm_adj(const Veh &V, const St &s, float lam[13])
{
    float sth, cth, sph, cph;
    sincos_r(s.th, sth, cth);
    sincos_r(s.ph, sph, cph);
    const float sg = fabsf(s.ph) < V.tip ? 1.f : -1.f;
    const float sabs = s.ph < 0.f ? -sph : sph;
    const float sv = fmaf(sabs, V.cpb, cph * V.spb);
    const float a_s = -V.MgRbar * cth * sg;
    const float a_cth = V.MgRbar * (1.f - sv) * sg;
    const float a_sph = (s.ph < 0.f ? -1.f : 1.f) * a_s * V.cpb;
    const float a_cph = a_s * V.spb;
    lam[4] -= a_cth * sth;
    lam[5] += a_sph * cph - a_cph * sph;
}

// The forward pass stores the checkpoints and the last segment's Euler-step
// start states.  Then round i walks segment n_seg - 1 - i backwards and
// recomputes the segment before it.
//   SPLIT = false: one quad per candidate walks, then recomputes into the
//   buffer it has just read (one buffer).
//   SPLIT = true (a grid that leaves most of the GPU idle): each CTA holds
//   its kGradCands candidates twice.  Its first half of threads walks, its
//   second half recomputes, both having run the forward pass (the same
//   bits), so the recomputation runs beside the walk instead of before it,
//   into the other of two buffers.  A CTA barrier ends each round; every
//   thread, a candidate-less one included, passes the same number of
//   barriers (n_seg, uniform over the grid).
template <bool SPLIT>
__global__ void __launch_bounds__(SPLIT ? 2 * kGradHalf : kGradHalf, 1) grad_kernel(const __grid_constant__ GradParams p)
{
    const bool walker = !SPLIT || threadIdx.x < kGradHalf;
    const bool recomp = !SPLIT || !walker;
    const int tid = blockIdx.x * kGradHalf + (threadIdx.x & (kGradHalf - 1));   // lane slot, either half
    const int j = tid / kGradLanes;
    const bool active = j < p.K;                // whole quads, in both halves alike
    const Lane ln = lane_of(p.V, tid & (kGradLanes - 1), 0xfu << (threadIdx.x & 28));
    const Terrain &T = p.T;
    const Cost &Cc = p.C;
    const size_t K = (size_t)p.K;
    const size_t KL = K * kGradLanes;           // every lane keeps its own copy of the states
    const int n_seg = (p.H + p.ckpt - 1) / p.ckpt;
    const int k_last = (n_seg - 1) * p.ckpt;    // first control step of the last segment
    const size_t seg_stride = (size_t)p.ckpt * p.n_sub * kStFloats * KL;
    float *ck = p.ckpt_buf + tid;               // [n_seg][20][K lanes]
    float *seg = p.seg_buf + tid;               // [1 or 2][ckpt * n_sub][20][K lanes]
    const bool want_margin = p.objective == kGradMargin;
    St s;
    float J = 0.f;
    float Umin = CUDART_INF_F;                   // the margin: min U_ESM over the states
    int emin = 0;                                // index of the state holding it (first on ties)
    int done_step = p.H * p.n_sub;               // Euler step index where the goal stopped the rollout
    float lam[13];
#pragma unroll
    for (int c = 0; c < 13; ++c) lam[c] = 0.f;
    if (active) {
        {
            float q[13];
            if (p.x0_soa) {
#pragma unroll
                for (int c = 0; c < 13; ++c) q[c] = p.x0_soa[c * K + j];
            } else {
#pragma unroll
                for (int c = 0; c < 13; ++c) q[c] = p.x0[c];
            }
            two_sum(q[0], -T.x0_hi, s.x, s.xl);
            s.xl -= T.x0_lo;
            two_sum(q[1], -T.y0_hi, s.y, s.yl);
            s.yl -= T.y0_lo;
            s.z = q[2]; s.psi = q[3]; s.th = q[4]; s.ph = q[5];
            s.vx = q[6]; s.vy = q[7]; s.vz = q[8];
            s.wx = q[9]; s.wy = q[10]; s.wz = q[11]; s.d = q[12];
            s.zl = s.psil = s.vxl = s.vyl = s.vzl = 0.f;
        }
        // forward: cost (or margin), checkpoints and the last segment's states
        bool done = false;
        for (int k = 0; k < p.H; ++k) {
            if (recomp && k % p.ckpt == 0) st_store(ck + (size_t)(k / p.ckpt) * kStFloats * KL, KL, s);
            const float2 u = __ldg(p.ctrl + (size_t)k * K + j);
            const float dd = clampf(u.x, -p.V.ddmax, p.V.ddmax);
            for (int q = 0; q < p.n_sub && !done; ++q) {
                if (recomp && k >= k_last)
                    st_store(seg + (size_t)((k - k_last) * p.n_sub + q) * kStFloats * KL, KL, s);
                if (want_margin) {
                    const float U = state_esm(p.V, s);
                    if (U < Umin) {
                        Umin = U;
                        emin = k * p.n_sub + q;
                    }
                }
                const StepOut o = step_fwd(p, s, dd, u.y, ln);
                if (!o.stepped) {
                    done = true;
                    done_step = k * p.n_sub + q;
                    break;
                }
                J = fmaf(p.h, o.L, J);
            }
        }
        // terminal cost and its gradient, or the final state's share of the margin
        if (walker) {
            if (want_margin) {
                const int e_final = done ? done_step : p.H * p.n_sub;
                const float U = state_esm(p.V, s);
                if (U < Umin) {
                    Umin = U;
                    emin = e_final;
                }
                if (emin == e_final) esm_adj(p.V, s, lam);
                if (ln.q == 0) p.cost[j] = Umin;
            } else {
                const float gdx = (s.x - Cc.gx_hi) + (s.xl - Cc.gx_lo);
                const float gdy = (s.y - Cc.gy_hi) + (s.yl - Cc.gy_lo);
                const float dist = sqrtf(fmaf(gdx, gdx, gdy * gdy));
                J = fmaf(Cc.wg, dist, J);
                if (ln.q == 0) p.cost[j] = J;
                if (dist > 0.f) {
                    lam[0] = Cc.wg * gdx / dist;
                    lam[1] = Cc.wg * gdy / dist;
                }
            }
        }
    }
    if (SPLIT) __syncthreads();                 // the last segment's states are stored
    // reverse: round i walks segment n_seg - 1 - i and recomputes the one before it
    for (int i = 0; i < n_seg; ++i) {
        const int sw = n_seg - 1 - i;
        if (active && walker) {
            const int k0 = sw * p.ckpt, k1 = min(p.H, k0 + p.ckpt);
            const float *buf = SPLIT ? seg + (size_t)(i & 1) * seg_stride : seg;
            for (int k = k1 - 1; k >= k0; --k) {
                const float2 u = __ldg(p.ctrl + (size_t)k * K + j);
                const bool inside = !(u.x < -p.V.ddmax || u.x > p.V.ddmax);   // as the clamp
                const float dd = clampf(u.x, -p.V.ddmax, p.V.ddmax);
                float g_dd = 0.f, g_ax = 0.f;
                for (int q = p.n_sub - 1; q >= 0; --q) {
                    const int e = k * p.n_sub + q;
                    if (e >= done_step) continue;
                    St r2;
                    st_load(buf + (size_t)(e - k0 * p.n_sub) * kStFloats * KL, KL, r2);
                    step_adj(p, r2, dd, u.y, lam, g_dd, g_ax, ln);
                    // lam is now the adjoint of the step's start state
                    if (want_margin && e == emin) esm_adj(p.V, r2, lam);
                }
                // the steering rate is clamped to +/- its limit before use
                if (ln.q == 0) {
                    p.grad[((size_t)k * K + j) * 2] = inside ? g_dd : 0.f;
                    p.grad[((size_t)k * K + j) * 2 + 1] = g_ax;
                }
            }
        }
        if (active && recomp && sw > 0) {
            // recompute segment sw - 1's Euler-step start states
            const int sr = sw - 1;
            const int k0 = sr * p.ckpt, k1 = k0 + p.ckpt;                 // never the last segment
            float *buf = SPLIT ? seg + (size_t)((i + 1) & 1) * seg_stride : seg;
            St r;
            st_load(ck + (size_t)sr * kStFloats * KL, KL, r);
            int n_steps = 0;
            for (int k = k0; k < k1; ++k) {
                const float2 u = __ldg(p.ctrl + (size_t)k * K + j);
                const float dd = clampf(u.x, -p.V.ddmax, p.V.ddmax);
                for (int q = 0; q < p.n_sub; ++q) {
                    const int e = k * p.n_sub + q;
                    if (e >= done_step) break;
                    st_store(buf + (size_t)n_steps * kStFloats * KL, KL, r);
                    ++n_steps;
                    step_fwd(p, r, dd, u.y, ln);
                }
            }
        }
        if (SPLIT && i + 1 < n_seg) __syncthreads();   // segment sw - 1 is stored; segment sw is read
    }
}

}  // namespace

int grad_split_ctas(int device)
{
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_kernel<true>, 2 * kGradHalf, 0) !=
        cudaSuccess)
        return 0;
    return sms * per_sm;
}

cudaError_t launch_grad(const GradParams &p, cudaStream_t stream)
{
    const unsigned blocks = (unsigned)((p.K + kGradCands - 1) / kGradCands);
    if (p.split)
        grad_kernel<true><<<blocks, 2 * kGradHalf, 0, stream>>>(p);
    else
        grad_kernel<false><<<blocks, kGradHalf, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace atp
