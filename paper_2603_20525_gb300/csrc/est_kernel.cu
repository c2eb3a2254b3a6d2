// est_kernel.cu - fused rollout, cost, lateral-acceleration margin and
// empirical argmin of the planar extended single-track (EST) model of arxiv
// 2603.20525 (App. "Extended Single-Track Vehicle Dynamics Model", Sec. IV-C),
// the formulation the paper sets beside the SRB model.
//
// One thread per candidate (the model has 7 states and one terrain lookup
// under the CoM per Euler step, plus four costmap lookups at the wheels when
// the terrain carries a costmap, reading Q17).  Pitch and roll are not states: they follow
// the terrain's normal under the CoM, whose components give their sines and
// cosines directly (1-2-3 convention), so the step needs two trigonometric
// evaluations (yaw and steering) and two arctangents (the virtual tires'
// slip).  The same FP32 conventions as the SRB kernel: explicit FMAs only,
// compensated sums for position, heading and velocity, positions relative to
// the terrain origin.  The reduction is the SRB kernel's fused tail.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "est_kernel.cuh"
#include "plan_tail.cuh"

namespace atp {

namespace {

// Costmap value at the point (cell icx + fcx + ox / cell, ...): bilinear over
// the texels' cost channel; sets `off` for a query outside the map.
template <int TEX>
__device__ __forceinline__ float cost_at(const Terrain &T, int icx, float fcx, int icy, float fcy, float ox,
                                         float oy, bool &off)
{
    float a, b;
    const int i = axis(icx, fcx, ox, T.inv_cell, T.nx, a, off);
    const int j = axis(icy, fcy, oy, T.inv_cell, T.ny, b, off);
    return bilerp<TEX>(T, i, j, a, b).w;
}

__device__ __forceinline__ float tire(const Veh &V, float Fz, float alpha)
{
    const float Ca = V.C * alpha;
    return Fz * (-Ca * V.mu) * rsq(fmaf(Ca, Ca, V.mu2));
}

template <bool PER_X0, int TEX>
__device__ __forceinline__ void est_one(const PlanParams &p, int j, float &J, float &margin, bool &feasible)
{
    const Veh &V = p.V;
    const Cost &Cc = p.C;
    const Terrain &T = p.T;
    // state x, y, psi, v_By, w_Bz, delta, v_Bx; x, y relative to the origin;
    // *_l the low parts of the compensated components
    float x, xl, y, yl, psi, psil = 0.f, vy, vyl = 0.f, wz, d, vx, vxl = 0.f;
    {
        float s[7];
        if (PER_X0) {
#pragma unroll
            for (int c = 0; c < 7; ++c) s[c] = p.x0_soa[(size_t)c * p.N + j];
        } else {
#pragma unroll
            for (int c = 0; c < 7; ++c) s[c] = p.x0[c];
        }
        two_sum(s[0], -T.x0_hi, x, xl);
        xl -= T.x0_lo;
        two_sum(s[1], -T.y0_hi, y, yl);
        yl -= T.y0_lo;
        psi = s[2]; vy = s[3]; wz = s[4]; d = s[5]; vx = s[6];
    }
    // wheel contact points in B (fl, fr, rl, rr): (+-L, +-e/2, -(h+R))
    bool done = false, off = false;
    const float h = p.h;
    const bool cm = T.has_cm != 0;
    double J64 = 0.0;
    float msm = CUDART_INF_F;      // smallest per-step margin so far and its control step
    int mstep = 0;
    // each interval's control is loaded one interval ahead, so the load's
    // latency overlaps the Euler steps
    float2 un = p.H > 0 ? __ldg(p.ctrl + j) : make_float2(0.f, 0.f);
    for (int k = 0; k < p.H; ++k) {
        const float2 u = un;
        if (k + 1 < p.H) un = __ldg(p.ctrl + (size_t)(k + 1) * p.N + j);
        const float dd = clamp_keep_nan(u.x, -V.ddmax, V.ddmax);
        const float ax = u.y;
        float sm = CUDART_INF_F;
        for (int sub = 0; sub < p.n_sub; ++sub) {
            if (done) continue;            // frozen at the goal
            const float gdx = (x - Cc.gx_hi) + (xl - Cc.gx_lo);
            const float gdy = (y - Cc.gy_hi) + (yl - Cc.gy_lo);
            if (fmaf(gdx, gdx, gdy * gdy) <= Cc.goal_r2) {
                done = true;
                continue;
            }
            // terrain under the CoM and its unit normal (reading Q1)
            int icx, icy;
            float fcx, fcy, a, b;
            cell_split(x, xl, T.inv_cell, icx, fcx);
            cell_split(y, yl, T.inv_cell, icy, fcy);
            const int ti = axis(icx, fcx, 0.f, T.inv_cell, T.nx, a, off);
            const int tj = axis(icy, fcy, 0.f, T.inv_cell, T.ny, b, off);
            const float4 t = bilerp<TEX>(T, ti, tj, a, b);
            const float rn = rsq(fmaf(t.y, t.y, fmaf(t.z, t.z, 1.f)));
            const float tx = -t.y * rn, ty = -t.z * rn, tz = rn;
            // 1-2-3 angles of the plane: sin(theta) = tau_x, cos(theta) =
            // |(tau_y, tau_z)|, sin(phi) = -tau_y / cos(theta), cos(phi) = tau_z / cos(theta)
            const float sth = tx;
            const float cth = sqrtf(fmaf(ty, ty, tz * tz));
            const float ict = rcp(cth);
            const float sph = -ty * ict, cph = tz * ict;
            float sps, cps, sd, cd;
            sincos_r(psi, sps, cps);
            sincos_r(d, sd, cd);
            // rotation body -> world (rows 0 and 1, and the third row's gravity)
            const float R00 = cth * cps, R01 = -cth * sps, R02 = sth;
            const float R10 = fmaf(cps * sph, sth, cph * sps);
            const float R11 = fmaf(-sph * sth, sps, cph * cps);
            const float R12 = -cth * sph;
            const float R21 = fmaf(cph * sth, sps, cps * sph);
            const float R22 = cph * cth;
            const float gBy = -V.g * R21, gBz = -V.g * R22;
            // virtual tires: normal forces with longitudinal load transfer, slip, force
            const float aBx = fmaf(-wz, vy, ax);
            const float Fzf = fmaf(-V.Kzzf, gBz, -V.Kzx * aBx);
            const float Fzr = fmaf(-V.Kzzr, gBz, V.Kzx * aBx);
            const float af = atan2_r(fmaf(wz, V.Lf, vy), vx) - d;
            const float ar = atan2_r(fmaf(-wz, V.Lr, vy), vx);
            const float Fyf = tire(V, Fzf, af);
            const float Fyr = tire(V, Fzr, ar);
            // A(xi) + B zeta
            const float dx = fmaf(R01, vy, R00 * vx);
            const float dy = fmaf(R11, vy, R10 * vx);
            const float dvy = fmaf(-wz, vx, fmaf(Fyf + Fyr, V.invM, gBy));
            const float dwz = fmaf(Fyf * V.Lf, cd, -Fyr * V.Lr) * V.invJzz;
            // lateral-acceleration constraint |a_By - g_By| < abar (Sec. IV-C)
            const float aBy = fmaf(wz, vx, dvy);
            const float m = V.abar - fabsf(aBy - gBy);
            margin = fminf(margin, m);
            sm = fminf(sm, m);
            // distance constraints: the costmap at the four contact points,
            // read only when the terrain has one (reading Q17)
            float csum = 0.f;
            if (cm) {
                const float ofx = fmaf(R02, -V.hR, R00 * V.Lf), ofy = fmaf(R12, -V.hR, R10 * V.Lf);
                const float orx = fmaf(R02, -V.hR, -R00 * V.Lr), ory = fmaf(R12, -V.hR, -R10 * V.Lr);
                const float lx = R01 * V.he, ly = R11 * V.he;
                const float cfl = cost_at<TEX>(T, icx, fcx, icy, fcy, ofx + lx, ofy + ly, off);
                const float cfr = cost_at<TEX>(T, icx, fcx, icy, fcy, ofx - lx, ofy - ly, off);
                const float crl = cost_at<TEX>(T, icx, fcx, icy, fcy, orx + lx, ory + ly, off);
                const float crr = cost_at<TEX>(T, icx, fcx, icy, fcy, orx - lx, ory - ly, off);
                csum = (cfl + cfr) + (crl + crr);
            }
            const float soft = fmaxf(fmaf(-m, Cc.inv_eps, 1.f), 0.f);
            const float L = fmaf(Cc.sigma * soft, soft, fmaf(Cc.wc * dd, dd, Cc.wt)) + csum;
            if (p.acc64) J64 += (double)(h * L);
            else J = fmaf(h, L, J);
            // forward Euler, steering angle clamped (reading Q5)
            acc2(x, xl, h * dx);
            acc2(y, yl, h * dy);
            acc2(psi, psil, h * wz);
            acc2(vy, vyl, h * dvy);
            wz = fmaf(h, dwz, wz);
            d = clamp_keep_nan(fmaf(h, dd, d), -V.dmax, V.dmax);
            acc2(vx, vxl, h * ax);
        }
        if (p.step_margin) p.step_margin[(size_t)k * p.N + j] = sm;
        if (sm < msm) {
            msm = sm;
            mstep = k;
        }
    }
    // final state: goal test and terminal cost Phi (Sec. IV-C)
    {
        const float gdx = (x - Cc.gx_hi) + (xl - Cc.gx_lo);
        const float gdy = (y - Cc.gy_hi) + (yl - Cc.gy_lo);
        const float d2 = fmaf(gdx, gdx, gdy * gdy);
        if (!done && d2 <= Cc.goal_r2) done = true;
        if (p.acc64) J = (float)(J64 + (double)(Cc.wg * sqrtf(d2)));
        else J = fmaf(Cc.wg, sqrtf(d2), J);
    }
    const float xs[7] = {(x + T.x0_hi) + (xl + T.x0_lo), (y + T.y0_hi) + (yl + T.y0_lo), psi + psil,
                         vy + vyl, wz, d, vx + vxl};
    bool finite = isfinite(J);
#pragma unroll
    for (int c = 0; c < 7; ++c) finite = finite && isfinite(xs[c]);
    if (!finite) J = CUDART_INF_F;
    feasible = finite && margin > 0.f;
    const uint8_t fl = (feasible ? ATP_FLAG_FEASIBLE : 0) | (done ? ATP_FLAG_DONE : 0) |
                       (off ? ATP_FLAG_OFFMAP : 0) | (finite ? 0 : ATP_FLAG_NONFINITE);
    if (p.cost) p.cost[j] = J;
    if (p.margin) p.margin[j] = margin;
    if (p.flags) p.flags[j] = fl;
    if (p.min_step) p.min_step[j] = mstep;
    if (p.xf) {
#pragma unroll
        for (int c = 0; c < 7; ++c) p.xf[(size_t)c * p.N + j] = xs[c];
    }
}

template <bool PER_X0, bool REDUCE, int TEX>
__global__ void __launch_bounds__(kPlanBlock) est_kernel(const __grid_constant__ PlanParams p)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < p.N;
    float J = 0.f, margin = CUDART_INF_F;
    bool feasible = false;
    if (live) est_one<PER_X0, TEX>(p, j, J, margin, feasible);
    if (!REDUCE) return;
    plan_tail(p, j, live, J, feasible, gridDim.x);
}

template <int TEX>
cudaError_t launch_tex(const PlanParams &p, bool reduce, cudaStream_t stream)
{
    const dim3 grid((unsigned)(((size_t)p.N + kPlanBlock - 1) / kPlanBlock));
    const bool per = p.x0_soa != nullptr;
    if (reduce) {
        if (per) est_kernel<true, true, TEX><<<grid, kPlanBlock, 0, stream>>>(p);
        else est_kernel<false, true, TEX><<<grid, kPlanBlock, 0, stream>>>(p);
    } else {
        if (per) est_kernel<true, false, TEX><<<grid, kPlanBlock, 0, stream>>>(p);
        else est_kernel<false, false, TEX><<<grid, kPlanBlock, 0, stream>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_est(const PlanParams &p, bool reduce, cudaStream_t stream)
{
    return p.tex_format == TEX_F32 ? launch_tex<TEX_F32>(p, reduce, stream)
                                   : launch_tex<TEX_BF16>(p, reduce, stream);
}

}  // namespace atp
