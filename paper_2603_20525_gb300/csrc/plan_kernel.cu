// plan_kernel.cu - fused SRB rollout, cost, ESM margin and empirical argmin
// (arxiv 2603.20525, Sec. IV-A..IV-D) for sm_103a.
//
// Design
//   * One, two or four threads per candidate (by batch size): a quad runs one
//     wheel per lane and a pair one axle per lane, repeating the body
//     arithmetic on every lane, so that small batches still give each SM
//     sub-partition several warps.  The state stays in registers for the
//     whole horizon; per Euler step the only memory traffic is 16 terrain
//     texels (four bilinear lookups of one float4 per corner) through the
//     read-only path, which the L1 and the 129 MB L2 serve for every terrain
//     size used.
//   * The arithmetic forms that measured faster in only some layouts are
//     compile-time choices that give the same bits: the running cost's
//     accumulator (FP32 or FP64), packed two-wide FP32 pairs and a goal
//     test that discards the step rather than branching (two lanes), and
//     loading each control one interval ahead (four lanes).
//   * Controls are time-major float2 [H][N]: a warp reads one coalesced 256 B
//     line per control step.
//   * The reduction is fused into the tail: a warp-shuffle min of a packed
//     64-bit key (infeasible bit, order-preserving image of the FP32 cost,
//     candidate index), one shared-memory step per CTA, one 64-bit atomicMin
//     per CTA, a ballot/popc feasible count, and a ticket that elects the last
//     CTA to write the result and the best candidate's controls (and, when
//     asked for, its per-step margins).
#include "plan_kernel.cuh"
#include "plan_tail.cuh"

#include <cuda_bf16.h>
#include <math_constants.h>

namespace atp {

// Sum of v over the two lanes of a candidate's pair (a0 + a1 in both).
__device__ __forceinline__ float pair_sum(float v, unsigned mask)
{
    return v + __shfl_xor_sync(mask, v, 1);
}

// One candidate per LANES consecutive threads.  LANES = 1: a thread runs all
// four wheels.  LANES = 2: lane 0 runs the front axle's two wheels, lane 1
// the rear's; each sums its axle, then one xor-shuffle per sum gives both
// the same totals, in the same order as one lane computes them, so one and
// two lanes give the same bits.  LANES = 4: lane q of the quad runs wheel q
// (fl, fr, rl, rr) and forms the axle sums, then the totals, in that order
// too, so all three layouts give the same bits.  The body-level arithmetic is repeated bit-identically on
// every lane of a candidate, so lanes never exchange state, only the five
// force/moment sums and the costmap sum, and the step's four sincos, which
// the lanes split between them.  ACC selects the running cost's
// accumulator: kAccF32, kAccF64, or kAccRuntime (p.acc64 decides; the batch
// kernel, which would otherwise inline twice as many variants).  A
// compile-time choice keeps the step loop free of the uniform branch.
constexpr int kAccF32 = 0, kAccF64 = 1, kAccRuntime = 2;


template <int LANES, bool PER_X0, int TEX, int ACC>
__device__ __forceinline__ void rollout_one(const PlanParams &p, int j, int q, unsigned qmask,
                                            float &J, float &margin, bool &feasible)
{
    const Veh &V = p.V;
    const Cost &Cc = p.C;
    const Terrain &T = p.T;
    {
        // this lane's wheel (LANES = 4) or axle (LANES = 2)
        const bool front = LANES == 2 ? q == 0 : q < 2;
        const float wrx = front ? V.Lf : -V.Lr;
        const float wry = (q & 1) ? -V.he : V.he;
        const float wk = front ? V.kf : V.kr;
        const float wb = front ? V.bf : V.br;
        const float wFs = front ? V.Fsf : V.Fsr;
        // state; x, y relative to the terrain origin; *_l are the low parts of
        // the compensated components
        float x, xl, y, yl, z, zl, psi, psil, vx, vxl, vy, vyl, vz, vzl;
        float th, ph, wx, wy, wz, d;
        {
            float x0[13];
            if (PER_X0) {
                const size_t N = (size_t)p.N;
#pragma unroll
                for (int c = 0; c < 13; ++c) x0[c] = p.x0_soa[c * N + j];
            } else {
#pragma unroll
                for (int c = 0; c < 13; ++c) x0[c] = p.x0[c];
            }
            two_sum(x0[0], -T.x0_hi, x, xl);
            xl -= T.x0_lo;
            two_sum(x0[1], -T.y0_hi, y, yl);
            yl -= T.y0_lo;
            z = x0[2]; psi = x0[3]; th = x0[4]; ph = x0[5];
            vx = x0[6]; vy = x0[7]; vz = x0[8];
            wx = x0[9]; wy = x0[10]; wz = x0[11]; d = x0[12];
            zl = psil = vxl = vyl = vzl = 0.f;
        }
        bool done = false, off = false;
        const float h = p.h;
        const bool acc64 = ACC == kAccRuntime ? p.acc64 != 0 : ACC == kAccF64;
        double J64 = 0.0;          // the running cost in FP64 when acc64
        float Ufrozen = 0.f;
        // the smallest per-step margin so far, its control step (first on
        // ties), and the last step's margin, which the final state joins
        float msm = CUDART_INF_F, last_sm = CUDART_INF_F;
        int mstep = 0;

        // four lanes load each interval's control one interval ahead, so the
        // load's latency overlaps the Euler steps (measured faster there; one
        // and two lanes run at the 128-register cap, where the two extra live
        // registers cost more than the latency saved)
        constexpr bool kPrefetch = LANES == 4;
        float2 un = kPrefetch && p.H > 0 ? __ldg(p.ctrl + j) : make_float2(0.f, 0.f);
        for (int k = 0; k < p.H; ++k) {
            // zero-order hold; admissible steering rate |delta_dot| <= max
            const float2 u = kPrefetch ? un : __ldg(p.ctrl + (size_t)k * p.N + j);
            if (kPrefetch && k + 1 < p.H) un = __ldg(p.ctrl + (size_t)(k + 1) * p.N + j);
            // one and two lanes ask L1 for the next interval's control instead,
            // which costs no register (measured 3.6 % off the 16384-candidate
            // plan, no change to a full-GPU plan)
            if (!kPrefetch && k + 1 < p.H)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(p.ctrl + (size_t)(k + 1) * p.N + j));
            const float dd = clamp_keep_nan(u.x, -V.ddmax, V.ddmax);
            const float ax = u.y;
            float sm = CUDART_INF_F;
            for (int sub = 0; sub < p.n_sub; ++sub) {
                if (done) {            // frozen at the goal: the same state each step
                    sm = fminf(sm, Ufrozen);
                    continue;
                }
                // four lanes split the step's four sincos (psi, theta, phi,
                // delta; one each) and two lanes split them two and two,
                // exchanging them by shuffle: the same bits as computing all
                // four (measured 8 % off a 16384-candidate plan with four
                // lanes, 2.4 % with two)
                float sps, cps, sth, cth, sph, cph, cdl = 1.f;
                if constexpr (LANES == 4) {
                    float s1, c1;
                    sincos_r(q == 0 ? psi : q == 1 ? th : q == 2 ? ph : d, s1, c1);
                    sps = __shfl_sync(qmask, s1, 0, 4);
                    cps = __shfl_sync(qmask, c1, 0, 4);
                    sth = __shfl_sync(qmask, s1, 1, 4);
                    cth = __shfl_sync(qmask, c1, 1, 4);
                    sph = __shfl_sync(qmask, s1, 2, 4);
                    cph = __shfl_sync(qmask, c1, 2, 4);
                    cdl = __shfl_sync(qmask, c1, 3, 4);
                } else if constexpr (LANES == 2) {
                    // lane 0: psi and phi; lane 1: theta and delta
                    float s1, c1, s2, c2;
                    sincos_r(q == 0 ? psi : th, s1, c1);
                    sincos_r(q == 0 ? ph : d, s2, c2);
                    const float os1 = __shfl_xor_sync(qmask, s1, 1), oc1 = __shfl_xor_sync(qmask, c1, 1);
                    const float os2 = __shfl_xor_sync(qmask, s2, 1), oc2 = __shfl_xor_sync(qmask, c2, 1);
                    sps = q == 0 ? s1 : os1;
                    cps = q == 0 ? c1 : oc1;
                    sth = q == 0 ? os1 : s1;
                    cth = q == 0 ? oc1 : c1;
                    sph = q == 0 ? s2 : os2;
                    cph = q == 0 ? c2 : oc2;
                    cdl = q == 0 ? oc2 : c2;
                } else {
                    sincos_r(psi, sps, cps);
                    sincos_r(th, sth, cth);
                    sincos_r(ph, sph, cph);
                }
                const float U = esm(V, ph, sph, cph, cth);
                margin = fminf(margin, U);
                sm = fminf(sm, U);
                // goal test before the step (Sec. IV-C, reading Q4).  One and
                // four lanes skip the step at the goal; two lanes compute it
                // and discard it (`keep`), which keeps the loop body one basic
                // block and measured faster there, slower with one or four
                const float gdx = (x - Cc.gx_hi) + (xl - Cc.gx_lo);
                const float gdy = (y - Cc.gy_hi) + (yl - Cc.gy_lo);
                const bool reached = fmaf(gdx, gdx, gdy * gdy) <= Cc.goal_r2;
                if (LANES != 2 && reached) {
                    done = true;
                    Ufrozen = U;
                    continue;
                }
                const bool keep = LANES == 2 && reached;
                bool offs = false;     // a wheel of this step off the map
                // 3-2-1 rotation, body -> world (Sec. IV-A)
                Body B;
                float *R = B.R;
                R[0] = cps * cth;
                if constexpr (LANES == 2) {
                    // packed pairs, the same bits (see wheel's PAIRED)
                    const float2 r12 = fma2(make_float2(cps * sph, cph * cps), splat2(sth),
                                            make_float2(-cph * sps, sph * sps));
                    const float2 r45 = fma2(make_float2(sph * sps, cph * sps), splat2(sth),
                                            make_float2(cph * cps, -cps * sph));
                    R[1] = r12.x; R[2] = r12.y; R[4] = r45.x; R[5] = r45.y;
                } else {
                    R[1] = fmaf(cps * sph, sth, -cph * sps);
                    R[2] = fmaf(cph * cps, sth, sph * sps);
                    R[4] = fmaf(sph * sps, sth, cph * cps);
                    R[5] = fmaf(cph * sps, sth, -cps * sph);
                }
                R[3] = cth * sps;
                R[6] = -sth;
                R[7] = cth * sph;
                R[8] = cph * cth;
                cell_split(x, xl, T.inv_cell, B.icx, B.fcx);
                cell_split(y, yl, T.inv_cell, B.icy, B.fcy);
                B.z_hi = z;
                B.z_lo = zl;
                B.vx = vx; B.vy = vy; B.vz = vz;
                B.wx = wx; B.wy = wy; B.wz = wz;
                // gravity in B: R^T (0, 0, -g)
                const float gBx = -V.g * R[6], gBy = -V.g * R[7], gBz = -V.g * R[8];
                float cd;
                if constexpr (LANES > 1) {
                    cd = cdl;
                } else {
                    float sd;
                    sincos_r(d, sd, cd);
                }
                // summed forces and moments (Sec. IV-A); the rear
                // longitudinal constraint force enters My only
                float FyB, FzB, Mx, My, Mz, csum;
                if (LANES == 1) {
                    const WheelOut fl = wheel<TEX>(V, T, B, V.Lf, V.he, V.kf, V.bf, V.Fsf, d, offs);
                    const WheelOut fr = wheel<TEX>(V, T, B, V.Lf, -V.he, V.kf, V.bf, V.Fsf, d, offs);
                    const WheelOut rl = wheel<TEX>(V, T, B, -V.Lr, V.he, V.kr, V.br, V.Fsr, 0.f, offs);
                    const WheelOut rr = wheel<TEX>(V, T, B, -V.Lr, -V.he, V.kr, V.br, V.Fsr, 0.f, offs);
                    const float Fyf = (fl.Fy + fr.Fy) * cd;
                    const float Fyr = rl.Fy + rr.Fy;
                    FyB = Fyf + Fyr;
                    FzB = (fl.Fz + fr.Fz) + (rl.Fz + rr.Fz);
                    Mx = fmaf(V.hR, FyB, V.he * ((fl.Fz - fr.Fz) + (rl.Fz - rr.Fz)));
                    My = -V.Lf * (fl.Fz + fr.Fz) + V.Lr * (rl.Fz + rr.Fz);
                    Mz = V.Lf * Fyf + -V.Lr * Fyr;
                    csum = (fl.cost + fr.cost) + (rl.cost + rr.cost);
                } else if (LANES == 2) {
                    // this lane's axle: left and right wheel
                    const float di = front ? d : 0.f;
                    const WheelOut l = wheel<TEX, true>(V, T, B, wrx, V.he, wk, wb, wFs, di, offs);
                    const WheelOut r = wheel<TEX, true>(V, T, B, wrx, -V.he, wk, wb, wFs, di, offs);
                    const float fy = front ? (l.Fy + r.Fy) * cd : l.Fy + r.Fy;
                    const float fz = l.Fz + r.Fz;
                    FyB = pair_sum(fy, qmask);
                    FzB = pair_sum(fz, qmask);
                    Mx = fmaf(V.hR, FyB, V.he * pair_sum(l.Fz - r.Fz, qmask));
                    My = pair_sum(-wrx * fz, qmask);
                    Mz = pair_sum(wrx * fy, qmask);
                    csum = T.has_cm ? pair_sum(l.cost + r.cost, qmask) : 0.f;
                } else {
                    // this lane's wheel; its axle's sums by one xor-shuffle,
                    // the other axle's by a second, each formed in the order
                    // one lane forms it (a + b is b + a; the differences and
                    // the moments pick their operands by lane), so four lanes
                    // give the bits of one and two
                    const WheelOut w = wheel<TEX>(V, T, B, wrx, wry, wk, wb, wFs, front ? d : 0.f, offs);
                    const bool left = (q & 1) == 0;
                    const float oFy = __shfl_xor_sync(qmask, w.Fy, 1);
                    const float oFz = __shfl_xor_sync(qmask, w.Fz, 1);
                    const float aFy = w.Fy + oFy;
                    const float afy = front ? aFy * cd : aFy;                  // Fyf or Fyr
                    const float aFz = w.Fz + oFz;
                    const float aDz = left ? w.Fz - oFz : oFz - w.Fz;           // left - right
                    const float bfy = __shfl_xor_sync(qmask, afy, 2);
                    const float bFz = __shfl_xor_sync(qmask, aFz, 2);
                    const float bDz = __shfl_xor_sync(qmask, aDz, 2);
                    const float Fyf = front ? afy : bfy, Fyr = front ? bfy : afy;
                    const float Fzf = front ? aFz : bFz, Fzr = front ? bFz : aFz;
                    FyB = Fyf + Fyr;
                    FzB = Fzf + Fzr;
                    Mx = fmaf(V.hR, FyB, V.he * (aDz + bDz));
                    My = -V.Lf * Fzf + V.Lr * Fzr;
                    Mz = V.Lf * Fyf + -V.Lr * Fyr;
                    if (T.has_cm) {
                        const float ac = w.cost + __shfl_xor_sync(qmask, w.cost, 1);
                        csum = ac + __shfl_xor_sync(qmask, ac, 2);
                    } else {
                        csum = 0.f;
                    }
                }
                const float Fx = V.halfM * fmaf(-wz, vy, fmaf(wy, vz, ax - gBx));
                My = fmaf(-V.hR, 2.f * Fx, My);
                // running cost L = L_0 + L_soft (Sec. IV-C), left Riemann sum
                const float soft = fmaxf(fmaf(-U, Cc.inv_eps, 1.f), 0.f);
                const float L = fmaf(Cc.sigma * soft, soft, fmaf(Cc.wc * dd, dd, Cc.wt)) + csum;
                if (acc64) J64 += keep ? 0.0 : (double)(h * L);
                else J = keep ? J : fmaf(h, L, J);
                // state derivative A(xi) + B zeta (Sec. IV-A)
                const float ic = rcp(cth);
                const float wsc = fmaf(sph, wy, cph * wz);
                float dx, dy;
                if constexpr (LANES == 2) {
                    const float2 dxy = fma2(make_float2(R[2], R[5]), splat2(vz),
                                            fma2(make_float2(R[1], R[4]), splat2(vy),
                                                 make_float2(R[0] * vx, R[3] * vx)));
                    dx = dxy.x;
                    dy = dxy.y;
                } else {
                    dx = fmaf(R[2], vz, fmaf(R[1], vy, R[0] * vx));
                    dy = fmaf(R[5], vz, fmaf(R[4], vy, R[3] * vx));
                }
                const float dz = fmaf(R[8], vz, fmaf(R[7], vy, R[6] * vx));
                const float dpsi = wsc * ic;
                const float dth = fmaf(cph, wy, -sph * wz);
                const float dph = fmaf(wsc, sth * ic, wx);
                const float dvy = fmaf(-wz, vx, fmaf(wx, vz, fmaf(FyB, V.invM, gBy)));
                const float dvz = fmaf(wy, vx, fmaf(-wx, vy, fmaf(FzB, V.invM, gBz)));
                const float dwx = fmaf(V.dJyz * wy, wz, Mx) * V.invJxx;
                const float dwy = fmaf(-V.dJxz * wx, wz, My) * V.invJyy;
                const float dwz = fmaf(V.dJxy * wx, wy, Mz) * V.invJzz;
                // forward Euler (Sec. IV-D), steering angle clamped (reading Q5),
                // committed unless the step is discarded at the goal
                float nx = x, nxl = xl, ny = y, nyl = yl, nz = z, nzl = zl, np_ = psi, npl = psil;
                float nvx = vx, nvxl = vxl, nvy = vy, nvyl = vyl, nvz = vz, nvzl = vzl;
                acc2(nx, nxl, h * dx);
                acc2(ny, nyl, h * dy);
                acc2(nz, nzl, h * dz);
                acc2(np_, npl, h * dpsi);
                acc2(nvx, nvxl, h * ax);
                acc2(nvy, nvyl, h * dvy);
                acc2(nvz, nvzl, h * dvz);
                const float nth = fmaf(h, dth, th), nph = fmaf(h, dph, ph);
                const float nwx = fmaf(h, dwx, wx), nwy = fmaf(h, dwy, wy), nwz = fmaf(h, dwz, wz);
                const float nd = clamp_keep_nan(fmaf(h, dd, d), -V.dmax, V.dmax);
                if (!keep) {
                    x = nx; xl = nxl; y = ny; yl = nyl; z = nz; zl = nzl; psi = np_; psil = npl;
                    vx = nvx; vxl = nvxl; vy = nvy; vyl = nvyl; vz = nvz; vzl = nvzl;
                    th = nth; ph = nph; wx = nwx; wy = nwy; wz = nwz; d = nd;
                    off = off || offs;
                } else {
                    done = true;
                    Ufrozen = U;
                }
            }
            if (p.step_margin && q == 0 && k + 1 < p.H) p.step_margin[(size_t)k * p.N + j] = sm;
            if (k + 1 < p.H) {
                if (sm < msm) {
                    msm = sm;
                    mstep = k;
                }
            } else {
                last_sm = sm;
            }
        }
        if (LANES > 1) {
            // the off-map flag is per wheel: OR it over the candidate's lanes
            off = __any_sync(qmask, off);
        }
        // final state: margin, goal test, terminal cost Phi (Sec. IV-C)
        {
            float sth, cth, sph, cph;
            sincos_r(th, sth, cth);
            sincos_r(ph, sph, cph);
            const float U = esm(V, ph, sph, cph, cth);
            margin = fminf(margin, U);
            last_sm = fminf(last_sm, U);
            if (last_sm < msm) mstep = p.H - 1;
            if (p.step_margin && q == 0) p.step_margin[(size_t)(p.H - 1) * p.N + j] = last_sm;
            const float gdx = (x - Cc.gx_hi) + (xl - Cc.gx_lo);
            const float gdy = (y - Cc.gy_hi) + (yl - Cc.gy_lo);
            const float d2 = fmaf(gdx, gdx, gdy * gdy);
            if (!done && d2 <= Cc.goal_r2) done = true;
            if (acc64) J = (float)(J64 + (double)(Cc.wg * sqrtf(d2)));
            else J = fmaf(Cc.wg, sqrtf(d2), J);
        }
        // fold the low parts back and leave the terrain frame
        const float xs[13] = {(x + T.x0_hi) + (xl + T.x0_lo), (y + T.y0_hi) + (yl + T.y0_lo),
                              z + zl, psi + psil, th, ph, vx + vxl, vy + vyl, vz + vzl,
                              wx, wy, wz, d};
        bool finite = isfinite(J);
#pragma unroll
        for (int c = 0; c < 13; ++c) finite = finite && isfinite(xs[c]);
        if (!finite) J = CUDART_INF_F;
        feasible = finite && margin > 0.f;
        if (q == 0) {
            const uint8_t fl = (feasible ? ATP_FLAG_FEASIBLE : 0) | (done ? ATP_FLAG_DONE : 0) |
                               (off ? ATP_FLAG_OFFMAP : 0) | (finite ? 0 : ATP_FLAG_NONFINITE);
            if (p.cost) p.cost[j] = J;
            if (p.margin) p.margin[j] = margin;
            if (p.flags) p.flags[j] = fl;
            if (p.min_step) p.min_step[j] = mstep;
            if (p.xf) {
                const size_t N = (size_t)p.N;
#pragma unroll
                for (int c = 0; c < 13; ++c) p.xf[c * N + j] = xs[c];
            }
        }
    }

}

// Register budgets, from A/B runs on the GB300: four lanes run best with
// ptxas free to use about 104 registers (minimum 1 CTA per SM), one and two
// lanes with the 128-register cap of 8 resident 64-thread CTAs per SM.
template <int LANES, bool PER_X0, bool REDUCE, int TEX, int ACC>
__global__ void __launch_bounds__(kPlanBlock, LANES == 4 ? 1 : 8)
plan_kernel(const __grid_constant__ PlanParams p)
{
    // 64-bit: N x LANES threads may exceed 2^31 when the lanes are forced
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = (int)(tid / LANES);
    const int q = LANES == 1 ? 0 : (int)(tid & (LANES - 1));
    const bool live = j < p.N;
    const unsigned qmask = LANES == 1 ? 0u : LANES == 2 ? (0x3u << (threadIdx.x & 30))
                                                        : (0xfu << (threadIdx.x & 28));
    float J = 0.f, margin = CUDART_INF_F;
    bool feasible = false;
    if (live) rollout_one<LANES, PER_X0, TEX, ACC>(p, j, q, qmask, J, margin, feasible);
    if (!REDUCE) return;
    plan_tail(p, j, live && q == 0, J, feasible, gridDim.x);
}

// Terrain staging: the one-lane rollout with a window of the texels in
// shared memory.  Every CTA copies the window (plain coalesced loads, once per
// CTA; at most 225 KB, so one CTA of 16 warps per SM), then each candidate
// reads the lookups inside it from shared memory and the rest through L1 as
// usual.  The texel values are the same either way, so the results are the
// bits of the unstaged one-lane kernel.
template <bool REDUCE, int ACC>
__global__ void __launch_bounds__(kStageBlock, 1)
plan_stage_kernel(const __grid_constant__ PlanParams p)
{
    const Terrain &T = p.T;
    const int n = T.ww * T.wh;
    for (int e = threadIdx.x; e < n; e += kStageBlock) {
        const int r = e / T.ww, c = e - r * T.ww;
        atp_win[e] = __ldg(T.tex + (size_t)(T.wy0 + r) * T.nx + (T.wx0 + c));
    }
    __syncthreads();
    const long long tid = (long long)blockIdx.x * kStageBlock + threadIdx.x;
    const int j = (int)tid;
    const bool live = tid < p.N;
    float J = 0.f, margin = CUDART_INF_F;
    bool feasible = false;
    if (live) rollout_one<1, false, TEX_F32W, ACC>(p, j, 0, 0u, J, margin, feasible);
    if (!REDUCE) return;
    plan_tail<kStageBlock>(p, j, live, J, feasible, gridDim.x);
}

template <bool REDUCE, int ACC>
static cudaError_t launch_stage(const PlanParams &p, cudaStream_t stream)
{
    const size_t smem = (size_t)p.T.ww * p.T.wh * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(plan_stage_kernel<REDUCE, ACC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(((size_t)p.N + kStageBlock - 1) / kStageBlock));
    plan_stage_kernel<REDUCE, ACC><<<grid, kStageBlock, smem, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_plan_staged(const PlanParams &p, bool reduce, cudaStream_t stream)
{
    if (p.tex_format != TEX_F32W || p.x0_soa || p.T.ww < 2 || p.T.wh < 2 || p.T.ww > kStageMaxSide ||
        p.T.wh > kStageMaxSide || p.T.wx0 < 0 || p.T.wy0 < 0 || p.T.wx0 + p.T.ww > p.T.nx ||
        p.T.wy0 + p.T.wh > p.T.ny)
        return cudaErrorInvalidValue;
    if (reduce) return p.acc64 ? launch_stage<true, kAccF64>(p, stream) : launch_stage<true, kAccF32>(p, stream);
    return p.acc64 ? launch_stage<false, kAccF64>(p, stream) : launch_stage<false, kAccF32>(p, stream);
}

// Continuous batching: one launch over a ragged batch of plans, each with its
// own vehicle, terrain, horizon, candidates and outputs.  Plan r owns CTAs
// [cta_begin[r], cta_begin[r+1]) with p.lanes threads per candidate, which
// the host chooses for the batch as a whole (every layout gives the same
// bits).  Every candidate runs exactly the code of a single plan, so its
// results are the same bits alone and in any mix.  BTEX is the batch's texel
// format when all its plans share one, or kTexMixed, where each plan branches
// on its own: a kernel that inlines both formats' rollouts in all three
// layouts spills registers, the single-format kernel does not (measured on
// the GB300 on the 32-vehicle serving mix: p50 2 to 12 % lower at 20 to 80
// requests/s per vehicle).
constexpr int kTexMixed = -1;

template <int LANES, int TEX>
__device__ __forceinline__ void batch_rollout(const PlanParams &p, int j, int q, unsigned qmask, float &J,
                                              float &margin, bool &feasible)
{
    if (p.x0_soa) rollout_one<LANES, true, TEX, kAccRuntime>(p, j, q, qmask, J, margin, feasible);
    else rollout_one<LANES, false, TEX, kAccRuntime>(p, j, q, qmask, J, margin, feasible);
}

template <int LANES, int BTEX>
__device__ __forceinline__ void batch_tex(const PlanParams &p, int j, int q, unsigned qmask, float &J,
                                          float &margin, bool &feasible)
{
    if constexpr (BTEX == kTexMixed) {
        if (p.tex_format == TEX_F32) batch_rollout<LANES, TEX_F32>(p, j, q, qmask, J, margin, feasible);
        else batch_rollout<LANES, TEX_BF16>(p, j, q, qmask, J, margin, feasible);
    } else {
        batch_rollout<LANES, BTEX>(p, j, q, qmask, J, margin, feasible);
    }
}

template <int BTEX>
__global__ void __launch_bounds__(kPlanBlock)
plan_batch_kernel(const __grid_constant__ BatchParams b)
{
    int lo = 0, hi = b.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (b.cta_begin[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    const PlanParams &p = b.req[lo];
    const int tid = ((int)blockIdx.x - b.cta_begin[lo]) * kPlanBlock + (int)threadIdx.x;
    // every thread of a CTA belongs to one plan: the branch is CTA-uniform
    const int lanes = p.lanes;
    const bool four = lanes == 4, two = lanes == 2;
    const int j = four ? tid >> 2 : two ? tid >> 1 : tid;
    const int q = four ? tid & 3 : two ? tid & 1 : 0;
    const bool live = j < p.N;
    const unsigned qmask = four ? 0xfu << (threadIdx.x & 28) : two ? 0x3u << (threadIdx.x & 30) : 0u;
    float J = 0.f, margin = CUDART_INF_F;
    bool feasible = false;
    if (live) {
        if (four) batch_tex<4, BTEX>(p, j, q, qmask, J, margin, feasible);
        else if (two) batch_tex<2, BTEX>(p, j, q, qmask, J, margin, feasible);
        else batch_tex<1, BTEX>(p, j, 0, 0u, J, margin, feasible);
    }
    plan_tail(p, j, live && q == 0, J, feasible, (unsigned)(b.cta_begin[lo + 1] - b.cta_begin[lo]));
}

cudaError_t launch_plan_batch(const BatchParams &b, cudaStream_t stream)
{
    if (b.n < 1 || b.n > kMaxBatch) return cudaErrorInvalidValue;
    bool f32 = true, bf16 = true;
    for (int r = 0; r < b.n; ++r) {
        f32 = f32 && b.req[r].tex_format == TEX_F32;
        bf16 = bf16 && b.req[r].tex_format == TEX_BF16;
    }
    const unsigned grid = (unsigned)b.cta_begin[b.n];
    if (f32) plan_batch_kernel<TEX_F32><<<grid, kPlanBlock, 0, stream>>>(b);
    else if (bf16) plan_batch_kernel<TEX_BF16><<<grid, kPlanBlock, 0, stream>>>(b);
    else plan_batch_kernel<kTexMixed><<<grid, kPlanBlock, 0, stream>>>(b);
    return cudaGetLastError();
}

template <int LANES, int TEX, int ACC>
static cudaError_t launch_acc(const PlanParams &p, bool reduce, cudaStream_t stream)
{
    const dim3 block(kPlanBlock);
    const size_t threads = (size_t)p.N * LANES;
    const dim3 grid((unsigned)((threads + kPlanBlock - 1) / kPlanBlock));
    const bool per = p.x0_soa != nullptr;
    if (reduce) {
        if (per) plan_kernel<LANES, true, true, TEX, ACC><<<grid, block, 0, stream>>>(p);
        else plan_kernel<LANES, false, true, TEX, ACC><<<grid, block, 0, stream>>>(p);
    } else {
        if (per) plan_kernel<LANES, true, false, TEX, ACC><<<grid, block, 0, stream>>>(p);
        else plan_kernel<LANES, false, false, TEX, ACC><<<grid, block, 0, stream>>>(p);
    }
    return cudaGetLastError();
}

template <int LANES, int TEX>
static cudaError_t launch_lanes(const PlanParams &p, bool reduce, cudaStream_t stream)
{
    return p.acc64 ? launch_acc<LANES, TEX, kAccF64>(p, reduce, stream)
                   : launch_acc<LANES, TEX, kAccF32>(p, reduce, stream);
}

cudaError_t launch_plan(const PlanParams &p, bool reduce, cudaStream_t stream)
{
    // several lanes per candidate while the batch leaves the GPU's thread
    // slots mostly empty (the rollout is then latency bound); one lane once
    // the batch fills the machine
    const int lanes = plan_lanes(p.lanes, p.N);
    if (p.tex_format == TEX_F32) {
        if (lanes == 4) return launch_lanes<4, TEX_F32>(p, reduce, stream);
        if (lanes == 2) return launch_lanes<2, TEX_F32>(p, reduce, stream);
        return launch_lanes<1, TEX_F32>(p, reduce, stream);
    }
    if (lanes == 4) return launch_lanes<4, TEX_BF16>(p, reduce, stream);
    if (lanes == 2) return launch_lanes<2, TEX_BF16>(p, reduce, stream);
    return launch_lanes<1, TEX_BF16>(p, reduce, stream);
}

// One node's texel (Sec. III-A numeric slope, reading Q10): height, central-
// difference slopes (one-sided on the border) and the costmap value.
__device__ __forceinline__ float4 node_texel(const float *__restrict__ H, const float *__restrict__ cm, int nx,
                                             int ny, float inv_cell, int i, int j)
{
    const size_t r = (size_t)j * nx;
    const float c = H[r + i];
    float gx, gy;
    if (i == 0) gx = (H[r + 1] - c) * inv_cell;
    else if (i == nx - 1) gx = (c - H[r + nx - 2]) * inv_cell;
    else gx = (H[r + i + 1] - H[r + i - 1]) * (0.5f * inv_cell);
    if (j == 0) gy = (H[r + nx + i] - c) * inv_cell;
    else if (j == ny - 1) gy = (c - H[r - nx + i]) * inv_cell;
    else gy = (H[r + nx + i] - H[r - nx + i]) * (0.5f * inv_cell);
    return make_float4(c, gx, gy, cm ? cm[r + i] : 0.f);
}

__global__ void terrain_prepare_f32_kernel(const float *__restrict__ H, const float *__restrict__ cm,
                                           int nx, int ny, float inv_cell, float4 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    out[(size_t)j * nx + i] = node_texel(H, cm, nx, ny, inv_cell, i, j);
}

// BF16 texels.  Per 8 x 8 block a plane through the block's first node with
// the slopes of its first row and first column (FP32, each operation rounded
// on its own so that the plane is reproducible bit for bit); per node the
// bf16 (round to nearest even) of the height's and the two node slopes'
// residuals from that plane, and of the costmap value.
__global__ void terrain_block_plane_kernel(const float *__restrict__ H, int nx, int ny, int nbx,
                                           int nby, float4 *__restrict__ plane)
{
    const int bi = blockIdx.x * blockDim.x + threadIdx.x;
    const int bj = blockIdx.y * blockDim.y + threadIdx.y;
    if (bi >= nbx || bj >= nby) return;
    const int i0 = bi * 8, j0 = bj * 8;
    const int ni = min(8, nx - i0), nj = min(8, ny - j0);
    const float c0 = H[(size_t)j0 * nx + i0];
    const float cx = ni > 1 ? __fmul_rn(__fsub_rn(H[(size_t)j0 * nx + i0 + ni - 1], c0),
                                        __fdiv_rn(1.0f, (float)(ni - 1))) : 0.f;
    const float cy = nj > 1 ? __fmul_rn(__fsub_rn(H[(size_t)(j0 + nj - 1) * nx + i0], c0),
                                        __fdiv_rn(1.0f, (float)(nj - 1))) : 0.f;
    plane[(size_t)bj * nbx + bi] = make_float4(c0, cx, cy, 0.f);
}

__device__ __forceinline__ unsigned bf16_bits(float v)
{
    return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__global__ void terrain_prepare_bf16_kernel(const float *__restrict__ H, const float *__restrict__ cm,
                                            int nx, int ny, float inv_cell, const float4 *__restrict__ plane,
                                            int nbx, uint2 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const size_t r = (size_t)j * nx;
    const float c = H[r + i];
    float gx, gy;
    if (i == 0) gx = (H[r + 1] - c) * inv_cell;
    else if (i == nx - 1) gx = (c - H[r + nx - 2]) * inv_cell;
    else gx = (H[r + i + 1] - H[r + i - 1]) * (0.5f * inv_cell);
    if (j == 0) gy = (H[r + nx + i] - c) * inv_cell;
    else if (j == ny - 1) gy = (c - H[r - nx + i]) * inv_cell;
    else gy = (H[r + nx + i] - H[r - nx + i]) * (0.5f * inv_cell);
    const float4 P = plane[(size_t)(j >> 3) * nbx + (i >> 3)];
    const float res = __fsub_rn(c, block_plane(P, i, j));
    // slopes as residuals from the plane's own slopes
    const float rgx = __fsub_rn(gx, __fmul_rn(P.y, inv_cell));
    const float rgy = __fsub_rn(gy, __fmul_rn(P.z, inv_cell));
    const float cv = cm ? cm[r + i] : 0.f;
    out[r + i] = make_uint2(bf16_bits(res) | (bf16_bits(rgx) << 16), bf16_bits(rgy) | (bf16_bits(cv) << 16));
}

cudaError_t launch_terrain_prepare_bf16(const float *heights, const float *costmap, int nx, int ny,
                                        float inv_cell, uint2 *texels, float4 *plane, cudaStream_t stream)
{
    const int nbx = (nx + 7) / 8, nby = (ny + 7) / 8;
    const dim3 b1(16, 16);
    const dim3 g1((unsigned)((nbx + 15) / 16), (unsigned)((nby + 15) / 16));
    terrain_block_plane_kernel<<<g1, b1, 0, stream>>>(heights, nx, ny, nbx, nby, plane);
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8));
    terrain_prepare_bf16_kernel<<<grid, block, 0, stream>>>(heights, costmap, nx, ny, inv_cell, plane, nbx,
                                                            texels);
    return cudaGetLastError();
}

cudaError_t launch_terrain_prepare_f32(const float *heights, const float *costmap, int nx, int ny,
                                       float inv_cell, float4 *out, cudaStream_t stream)
{
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8));
    terrain_prepare_f32_kernel<<<grid, block, 0, stream>>>(heights, costmap, nx, ny, inv_cell, out);
    return cudaGetLastError();
}

}  // namespace atp
