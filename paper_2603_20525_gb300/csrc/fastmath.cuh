// fastmath.cuh - the FP32 elementary functions of the rollout, written for the
// argument ranges the SRB model produces, each a few FMAs instead of a general
// library sequence.  Accuracy against CUDA's own functions is checked on the
// GPU by tests/test_gpu_math.py (atp_math_check).
#pragma once

#include <cuda_runtime.h>

namespace atp {

// Single MUFU reciprocal (rcp.approx.ftz.f32, max error 1 ulp).  The .ftz
// form is one instruction; the form that handles subnormal inputs adds a
// fix-up sequence.  Every reciprocal of the rollout takes an O(1) quantity
// (cos theta, the normal's vertical component, a slip ratio's larger side),
// never a subnormal.
__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Single MUFU reciprocal square root (rsqrt.approx.ftz.f32), for the tire's
// mu^2 + (C alpha)^2 >= mu^2 and the unit normal's 1 + |grad f|^2 >= 1.
__device__ __forceinline__ float rsq(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// sin and cos of |x| <= pi/4 from their Taylor series, truncated after x^11
// and x^12: the first omitted terms are below 7e-12 and 2e-13 on the interval.
__device__ __forceinline__ void sincos_q(float x, float &s, float &c)
{
    const float x2 = x * x;
    float ps = fmaf(x2, -2.50521084e-08f, 2.75573192e-06f);    // -1/11!, 1/9!
    ps = fmaf(x2, ps, -1.98412698e-04f);                        // -1/7!
    ps = fmaf(x2, ps, 8.33333333e-03f);                         //  1/5!
    ps = fmaf(x2, ps, -1.66666667e-01f);                        // -1/3!
    s = fmaf(x * x2, ps, x);
    float pc = fmaf(x2, 2.08767570e-09f, -2.75573192e-07f);     // 1/12!, -1/10!
    pc = fmaf(x2, pc, 2.48015873e-05f);                         //  1/8!
    pc = fmaf(x2, pc, -1.38888889e-03f);                        // -1/6!
    pc = fmaf(x2, pc, 4.16666667e-02f);                         //  1/4!
    pc = fmaf(x2, pc, -0.5f);                                   // -1/2!
    c = fmaf(x2, pc, 1.0f);
}

// sin and cos of any |x| < 2^17: Cody-Waite reduction by pi/2, split into
// three floats (pi/2 = P1 + P2 + P3 to 72 bits), then the quadrant's
// polynomial.  Larger and infinite arguments take CUDA's sincosf.  A NaN
// takes the reduction and comes out NaN, as from sincosf: a candidate whose
// state has gone NaN (one that tipped over and diverged) then shares its
// warp's path instead of sending the warp through sincosf's too (measured on
// the GB300: 3.5 % off the paper's configuration, where half the candidates
// end non-finite; the same bits).
__device__ __forceinline__ void sincos_r(float x, float &s, float &c)
{
    if (fabsf(x) <= 0.785398163f) {
        sincos_q(x, s, c);
        return;
    }
    if (fabsf(x) >= 131072.f) {
        sincosf(x, &s, &c);
        return;
    }
    const float k = rintf(x * 6.36619747e-01f);                 // x / (pi/2)
    float r = fmaf(-k, 1.57079637e+00f, x);                     // P1 = fl(pi/2)
    r = fmaf(-k, -4.37113883e-08f, r);                          // P2 = fl(pi/2 - P1)
    r = fmaf(-k, -1.71512451e-15f, r);                          // P3 = fl(pi/2 - P1 - P2)
    float sr, cr;
    sincos_q(r, sr, cr);
    const int q = ((int)k) & 3;
    s = (q == 0) ? sr : (q == 1) ? cr : (q == 2) ? -sr : -cr;
    c = (q == 0) ? cr : (q == 1) ? -sr : (q == 2) ? -cr : sr;
}

// atan(r) for r in [0, 1] as r P(r^2), P of degree 8 fitted for minimum
// maximum relative error (fit_atan.py): 1.1e-7 including FP32 evaluation.
__device__ __forceinline__ float atan01(float r)
{
    const float s = r * r;
    float p = fmaf(s, 0.0028498878236860037f, -0.016068624332547188f);
    p = fmaf(s, p, 0.04269151762127876f);
    p = fmaf(s, p, -0.07504294812679291f);
    p = fmaf(s, p, 0.10640934109687805f);
    p = fmaf(s, p, -0.14203645288944244f);
    p = fmaf(s, p, 0.1999261975288391f);
    p = fmaf(s, p, -0.3333307206630707f);
    p = fmaf(s, p, 1.0f);
    return r * p;
}

// atan2(y, x) by octant reduction to atan01; atan2(+-0, +-0) = 0 like the
// FP64 oracle's libm for x = +0.  A NaN argument gives a finite, meaningless
// angle: the rollout's state is then NaN already and the candidate is
// flagged non-finite from its final state (measured on the GB300: dropping
// the NaN select took 9 % off a full-GPU plan, the same bits otherwise).
__device__ __forceinline__ float atan2_r(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float r = mn * rcp(fmaxf(mx, 1e-30f));
    float t = atan01(r);
    if (ay > ax) t = 1.57079633f - t;
    if (x < 0.f) t = 3.14159265f - t;
    return copysignf(t, y);
}

// Packed two-wide FP32 (fma.rn.f32x2, sub.rn.f32x2; Blackwell): each half is
// the round-to-nearest IEEE operation of its scalar form, subnormals kept, so
// the results are the scalar code's bits while one instruction issues both
// halves.  The rollout is issue-bound once the batch fills the GPU, and the
// FMA pipe runs a packed instruction at half rate, so packing pays where
// pairs are already adjacent (a texel's (h, f_x) and (f_y, c) halves) or
// share an operand.  Only fused multiply-adds and differences are packed: a
// packed multiply feeding a packed add is fused into one rounding by the
// compiler despite the explicit rounding mode (measured on the GB300 in every
// case where the two differ), so the scalar code's separate multiply and add
// stay scalar.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

}  // namespace atp
