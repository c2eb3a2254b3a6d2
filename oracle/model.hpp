// model.hpp - the SRB rollout (Sec. IV-A..IV-D) and the planar EST rollout
// (appendix "Extended Single-Track Vehicle Dynamics Model", Sec. IV-C
// lateral-acceleration constraint) of arxiv 2603.20525, restated once more in
// the paper's order and with the readings of oracle.h, templated on
//
//   T  the arithmetic type of every model quantity, and
//   S  the storage type of the state vector (x, y, z of the SRB model are
//      also used in S to place the contact points and read the terrain).
//
// TEST INFRASTRUCTURE.  Only oracle/ includes it and only the test suite calls
// what it builds; it shares no code with the CUDA path.  Instantiations:
//   T = S = double      reproduces srb.c / est.c (checked by the tests);
//   T = S = tape scalar the FP64 reverse-mode adjoint (adjoint.cpp);
//   T = FP32 scalar, S = FP64 scalar   the FP32 arithmetic reference
//                       (emul32.cpp): every model quantity rounded to FP32,
//                       the state accumulated in FP64 where a compensated
//                       FP32 implementation keeps it exactly (position,
//                       heading, linear velocity) and rounded to FP32 after
//                       every Euler step elsewhere;
//   T = S = counting scalar  the operation count per Euler step (emul32.cpp).
#pragma once

#include <cmath>
#include <cstring>

extern "C" {
#include "oracle.h"
}

namespace orcm {

inline double value(double a) { return a; }

// elementary functions: std:: for double, argument-dependent lookup for the
// scalar wrappers
template <class T> T Tsin(const T &a) { using std::sin; return sin(a); }
template <class T> T Tcos(const T &a) { using std::cos; return cos(a); }
template <class T> T Tsqrt(const T &a) { using std::sqrt; return sqrt(a); }
template <class T> T Tfabs(const T &a) { using std::fabs; return fabs(a); }
template <class T> T Tatan2(const T &y, const T &x) { using std::atan2; return atan2(y, x); }
template <class T> T Tasin(const T &a) { using std::asin; return asin(a); }

// sin and cos of a stored state angle, as an arithmetic value: evaluated at
// the stored (possibly wider) argument, then converted
template <class T, class S> T Ssin(const S &a) { return T(Tsin(a)); }
template <class T, class S> T Scos(const S &a) { return T(Tcos(a)); }

template <class T> T clampT(const T &v, double lo, double hi)
{
    if (value(v) < lo) return T(lo);
    if (value(v) > hi) return T(hi);
    return v;
}

// ---- SRB model --------------------------------------------------------------
enum { X = 0, Y, Z, PSI, THETA, PHI, VX, VY, VZ, WX, WY, WZ, DELTA };

struct K {
    double Fs[4], k[4], b[4], rho[4][3], U0, eps;
};

inline void consts(const orc_vehicle *v, const orc_cost *c, K &k)
{
    double L = v->Lf + v->Lr, he = 0.5 * v->e;
    // Sec. III-A load transfer, Sec. IV-A nominal tire loading (g/2) K_zz,i
    double Kzz[4] = {v->M * v->Lr / L, v->M * v->Lr / L, v->M * v->Lf / L, v->M * v->Lf / L};
    double rx[4] = {v->Lf, v->Lf, -v->Lr, -v->Lr}, ry[4] = {he, -he, he, -he};
    for (int i = 0; i < 4; ++i) {
        k.Fs[i] = 0.5 * v->g * Kzz[i];
        k.k[i] = i < 2 ? v->kf : v->kr;
        k.b[i] = i < 2 ? v->bf : v->br;
        k.rho[i][0] = rx[i];
        k.rho[i][1] = ry[i];
        k.rho[i][2] = -v->hR;
    }
    k.U0 = orc_esm(v, 0.0, 0.0);
    k.eps = c->eps_esm > 0 ? c->eps_esm : 0.1 * k.U0;
}

// ESM (Sec. IV-B): +/- M g Rbar (1 - sin(|phi| + phibar)) cos(theta)
template <class T> T esmT(const orc_vehicle *v, const T &phi, const T &theta)
{
    double Rbar = std::sqrt(v->hR * v->hR + 0.25 * v->e * v->e);
    double phibar = std::atan(2.0 * v->hR / v->e);
    T a = Tfabs(phi) + phibar;
    T dh = Rbar * (1.0 - Tsin(a)) * Tcos(theta);
    double s = value(a) < 0.5 * M_PI ? 1.0 : -1.0;
    return s * v->M * v->g * dh;
}

// bilinear height, slopes and costmap at (x, y), given in the state's type
// (reading Q10); returns 1 for a query off the map
template <class T, class P> int sampleT(const orc_terrain *t, const P &x, const P &y, T out[4])
{
    P u = (x - t->x0) / t->cell, w = (y - t->y0) / t->cell;
    double umax = t->nx - 1, wmax = t->ny - 1;
    int off = !(value(u) >= 0.0 && value(u) <= umax && value(w) >= 0.0 && value(w) <= wmax);
    if (std::isnan(value(u))) u = P(0.0);
    if (std::isnan(value(w))) w = P(0.0);
    u = clampT(u, 0.0, umax);
    w = clampT(w, 0.0, wmax);
    int i = (int)std::floor(value(u)), j = (int)std::floor(value(w));
    if (i > t->nx - 2) i = t->nx - 2;
    if (j > t->ny - 2) j = t->ny - 2;
    T a = T(u - (double)i), b = T(w - (double)j);
    T w00 = (1.0 - a) * (1.0 - b), w10 = a * (1.0 - b), w01 = (1.0 - a) * b, w11 = a * b;
    const int i00 = j * t->nx + i, i10 = i00 + 1, i01 = i00 + t->nx, i11 = i01 + 1;
    out[0] = w00 * (double)t->heights[i00] + w10 * (double)t->heights[i10] +
             w01 * (double)t->heights[i01] + w11 * (double)t->heights[i11];
    out[1] = w00 * t->gx[i00] + w10 * t->gx[i10] + w01 * t->gx[i01] + w11 * t->gx[i11];
    out[2] = w00 * t->gy[i00] + w10 * t->gy[i10] + w01 * t->gy[i01] + w11 * t->gy[i11];
    if (t->costmap)
        out[3] = w00 * (double)t->costmap[i00] + w10 * (double)t->costmap[i10] +
                 w01 * (double)t->costmap[i01] + w11 * (double)t->costmap[i11];
    else
        out[3] = T(0.0);
    return off;
}

// xi_dot = A(xi) + B zeta and the running cost rate L (Sec. IV-A, IV-C),
// given the state's ESM U; returns 1 if a wheel read the terrain off the map
template <class T, class S>
int derivT(const orc_vehicle *v, const K &k, const orc_cost *c, const orc_terrain *t, const S xi[13],
           const T zeta[2], const T &U, T xd[13], T &L)
{
    T cps = Scos<T>(xi[PSI]), sps = Ssin<T>(xi[PSI]), cth = Scos<T>(xi[THETA]), sth = Ssin<T>(xi[THETA]);
    T cph = Scos<T>(xi[PHI]), sph = Ssin<T>(xi[PHI]);
    T R[9];
    R[0] = cps * cth;
    R[1] = cps * sph * sth - cph * sps;
    R[2] = sph * sps + cph * cps * sth;
    R[3] = cth * sps;
    R[4] = cph * cps + sph * sps * sth;
    R[5] = cph * sps * sth - cps * sph;
    R[6] = -sth;
    R[7] = cth * sph;
    R[8] = cph * cth;
    T gB[3] = {-v->g * R[6], -v->g * R[7], -v->g * R[8]};
    T vB[3] = {T(xi[VX]), T(xi[VY]), T(xi[VZ])}, w[3] = {T(xi[WX]), T(xi[WY]), T(xi[WZ])};
    T wxbz[3] = {w[1], -w[0], T(0.0)};
    T Fy_sum(0.0), Fz_sum(0.0), M[3] = {T(0.0), T(0.0), T(0.0)}, cmap(0.0);
    int off = 0;
    for (int i = 0; i < 4; ++i) {
        const double *rho = k.rho[i];
        T vi[3], ter[4], tauB[3];
        // contact point in W (in the state's type) and its velocity in B
        S P[3];
        P[0] = xi[X] + R[0] * rho[0] + R[1] * rho[1] + R[2] * rho[2];
        P[1] = xi[Y] + R[3] * rho[0] + R[4] * rho[1] + R[5] * rho[2];
        P[2] = xi[Z] + R[6] * rho[0] + R[7] * rho[1] + R[8] * rho[2];
        vi[0] = vB[0] + (w[1] * rho[2] - w[2] * rho[1]);
        vi[1] = vB[1] + (w[2] * rho[0] - w[0] * rho[2]);
        vi[2] = vB[2] + (w[0] * rho[1] - w[1] * rho[0]);
        off |= sampleT(t, P[0], P[1], ter);
        // slope-normal direction (reading Q1) in B
        T tW[3] = {-ter[1], -ter[2], T(1.0)};
        tauB[0] = R[0] * tW[0] + R[3] * tW[1] + R[6] * tW[2];
        tauB[1] = R[1] * tW[0] + R[4] * tW[1] + R[7] * tW[2];
        tauB[2] = R[2] * tW[0] + R[5] * tW[1] + R[8] * tW[2];
        // suspension extension and rate, spring and damper with liftoff
        T chi = T(P[2] - ter[0]) / tauB[2];
        T rel[3] = {vi[0] - chi * wxbz[0], vi[1] - chi * wxbz[1], vi[2] - chi * wxbz[2]};
        T chid = (tauB[0] * rel[0] + tauB[1] * rel[1] + tauB[2] * rel[2]) / tauB[2];
        T Fk = k.Fs[i] - k.k[i] * chi;
        if (value(Fk) < 0.0) Fk = T(0.0);
        T Fb(0.0);
        if (value(Fk) > 0.0) {
            Fb = -k.b[i] * chid;
            if (value(Fb) < -value(Fk)) Fb = -Fk;
        }
        T Fz = Fk + Fb;
        // slip angle (reading Q11) and the sigmoid tire (Sec. III-A)
        T di = i < 2 ? T(xi[DELTA]) : T(0.0);
        T alpha = Tatan2(vi[1], vi[0]) - di;
        T Ca = v->C * alpha;
        T den = Tsqrt(v->mu * v->mu + Ca * Ca);
        T Fy = (value(den) == 0.0) ? T(0.0) : Fz * (-Ca * v->mu / den);
        // rear longitudinal constraint force holding the prescribed v_x rate
        T Fx = (i >= 2) ? 0.5 * v->M * (zeta[1] - gB[0] + w[1] * vB[2] - w[2] * vB[1]) : T(0.0);
        T cdi = Tcos(di);
        Fy_sum += Fy * cdi;
        Fz_sum += Fz;
        T F[3] = {Fx, Fy * cdi, Fz};
        M[0] += rho[1] * F[2] - rho[2] * F[1];
        M[1] += rho[2] * F[0] - rho[0] * F[2];
        M[2] += rho[0] * F[1] - rho[1] * F[0];
        cmap += ter[3];
    }
    xd[X] = R[0] * vB[0] + R[1] * vB[1] + R[2] * vB[2];
    xd[Y] = R[3] * vB[0] + R[4] * vB[1] + R[5] * vB[2];
    xd[Z] = R[6] * vB[0] + R[7] * vB[1] + R[8] * vB[2];
    xd[PSI] = (sph / cth) * w[1] + (cph / cth) * w[2];
    xd[THETA] = cph * w[1] - sph * w[2];
    xd[PHI] = w[0] + (sph * sth / cth) * w[1] + (cph * sth / cth) * w[2];
    xd[VX] = zeta[1];
    xd[VY] = Fy_sum / v->M + gB[1] + w[0] * vB[2] - w[2] * vB[0];
    xd[VZ] = Fz_sum / v->M + gB[2] - w[0] * vB[1] + w[1] * vB[0];
    xd[WX] = (M[0] + (v->Jyy - v->Jzz) * w[1] * w[2]) / v->Jxx;
    xd[WY] = (M[1] - (v->Jxx - v->Jzz) * w[0] * w[2]) / v->Jyy;
    xd[WZ] = (M[2] + (v->Jxx - v->Jyy) * w[0] * w[1]) / v->Jzz;
    xd[DELTA] = zeta[0];
    T s = 1.0 - U / k.eps;
    if (value(s) < 0.0) s = T(0.0);
    L = (c->wt + c->wc * zeta[0] * zeta[0]) + (c->sigma * s * s + cmap);
    return off;
}

// Which state components a compensated FP32 implementation accumulates
// exactly: position, heading, linear velocity (SRB); position, heading,
// lateral and longitudinal velocity (EST).
constexpr bool kSrbWide[13] = {true, true, true, true, false, false, true, true, true,
                               false, false, false, false};
constexpr bool kEstWide[7] = {true, true, true, true, false, false, true};

// The result of one rollout.
template <class T> struct Result {
    T J, margin;
    double xf[13];
    unsigned char flags;
    int min_step;         // control step of the smallest per-step margin
};

// One SRB candidate: forward Euler with zero-order-hold controls u[H][2],
// goal truncation, ESM margin, cost (Sec. IV-C, IV-D); the same semantics
// as srb.c's rollout.  The components a compensated FP32 implementation
// would not keep exactly are rounded to T after each Euler step (a no-op
// when T and S are one type).
template <class T, class S>
Result<T> rolloutT(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13],
                   const T *u, int H, double dt, int n_sub, long *euler_steps = nullptr)
{
    K k;
    consts(v, c, k);
    const double h = dt / n_sub;
    S xi[13];
    T xd[13], L;
    for (int q = 0; q < 13; ++q) xi[q] = S(x0[q]);
    T J(0.0), margin(INFINITY), best_sm(INFINITY);
    int done = 0, off = 0, min_step = 0;
    for (int kk = 0; kk < H; ++kk) {
        T zeta[2] = {clampT(u[2 * kk], -v->delta_rate_max, v->delta_rate_max), u[2 * kk + 1]};
        T sm(INFINITY);
        for (int s = 0; s < n_sub; ++s) {
            T U = esmT(v, T(xi[PHI]), T(xi[THETA]));
            if (value(U) < value(margin)) margin = U;
            if (value(U) < value(sm)) sm = U;
            if (!done) {
                T gdx = T(xi[X] - c->goal_x), gdy = T(xi[Y] - c->goal_y);
                if (value(Tsqrt(gdx * gdx + gdy * gdy)) <= c->goal_r) done = 1;
            }
            if (!done) {
                off |= derivT(v, k, c, t, xi, zeta, U, xd, L);
                J += h * L;
                for (int q = 0; q < 13; ++q) {
                    xi[q] = xi[q] + S(h * xd[q]);
                    if (!kSrbWide[q]) xi[q] = S(T(xi[q]));
                }
                xi[DELTA] = S(clampT(T(xi[DELTA]), -v->delta_max, v->delta_max));
                if (euler_steps) ++*euler_steps;
            }
        }
        if (kk == H - 1) {
            // the final state folds into the last control step's margin
            T U = esmT(v, T(xi[PHI]), T(xi[THETA]));
            if (value(U) < value(margin)) margin = U;
            if (value(U) < value(sm)) sm = U;
        }
        if (value(sm) < value(best_sm)) {
            best_sm = sm;
            min_step = kk;
        }
    }
    T gx = T(xi[X] - c->goal_x), gy = T(xi[Y] - c->goal_y);
    T gd = Tsqrt(gx * gx + gy * gy);
    if (!done && value(gd) <= c->goal_r) done = 1;
    J += c->wg * gd;
    Result<T> r;
    r.flags = 0;
    if (done) r.flags |= ORC_DONE;
    if (off) r.flags |= ORC_OFFMAP;
    int finite = std::isfinite(value(J));
    for (int q = 0; q < 13; ++q) {
        r.xf[q] = value(xi[q]);
        finite = finite && std::isfinite(r.xf[q]);
    }
    if (!finite) {
        r.flags |= ORC_NONFINITE;
        J = T(INFINITY);
    }
    if (finite && value(margin) > 0.0) r.flags |= ORC_FEASIBLE;
    r.J = J;
    r.margin = margin;
    r.min_step = min_step;
    return r;
}

// ---- planar EST model ---------------------------------------------------------
enum { EX = 0, EY, EPSI, EVY, EWZ, EDELTA, EVX };

struct EK {
    double Kzzf, Kzzr, Kzx, abar, eps, rho[4][3];
};

inline void est_consts(const orc_vehicle *v, const orc_cost *c, EK &k)
{
    const double L = v->Lf + v->Lr;
    const double Kzy = v->M * v->hR / v->e;
    k.Kzzf = v->M * v->Lr / L;
    k.Kzzr = v->M * v->Lf / L;
    k.Kzx = v->M * v->hR / L;
    k.abar = v->M * v->g / (2.0 * Kzy);
    k.eps = c->eps_esm > 0.0 ? c->eps_esm : 0.1 * k.abar;
    for (int i = 0; i < 4; ++i) {
        k.rho[i][0] = i < 2 ? v->Lf : -v->Lr;
        k.rho[i][1] = (i & 1) ? -0.5 * v->e : 0.5 * v->e;
        k.rho[i][2] = -v->hR;
    }
}

// EST derivative, running cost rate and lateral-acceleration margin (the
// appendix model, readings Q1, Q15-Q17 of est.c); returns 1 off the map
template <class T, class S>
int est_derivT(const orc_vehicle *v, const EK &k, const orc_cost *c, const orc_terrain *t, const S xi[7],
               const T zeta[2], T xd[7], T &L, T &margin)
{
    T ter[4];
    int off = sampleT(t, xi[EX], xi[EY], ter);
    // unit normal under the CoM; pitch and roll of the local plane (1-2-3)
    T n = Tsqrt(ter[1] * ter[1] + ter[2] * ter[2] + 1.0);
    T tau[3] = {-ter[1] / n, -ter[2] / n, 1.0 / n};
    T theta = Tasin(tau[0]);
    T phi = Tatan2(-tau[1], tau[2]);
    T cf = Tcos(phi), sf = Tsin(phi), ct = Tcos(theta), st = Tsin(theta);
    T cp = Scos<T>(xi[EPSI]), sp = Ssin<T>(xi[EPSI]);
    T R[9];
    R[0] = ct * cp;
    R[1] = -ct * sp;
    R[2] = st;
    R[3] = cf * sp + cp * sf * st;
    R[4] = cf * cp - sf * st * sp;
    R[5] = -ct * sf;
    R[6] = sf * sp - cf * cp * st;
    R[7] = cp * sf + cf * st * sp;
    R[8] = cf * ct;
    T gB[3] = {-v->g * R[6], -v->g * R[7], -v->g * R[8]};
    T vx = T(xi[EVX]), vy = T(xi[EVY]), wz = T(xi[EWZ]), delta = T(xi[EDELTA]);
    T aBx = zeta[1] - wz * vy;
    T Fzf = -k.Kzzf * gB[2] - k.Kzx * aBx;
    T Fzr = -k.Kzzr * gB[2] + k.Kzx * aBx;
    T af = Tatan2(vy + wz * v->Lf, vx) - delta;
    T ar = Tatan2(vy - wz * v->Lr, vx);
    T Caf = v->C * af, Car = v->C * ar;
    T denf = Tsqrt(v->mu * v->mu + Caf * Caf), denr = Tsqrt(v->mu * v->mu + Car * Car);
    T Fyf = Fzf * ((value(denf) == 0.0) ? T(0.0) : -Caf * v->mu / denf);
    T Fyr = Fzr * ((value(denr) == 0.0) ? T(0.0) : -Car * v->mu / denr);
    xd[EX] = R[0] * vx + R[1] * vy;
    xd[EY] = R[3] * vx + R[4] * vy;
    xd[EPSI] = wz;
    xd[EVY] = (Fyf + Fyr) / v->M + gB[1] - wz * vx;
    xd[EWZ] = (Fyf * v->Lf * Tcos(delta) - Fyr * v->Lr) / v->Jzz;
    xd[EDELTA] = zeta[0];
    xd[EVX] = zeta[1];
    T aBy = xd[EVY] + wz * vx;
    margin = k.abar - Tfabs(aBy - gB[1]);
    T viol = 1.0 - margin / k.eps;
    L = c->wt + c->wc * zeta[0] * zeta[0];
    if (value(viol) > 0.0) L += c->sigma * viol * viol;
    for (int i = 0; i < 4 && t->costmap; ++i) {
        S px = xi[EX] + R[0] * k.rho[i][0] + R[1] * k.rho[i][1] + R[2] * k.rho[i][2];
        S py = xi[EY] + R[3] * k.rho[i][0] + R[4] * k.rho[i][1] + R[5] * k.rho[i][2];
        T w[4];
        off |= sampleT(t, px, py, w);
        L += w[3];
    }
    return off;
}

// One EST candidate (est.c's semantics: the margin covers integrated steps)
template <class T, class S>
Result<T> est_rolloutT(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[7],
                       const T *u, int H, double dt, int n_sub, long *euler_steps = nullptr)
{
    EK k;
    est_consts(v, c, k);
    const double h = dt / n_sub;
    S xi[7];
    T xd[7], L, m;
    for (int q = 0; q < 7; ++q) xi[q] = S(x0[q]);
    T J(0.0), margin(INFINITY), best_sm(INFINITY);
    int done = 0, off = 0, min_step = 0;
    for (int kk = 0; kk < H; ++kk) {
        T zeta[2] = {clampT(u[2 * kk], -v->delta_rate_max, v->delta_rate_max), u[2 * kk + 1]};
        T sm(INFINITY);
        for (int s = 0; s < n_sub; ++s) {
            if (!done && std::hypot(value(xi[EX]) - c->goal_x, value(xi[EY]) - c->goal_y) <= c->goal_r)
                done = 1;
            if (!done) {
                off |= est_derivT(v, k, c, t, xi, zeta, xd, L, m);
                if (value(m) < value(margin)) margin = m;
                if (value(m) < value(sm)) sm = m;
                J += h * L;
                for (int q = 0; q < 7; ++q) {
                    xi[q] = xi[q] + S(h * xd[q]);
                    if (!kEstWide[q]) xi[q] = S(T(xi[q]));
                }
                xi[EDELTA] = S(clampT(T(xi[EDELTA]), -v->delta_max, v->delta_max));
                if (euler_steps) ++*euler_steps;
            }
        }
        if (value(sm) < value(best_sm)) {
            best_sm = sm;
            min_step = kk;
        }
    }
    double dx = value(xi[EX]) - c->goal_x, dy = value(xi[EY]) - c->goal_y;
    if (!done && std::hypot(dx, dy) <= c->goal_r) done = 1;
    T gx = T(xi[EX] - c->goal_x), gy = T(xi[EY] - c->goal_y);
    J += c->wg * Tsqrt(gx * gx + gy * gy);
    Result<T> r;
    r.flags = 0;
    if (done) r.flags |= ORC_DONE;
    if (off) r.flags |= ORC_OFFMAP;
    int finite = std::isfinite(value(J));
    for (int q = 0; q < 13; ++q) r.xf[q] = 0.0;
    for (int q = 0; q < 7; ++q) {
        r.xf[q] = value(xi[q]);
        finite = finite && std::isfinite(r.xf[q]);
    }
    if (!finite) {
        r.flags |= ORC_NONFINITE;
        J = T(INFINITY);
    }
    if (finite && value(margin) > 0.0) r.flags |= ORC_FEASIBLE;
    r.J = J;
    r.margin = margin;
    r.min_step = min_step;
    return r;
}

}  // namespace orcm
