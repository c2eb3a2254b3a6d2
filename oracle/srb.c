/*
 * srb.c - FP64 CPU oracle of the SRB rollout planner of arxiv 2603.20525.
 *
 * TEST INFRASTRUCTURE.  This file checks the CUDA path; only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it, and
 * the product never routes through it.  It shares no code with the CUDA path.
 *
 * The model is written out plainly, in the paper's order and notation:
 *   Sec. IV-A  single-rigid-body model: state, A(xi) + B zeta, 3-2-1 rotation,
 *              Euler-angle rates, wheel contact kinematics, suspension
 *              extension chi and rate, spring/damper with liftoff, slip angle,
 *              summed forces and moments, rear longitudinal constraint force;
 *   Sec. III-A sigmoid tire model and the vertical load-transfer coefficients
 *              K_zz,f = M L_r / (L_f + L_r), K_zz,r = M L_f / (L_f + L_r);
 *   Sec. IV-B  energy stability margin;
 *   Sec. IV-C  cost J = int L dt + Phi, L = L_0 + L_soft, goal truncation,
 *              zero-order hold of the controls, admissible control set;
 *   Sec. IV-D  forward Euler at a step of at most 5 ms, empirical argmin.
 */
#include "oracle.h"

#include <math.h>
#include <stddef.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* state indices, in the order of the SRB state vector (Sec. IV-A) */
enum { X = 0, Y, Z, PSI, THETA, PHI, VX, VY, VZ, WX, WY, WZ, DELTA };
/* wheels fl, fr, rl, rr (Sec. IV-A) */
enum { FL = 0, FR, RL, RR };

typedef struct {
    double Kzz[4];     /* vertical load-transfer coefficient of each wheel */
    double Fs[4];      /* nominal tire loading F_s,i = (g/2) K_zz,i */
    double k[4], b[4]; /* spring, damper of each wheel */
    double rho[4][3];  /* contact point of each wheel in B */
    double U0;         /* U_ESM on level ground */
    double eps_esm;    /* ESM soft-constraint normaliser */
} orc_consts;

static double clampd(double v, double lo, double hi)
{
    if (v < lo) return lo;
    if (v > hi) return hi;
    return v;
}

static void cross(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* Sec. IV-A: rotation matrix of the 3-2-1 (Z-Y-X) Euler angles, body->world */
void orc_rotation(double psi, double theta, double phi, double R[9])
{
    double cps = cos(psi), sps = sin(psi);
    double cth = cos(theta), sth = sin(theta);
    double cph = cos(phi), sph = sin(phi);
    R[0] = cps * cth;
    R[1] = cps * sph * sth - cph * sps;
    R[2] = sph * sps + cph * cps * sth;
    R[3] = cth * sps;
    R[4] = cph * cps + sph * sps * sth;
    R[5] = cph * sps * sth - cps * sph;
    R[6] = -sth;
    R[7] = cth * sph;
    R[8] = cph * cth;
}

/* Sec. III-A: sigmoid tire model, F_y / F_z = -C alpha mu / sqrt(mu^2 + (C alpha)^2) */
double orc_tire(double C, double mu, double alpha)
{
    double Ca = C * alpha;
    double den = sqrt(mu * mu + Ca * Ca);
    if (den == 0.0) return 0.0;   /* mu = 0 and C alpha = 0: no lateral force */
    return -Ca * mu / den;
}

/* Sec. IV-B: Delta h = Rbar (1 - sin(|phi| + phibar)) cos(theta),
 * Rbar = sqrt((h+R)^2 + (e/2)^2), phibar = atan(2 (h+R) / e);
 * U = +M g Delta h while the CoM is inside the footprint, -M g Delta h outside.
 * Inside the footprint (rollover about a side edge, the paper's assumption)
 * means |phi| + phibar < pi/2. */
double orc_esm(const orc_vehicle *v, double phi, double theta)
{
    double Rbar = sqrt(v->hR * v->hR + 0.25 * v->e * v->e);
    double phibar = atan(2.0 * v->hR / v->e);
    double a = fabs(phi) + phibar;
    double dh = Rbar * (1.0 - sin(a)) * cos(theta);
    double s = (a < 0.5 * M_PI) ? 1.0 : -1.0;
    return s * v->M * v->g * dh;
}

static void make_consts(const orc_vehicle *v, const orc_cost *c, orc_consts *k)
{
    double L = v->Lf + v->Lr;
    double Kzzf = v->M * v->Lr / L;   /* Sec. III-A, front vertical load transfer */
    double Kzzr = v->M * v->Lf / L;   /* Sec. III-A, rear vertical load transfer */
    double half_e = 0.5 * v->e;
    int i;
    k->Kzz[FL] = k->Kzz[FR] = Kzzf;
    k->Kzz[RL] = k->Kzz[RR] = Kzzr;
    for (i = 0; i < 4; ++i) k->Fs[i] = 0.5 * v->g * k->Kzz[i];
    k->k[FL] = k->k[FR] = v->kf;
    k->k[RL] = k->k[RR] = v->kr;
    k->b[FL] = k->b[FR] = v->bf;
    k->b[RL] = k->b[RR] = v->br;
    /* contact-point offsets rho^i in B (Sec. IV-A) */
    k->rho[FL][0] = v->Lf;  k->rho[FL][1] = half_e;  k->rho[FL][2] = -v->hR;
    k->rho[FR][0] = v->Lf;  k->rho[FR][1] = -half_e; k->rho[FR][2] = -v->hR;
    k->rho[RL][0] = -v->Lr; k->rho[RL][1] = half_e;  k->rho[RL][2] = -v->hR;
    k->rho[RR][0] = -v->Lr; k->rho[RR][1] = -half_e; k->rho[RR][2] = -v->hR;
    k->U0 = orc_esm(v, 0.0, 0.0);
    k->eps_esm = (c && c->eps_esm > 0.0) ? c->eps_esm : 0.1 * k->U0;
}

/* ------------------------------------------------------------------------ */
/* Terrain (reading Q10): node gradients by central differences, one-sided on
 * the border; bilinear interpolation of heights, gradients and costmap. */
void orc_terrain_gradients(const float *H, int nx, int ny, double cell,
                           double *gx, double *gy)
{
    int i, j;
    for (j = 0; j < ny; ++j) {
        for (i = 0; i < nx; ++i) {
            double a, b;
            if (i == 0)           { a = H[j * nx + 1];      b = H[j * nx + 0];      gx[j * nx + i] = (a - b) / cell; }
            else if (i == nx - 1) { a = H[j * nx + nx - 1]; b = H[j * nx + nx - 2]; gx[j * nx + i] = (a - b) / cell; }
            else                  { a = H[j * nx + i + 1];  b = H[j * nx + i - 1];  gx[j * nx + i] = (a - b) / (2.0 * cell); }
            if (j == 0)           { a = H[1 * nx + i];        b = H[0 * nx + i];        gy[j * nx + i] = (a - b) / cell; }
            else if (j == ny - 1) { a = H[(ny - 1) * nx + i]; b = H[(ny - 2) * nx + i]; gy[j * nx + i] = (a - b) / cell; }
            else                  { a = H[(j + 1) * nx + i];  b = H[(j - 1) * nx + i];  gy[j * nx + i] = (a - b) / (2.0 * cell); }
        }
    }
}

int orc_terrain_sample(const orc_terrain *t, double x, double y, double out[4])
{
    double u = (x - t->x0) / t->cell;
    double w = (y - t->y0) / t->cell;
    double umax = (double)(t->nx - 1), wmax = (double)(t->ny - 1);
    int off = !(u >= 0.0 && u <= umax && w >= 0.0 && w <= wmax);
    int i, j, i1, j1;
    double a, b, w00, w10, w01, w11;
    if (isnan(u)) u = 0.0;
    if (isnan(w)) w = 0.0;
    u = clampd(u, 0.0, umax);
    w = clampd(w, 0.0, wmax);
    i = (int)floor(u);
    j = (int)floor(w);
    if (i > t->nx - 2) i = t->nx - 2;
    if (j > t->ny - 2) j = t->ny - 2;
    a = u - i;
    b = w - j;
    i1 = i + 1;
    j1 = j + 1;
    w00 = (1.0 - a) * (1.0 - b);
    w10 = a * (1.0 - b);
    w01 = (1.0 - a) * b;
    w11 = a * b;
#define BIL(arr) (w00 * (double)(arr)[j * t->nx + i] + w10 * (double)(arr)[j * t->nx + i1] + \
                  w01 * (double)(arr)[j1 * t->nx + i] + w11 * (double)(arr)[j1 * t->nx + i1])
    out[0] = BIL(t->heights);
    out[1] = BIL(t->gx);
    out[2] = BIL(t->gy);
    out[3] = t->costmap ? BIL(t->costmap) : 0.0;
#undef BIL
    return off;
}

/* ------------------------------------------------------------------------ */
/* The SRB state derivative (Sec. IV-A) and the running cost rate (Sec. IV-C).
 * Returns 1 if any wheel queried the terrain off the map. */
static int srb_derivative(const orc_vehicle *v, const orc_consts *k, const orc_cost *c,
                          const orc_terrain *t, const double xi[13], const double zeta[2],
                          double xidot[13], double *L_out, double *wheel, double *body,
                          double *contact_dist)
{
    double R[9];
    double gB[3];
    double vB[3] = { xi[VX], xi[VY], xi[VZ] };
    double w[3] = { xi[WX], xi[WY], xi[WZ] };
    double wxbz[3];                 /* omega x b_z, resolved in B: (w_y, -w_x, 0) */
    double delta = xi[DELTA];
    double Fy_sum = 0.0, Fz_sum = 0.0, Msum[3] = { 0.0, 0.0, 0.0 };
    double cost_map = 0.0;
    double U, L0, Lsoft;
    double sphi, cphi, sth, cth;
    int i, off = 0;
    double ez[3] = { 0.0, 0.0, 1.0 };

    /* rotation and gravity resolved in B: g_B = R^T (0, 0, -g) */
    orc_rotation(xi[PSI], xi[THETA], xi[PHI], R);
    gB[0] = -v->g * R[6];
    gB[1] = -v->g * R[7];
    gB[2] = -v->g * R[8];
    cross(w, ez, wxbz);

    for (i = 0; i < 4; ++i) {
        const double *rho = k->rho[i];
        double P[3], wr[3], vi[3], ter[4], tauW[3], tauB[3], rel[3];
        double chi, chidot, Fk, Fb, Fz, alpha, di, Fy, Fx, Fvec[3], m[3];
        int woff;
        /* contact point in W and its velocity in B (Sec. IV-A) */
        P[0] = xi[X] + R[0] * rho[0] + R[1] * rho[1] + R[2] * rho[2];
        P[1] = xi[Y] + R[3] * rho[0] + R[4] * rho[1] + R[5] * rho[2];
        P[2] = xi[Z] + R[6] * rho[0] + R[7] * rho[1] + R[8] * rho[2];
        cross(w, rho, wr);
        vi[0] = vB[0] + wr[0];
        vi[1] = vB[1] + wr[1];
        vi[2] = vB[2] + wr[2];
        /* terrain height and slope below the nominal contact point */
        woff = orc_terrain_sample(t, P[0], P[1], ter);
        off |= woff;
        /* slope-normal direction (reading Q1): tau ~ (-f_x, -f_y, 1) in W */
        tauW[0] = -ter[1];
        tauW[1] = -ter[2];
        tauW[2] = 1.0;
        tauB[0] = R[0] * tauW[0] + R[3] * tauW[1] + R[6] * tauW[2];
        tauB[1] = R[1] * tauW[0] + R[4] * tauW[1] + R[7] * tauW[2];
        tauB[2] = R[2] * tauW[0] + R[5] * tauW[1] + R[8] * tauW[2];
        /* suspension extension and its rate */
        chi = (P[2] - ter[0]) / tauB[2];
        rel[0] = vi[0] - chi * wxbz[0];
        rel[1] = vi[1] - chi * wxbz[1];
        rel[2] = vi[2] - chi * wxbz[2];
        chidot = (tauB[0] * rel[0] + tauB[1] * rel[1] + tauB[2] * rel[2]) / tauB[2];
        /* spring and damper with liftoff: never attractive */
        Fk = k->Fs[i] - k->k[i] * chi;
        if (Fk < 0.0) Fk = 0.0;
        if (Fk > 0.0) {
            Fb = -k->b[i] * chidot;
            if (Fb < -Fk) Fb = -Fk;
        } else {
            Fb = 0.0;
        }
        Fz = Fk + Fb;
        if (contact_dist) {
            double d = fabs(k->Fs[i] - k->k[i] * chi) / k->Fs[i];
            if (d < *contact_dist) *contact_dist = d;
        }
        /* slip angle and lateral tire force */
        di = (i == FL || i == FR) ? delta : 0.0;
        alpha = atan2(vi[1], vi[0]) - di;
        Fy = Fz * orc_tire(v->C, v->mu, alpha);
        /* rear longitudinal constraint force that holds the prescribed v_x rate */
        if (i == RL || i == RR)
            Fx = 0.5 * v->M * (zeta[1] - gB[0] + w[1] * vB[2] - w[2] * vB[1]);
        else
            Fx = 0.0;
        /* summed forces and moments */
        Fy_sum += Fy * cos(di);
        Fz_sum += Fz;
        Fvec[0] = Fx;
        Fvec[1] = Fy * cos(di);
        Fvec[2] = Fz;
        cross(rho, Fvec, m);
        Msum[0] += m[0];
        Msum[1] += m[1];
        Msum[2] += m[2];
        cost_map += ter[3];
        if (wheel) {
            double *o = wheel + i * ORC_WHEEL_FIELDS;
            o[0] = P[0]; o[1] = P[1]; o[2] = P[2];
            o[3] = vi[0]; o[4] = vi[1]; o[5] = vi[2];
            o[6] = ter[0]; o[7] = ter[1]; o[8] = ter[2]; o[9] = ter[3];
            o[10] = tauB[0]; o[11] = tauB[1]; o[12] = tauB[2];
            o[13] = chi; o[14] = chidot; o[15] = Fk; o[16] = Fb; o[17] = Fz;
            o[18] = alpha; o[19] = Fy; o[20] = Fx; o[21] = (double)woff;
        }
    }

    /* A(xi) + B zeta (Sec. IV-A) */
    sphi = sin(xi[PHI]);
    cphi = cos(xi[PHI]);
    sth = sin(xi[THETA]);
    cth = cos(xi[THETA]);
    /* position rates: world velocity v_W = R v_B */
    xidot[X] = R[0] * vB[0] + R[1] * vB[1] + R[2] * vB[2];
    xidot[Y] = R[3] * vB[0] + R[4] * vB[1] + R[5] * vB[2];
    xidot[Z] = R[6] * vB[0] + R[7] * vB[1] + R[8] * vB[2];
    /* Euler-angle rates from body angular velocity */
    xidot[PSI] = (sphi / cth) * w[1] + (cphi / cth) * w[2];
    xidot[THETA] = cphi * w[1] - sphi * w[2];
    xidot[PHI] = w[0] + (sphi * sth / cth) * w[1] + (cphi * sth / cth) * w[2];
    /* prescribed longitudinal velocity rate enters through B */
    xidot[VX] = zeta[1];
    xidot[VY] = Fy_sum / v->M + gB[1] + w[0] * vB[2] - w[2] * vB[0];
    xidot[VZ] = Fz_sum / v->M + gB[2] - w[0] * vB[1] + w[1] * vB[0];
    xidot[WX] = (Msum[0] + (v->Jyy - v->Jzz) * w[1] * w[2]) / v->Jxx;
    xidot[WY] = (Msum[1] - (v->Jxx - v->Jzz) * w[0] * w[2]) / v->Jyy;
    xidot[WZ] = (Msum[2] + (v->Jxx - v->Jyy) * w[0] * w[1]) / v->Jzz;
    xidot[DELTA] = zeta[0];

    /* running cost rate L = L_0 + L_soft (Sec. IV-C) with pi_ESM = -U_ESM */
    U = orc_esm(v, xi[PHI], xi[THETA]);
    L0 = c->wt + c->wc * zeta[0] * zeta[0];
    {
        double s = 1.0 - U / k->eps_esm;
        if (s < 0.0) s = 0.0;
        Lsoft = c->sigma * s * s + cost_map;
    }
    if (L_out) *L_out = L0 + Lsoft;
    if (body) {
        for (i = 0; i < 9; ++i) body[i] = R[i];
        body[9] = gB[0]; body[10] = gB[1]; body[11] = gB[2];
        body[12] = Fy_sum; body[13] = Fz_sum;
        body[14] = Msum[0]; body[15] = Msum[1]; body[16] = Msum[2];
        body[17] = U; body[18] = L0 + Lsoft;
        for (i = 0; i < 4; ++i) body[19 + i] = k->Fs[i];
    }
    return off;
}

void orc_eval(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
              const double xi[13], const double zeta[2], double xidot[13],
              double *wheel, double *body)
{
    orc_consts k;
    double L;
    make_consts(v, c, &k);
    srb_derivative(v, &k, c, t, xi, zeta, xidot, &L, wheel, body, NULL);
}

/* ------------------------------------------------------------------------ */
static double goal_dist(const orc_cost *c, const double xi[13])
{
    double dx = xi[X] - c->goal_x, dy = xi[Y] - c->goal_y;
    return sqrt(dx * dx + dy * dy);
}

static int all_finite(const double *a, int n)
{
    int i;
    for (i = 0; i < n; ++i)
        if (!isfinite(a[i])) return 0;
    return 1;
}

/* One candidate: the forward-Euler rollout with zero-order-hold controls,
 * goal truncation, ESM margin and cost (Sec. IV-C, IV-D). */
static void rollout_one(const orc_vehicle *v, const orc_consts *k, const orc_cost *c,
                        const orc_terrain *t, const double x0[13], const float *ctrl,
                        int ctrl_stride, int H, double dt, int n_sub,
                        double *J_out, double *margin_out, unsigned char *flags_out,
                        double *xf, double *step_margin, int sm_stride, double *diag,
                        double *states, double *Jrun, int *done_step)
{
    double xi[13], xidot[13];
    double h = dt / (double)n_sub;
    double J = 0.0, margin = INFINITY;
    double d_contact = INFINITY, d_esm = INFINITY, d_goal = INFINITY;
    int done = 0, off = 0, kk, s, q, step = 0;
    unsigned char flags = 0;

    memcpy(xi, x0, sizeof xi);
    if (done_step) *done_step = -1;
    if (states) memcpy(states, xi, sizeof xi);
    if (Jrun) Jrun[0] = 0.0;

    for (kk = 0; kk < H; ++kk) {
        /* zero-order hold; admissible set |delta_dot| <= delta_rate_max */
        double zeta[2];
        double sm = INFINITY;
        zeta[0] = clampd((double)ctrl[(size_t)kk * ctrl_stride + 0], -v->delta_rate_max, v->delta_rate_max);
        zeta[1] = (double)ctrl[(size_t)kk * ctrl_stride + 1];
        for (s = 0; s < n_sub; ++s) {
            double U = orc_esm(v, xi[PHI], xi[THETA]);
            double gd;
            if (U < margin) margin = U;
            if (U < sm) sm = U;
            if (fabs(U) / k->U0 < d_esm) d_esm = fabs(U) / k->U0;
            if (!done) {
                gd = goal_dist(c, xi);
                if (fabs(gd - c->goal_r) < d_goal) d_goal = fabs(gd - c->goal_r);
                if (gd <= c->goal_r) {
                    done = 1;
                    if (done_step) *done_step = step;
                }
            }
            if (!done) {
                double L;
                off |= srb_derivative(v, k, c, t, xi, zeta, xidot, &L, NULL, NULL, &d_contact);
                J += h * L;
                for (q = 0; q < 13; ++q) xi[q] += h * xidot[q];
                xi[DELTA] = clampd(xi[DELTA], -v->delta_max, v->delta_max);
            }
            ++step;
            if (states) memcpy(states + (size_t)step * 13, xi, sizeof xi);
            if (Jrun) Jrun[step] = J;
        }
        if (step_margin) step_margin[(size_t)kk * sm_stride] = sm;
    }
    /* final state: margin and goal test, then the terminal cost Phi */
    {
        double U = orc_esm(v, xi[PHI], xi[THETA]);
        double gd = goal_dist(c, xi);
        if (U < margin) margin = U;
        if (fabs(U) / k->U0 < d_esm) d_esm = fabs(U) / k->U0;
        if (step_margin && H > 0) {
            double *p = &step_margin[(size_t)(H - 1) * sm_stride];
            if (U < *p) *p = U;
        }
        if (!done) {
            if (fabs(gd - c->goal_r) < d_goal) d_goal = fabs(gd - c->goal_r);
            if (gd <= c->goal_r) {
                done = 1;
                if (done_step) *done_step = step;
            }
        }
        J += c->wg * gd;
    }
    if (done) flags |= ORC_DONE;
    if (off) flags |= ORC_OFFMAP;
    if (!isfinite(J) || !all_finite(xi, 13)) {
        flags |= ORC_NONFINITE;
        J = INFINITY;
    }
    if (margin > 0.0 && !(flags & ORC_NONFINITE)) flags |= ORC_FEASIBLE;
    *J_out = J;
    *margin_out = margin;
    *flags_out = flags;
    if (xf) memcpy(xf, xi, sizeof xi);
    if (diag) {
        diag[0] = d_contact;
        diag[1] = d_esm;
        diag[2] = d_goal;
    }
}

int orc_rollout(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                const float *x0, int x0_per_cand, const float *ctrl,
                int N, int H, double dt, int n_sub,
                double *J, double *margin, unsigned char *flags,
                double *xf, double *step_margin, double *diag, int nthreads)
{
    orc_consts k;
    int j;
    if (N <= 0 || H <= 0 || n_sub <= 0 || !(dt > 0.0)) return -1;
    make_consts(v, c, &k);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
#endif
    for (j = 0; j < N; ++j) {
        double xs[13];
        int q;
        const float *src = x0 + (x0_per_cand ? (size_t)j * 13 : 0);
        for (q = 0; q < 13; ++q) xs[q] = (double)src[q];
        rollout_one(v, &k, c, t, xs, ctrl + (size_t)j * 2, 2 * N, H, dt, n_sub,
                    &J[j], &margin[j], &flags[j],
                    xf ? xf + (size_t)j * 13 : NULL,
                    step_margin ? step_margin + j : NULL, N,
                    diag ? diag + (size_t)j * 3 : NULL, NULL, NULL, NULL);
    }
    (void)nthreads;
    return 0;
}

int orc_trajectory(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                   const double x0[13], const float *ctrl, int H, double dt, int n_sub,
                   double *states, double *Jrun)
{
    orc_consts k;
    double J, margin;
    unsigned char flags;
    int done_step;
    make_consts(v, c, &k);
    rollout_one(v, &k, c, t, x0, ctrl, 2, H, dt, n_sub, &J, &margin, &flags,
                NULL, NULL, 0, NULL, states, Jrun, &done_step);
    return done_step;
}

/* Empirical argmin (Sec. IV-D), reading Q7: feasible candidates first, then
 * the smaller cost, then the smaller index. */
int orc_select(const double *J, const unsigned char *flags, int N)
{
    int best = -1, j;
    for (j = 0; j < N; ++j) {
        int inf_j = !(flags[j] & ORC_FEASIBLE);
        if (best < 0) {
            best = j;
            continue;
        }
        {
            int inf_b = !(flags[best] & ORC_FEASIBLE);
            if (inf_j < inf_b || (inf_j == inf_b && J[j] < J[best])) best = j;
        }
    }
    return best;
}
