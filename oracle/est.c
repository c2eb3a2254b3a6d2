/*
 * est.c - FP64 oracle of the extended single-track (EST) planar vehicle
 * model of arxiv 2603.20525 (App. "Extended Single-Track Vehicle Dynamics
 * Model") with the lateral-acceleration soft constraint of Sec. IV-C: the
 * planar formulation the paper sets beside the SRB model, with the same
 * cost, zero-order hold, Euler steps, goal truncation and argmin.
 *
 * TEST INFRASTRUCTURE: only the test suite may call this.  It shares no code
 * with the CUDA path.
 *
 * Readings (beside Q1-Q14 of the SRB oracle):
 *   Q1  the terrain normal is proportional to (-f_x, -f_y, 1), as for the SRB
 *       model; pitch and roll follow from it through the 1-2-3 convention:
 *       theta = asin(tau_x), phi = atan2(-tau_y, tau_z);
 *   Q15 the slip angles use atan2(., v_Bx), equal to the paper's arctan of the
 *       quotient while v_Bx > 0;
 *   Q16 the lateral-acceleration margin abar - |a_By - g_By| is evaluated
 *       with each integrated Euler step (it needs the held control); frozen
 *       states after the goal and the final state add nothing; a candidate is
 *       feasible when its minimum margin is > 0 and its rollout finite;
 *   Q2  eps of the constraint defaults to 10 % of abar = M g / (2 K_zy);
 *   Q17 the planar model reads the terrain under the CoM only, and the
 *       costmap under the four wheels when a costmap is given; the off-map
 *       flag covers the reads that happen.
 */
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

/* EST state indices (the paper's order) */
enum { EX = 0, EY, EPSI, EVY, EWZ, EDELTA, EVX };

typedef struct {
    double Kzzf, Kzzr, Kzx, Kzy;   /* load-transfer coefficients */
    double abar, eps;              /* critical lateral acceleration, normaliser */
    double rho[4][3];              /* wheel contact points in B: fl, fr, rl, rr */
} est_consts;

static void est_make(const orc_vehicle *v, const orc_cost *c, est_consts *k)
{
    const double L = v->Lf + v->Lr;
    k->Kzzf = v->M * v->Lr / L;
    k->Kzzr = v->M * v->Lf / L;
    k->Kzx = v->M * v->hR / L;
    k->Kzy = v->M * v->hR / v->e;
    k->abar = v->M * v->g / (2.0 * k->Kzy);
    k->eps = c->eps_esm > 0.0 ? c->eps_esm : 0.1 * k->abar;
    for (int i = 0; i < 4; ++i) {
        k->rho[i][0] = i < 2 ? v->Lf : -v->Lr;
        k->rho[i][1] = (i & 1) ? -0.5 * v->e : 0.5 * v->e;
        k->rho[i][2] = -v->hR;
    }
}

static double clampv(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* The 1-2-3 rotation (roll phi about w_x, pitch theta, yaw psi about b_z),
 * body -> world, row-major, as printed with the EST model. */
void orc_est_rotation(double phi, double theta, double psi, double R[9])
{
    const double cf = cos(phi), sf = sin(phi), ct = cos(theta), st = sin(theta);
    const double cp = cos(psi), sp = sin(psi);
    R[0] = ct * cp;
    R[1] = -ct * sp;
    R[2] = st;
    R[3] = cf * sp + cp * sf * st;
    R[4] = cf * cp - sf * st * sp;
    R[5] = -ct * sf;
    R[6] = sf * sp - cf * cp * st;
    R[7] = cp * sf + cf * st * sp;
    R[8] = cf * ct;
}

/* State derivative A(xi) + B zeta, running cost rate, lateral margin.
 * diag (ORC_EST_FIELDS, may be NULL): 0 theta  1 phi  2-4 g_B  5 a_Bx
 * 6 F_zf  7 F_zr  8 alpha_f  9 alpha_r  10 F_yf  11 F_yr  12 a_By
 * 13 margin  14 L  15-18 costmap at fl, fr, rl, rr.  Returns 1 if a lookup
 * left the map. */
static int est_derivative(const orc_vehicle *v, const est_consts *k, const orc_cost *c,
                          const orc_terrain *t, const double xi[7], const double zeta[2],
                          double xidot[7], double *L_out, double *margin_out, double *diag)
{
    double ter[4], R[9];
    int off = orc_terrain_sample(t, xi[EX], xi[EY], ter);
    /* unit normal of the local plane under the CoM (reading Q1) */
    const double n = sqrt(ter[1] * ter[1] + ter[2] * ter[2] + 1.0);
    const double tau[3] = {-ter[1] / n, -ter[2] / n, 1.0 / n};
    const double theta = asin(tau[0]);
    const double phi = atan2(-tau[1], tau[2]);
    orc_est_rotation(phi, theta, xi[EPSI], R);
    /* gravity in B: R^T (0, 0, -g) */
    const double gB[3] = {-v->g * R[6], -v->g * R[7], -v->g * R[8]};
    const double vx = xi[EVX], vy = xi[EVY], wz = xi[EWZ], delta = xi[EDELTA];
    /* longitudinal acceleration and the virtual tires' normal forces */
    const double aBx = zeta[1] - wz * vy;
    const double Fzf = -k->Kzzf * gB[2] - k->Kzx * aBx;
    const double Fzr = -k->Kzzr * gB[2] + k->Kzx * aBx;
    /* slip angles (reading Q15) and the sigmoid tire */
    const double af = atan2(vy + wz * v->Lf, vx) - delta;
    const double ar = atan2(vy - wz * v->Lr, vx);
    const double Fyf = Fzf * orc_tire(v->C, v->mu, af);
    const double Fyr = Fzr * orc_tire(v->C, v->mu, ar);
    /* A(xi) + B zeta */
    xidot[EX] = R[0] * vx + R[1] * vy;
    xidot[EY] = R[3] * vx + R[4] * vy;
    xidot[EPSI] = wz;
    xidot[EVY] = (Fyf + Fyr) / v->M + gB[1] - wz * vx;
    xidot[EWZ] = (Fyf * v->Lf * cos(delta) - Fyr * v->Lr) / v->Jzz;
    xidot[EDELTA] = zeta[0];
    xidot[EVX] = zeta[1];
    /* lateral acceleration and the constraint |a_By - g_By| < abar */
    const double aBy = xidot[EVY] + wz * vx;
    const double margin = k->abar - fabs(aBy - gB[1]);
    const double viol = 1.0 - margin / k->eps;          /* 1 + pi / eps, pi = -margin */
    double L = c->wt + c->wc * zeta[0] * zeta[0];
    if (viol > 0.0) L += c->sigma * viol * viol;
    /* distance constraints: the costmap under each wheel (reading Q17: read
     * only when there is a costmap) */
    double cm[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < 4 && t->costmap; ++i) {
        const double px = xi[EX] + R[0] * k->rho[i][0] + R[1] * k->rho[i][1] + R[2] * k->rho[i][2];
        const double py = xi[EY] + R[3] * k->rho[i][0] + R[4] * k->rho[i][1] + R[5] * k->rho[i][2];
        double w[4];
        off |= orc_terrain_sample(t, px, py, w);
        cm[i] = w[3];
        L += cm[i];
    }
    *L_out = L;
    *margin_out = margin;
    if (diag) {
        const double d[ORC_EST_FIELDS] = {theta, phi, gB[0], gB[1], gB[2], aBx, Fzf, Fzr, af, ar,
                                          Fyf, Fyr, aBy, margin, L, cm[0], cm[1], cm[2], cm[3]};
        memcpy(diag, d, sizeof d);
    }
    return off;
}

void orc_est_eval(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double xi[7],
                  const double zeta[2], double xidot[7], double *diag)
{
    est_consts k;
    double L, m;
    est_make(v, c, &k);
    est_derivative(v, &k, c, t, xi, zeta, xidot, &L, &m, diag);
}

static void est_one(const orc_vehicle *v, const est_consts *k, const orc_cost *c,
                    const orc_terrain *t, const double x0[7], const float *ctrl, int ctrl_stride,
                    int H, double dt, int n_sub, double *J_out, double *margin_out,
                    unsigned char *flags_out, double *xf, double *step_margin, int sm_stride,
                    double *diag, double *states)
{
    double xi[7], xidot[7];
    const double h = dt / (double)n_sub;
    double J = 0.0, margin = INFINITY, d_ay = INFINITY, d_goal = INFINITY;
    int done = 0, off = 0, step = 0;
    memcpy(xi, x0, sizeof xi);
    if (states) memcpy(states, xi, sizeof xi);
    for (int kk = 0; kk < H; ++kk) {
        double zeta[2], sm = INFINITY;
        zeta[0] = clampv((double)ctrl[(size_t)kk * ctrl_stride], -v->delta_rate_max, v->delta_rate_max);
        zeta[1] = (double)ctrl[(size_t)kk * ctrl_stride + 1];
        for (int s = 0; s < n_sub; ++s) {
            if (!done) {
                const double gd = hypot(xi[EX] - c->goal_x, xi[EY] - c->goal_y);
                if (fabs(gd - c->goal_r) < d_goal) d_goal = fabs(gd - c->goal_r);
                if (gd <= c->goal_r) done = 1;
            }
            if (!done) {
                double L, m;
                off |= est_derivative(v, k, c, t, xi, zeta, xidot, &L, &m, NULL);
                if (m < margin) margin = m;
                if (m < sm) sm = m;
                if (fabs(m) / k->abar < d_ay) d_ay = fabs(m) / k->abar;
                J += h * L;
                for (int q = 0; q < 7; ++q) xi[q] += h * xidot[q];
                xi[EDELTA] = clampv(xi[EDELTA], -v->delta_max, v->delta_max);
            }
            ++step;
            if (states) memcpy(states + (size_t)step * 7, xi, sizeof xi);
        }
        if (step_margin) step_margin[(size_t)kk * sm_stride] = sm;
    }
    {
        const double gd = hypot(xi[EX] - c->goal_x, xi[EY] - c->goal_y);
        if (!done) {
            if (fabs(gd - c->goal_r) < d_goal) d_goal = fabs(gd - c->goal_r);
            if (gd <= c->goal_r) done = 1;
        }
        J += c->wg * gd;
    }
    unsigned char fl = 0;
    int finite = isfinite(J);
    for (int q = 0; q < 7; ++q) finite = finite && isfinite(xi[q]);
    if (done) fl |= ORC_DONE;
    if (off) fl |= ORC_OFFMAP;
    if (!finite) {
        fl |= ORC_NONFINITE;
        J = INFINITY;
    }
    if (finite && margin > 0.0) fl |= ORC_FEASIBLE;
    *J_out = J;
    *margin_out = margin;
    *flags_out = fl;
    if (xf) memcpy(xf, xi, sizeof xi);
    if (diag) {
        diag[0] = INFINITY;      /* no contact switch in the planar model */
        diag[1] = d_ay;
        diag[2] = d_goal;
    }
}

int orc_est_rollout(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const float *x0,
                    int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub, double *J,
                    double *margin, unsigned char *flags, double *xf, double *step_margin, double *diag,
                    int nthreads)
{
    est_consts k;
    if (N <= 0 || H <= 0 || n_sub <= 0 || !(dt > 0.0)) return -1;
    est_make(v, c, &k);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads)
#endif
    for (int j = 0; j < N; ++j) {
        double xs[7];
        const float *src = x0 + (x0_per_cand ? (size_t)j * 7 : 0);
        for (int q = 0; q < 7; ++q) xs[q] = (double)src[q];
        est_one(v, &k, c, t, xs, ctrl + (size_t)j * 2, 2 * N, H, dt, n_sub, &J[j], &margin[j],
                &flags[j], xf ? xf + (size_t)j * 7 : NULL, step_margin ? step_margin + j : NULL, N,
                diag ? diag + (size_t)j * 3 : NULL, NULL);
    }
    (void)nthreads;
    return 0;
}

int orc_est_trajectory(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                       const double x0[7], const float *ctrl, int H, double dt, int n_sub,
                       double *states)
{
    est_consts k;
    double J, m;
    unsigned char fl;
    if (H <= 0 || n_sub <= 0 || !(dt > 0.0)) return -1;
    est_make(v, c, &k);
    est_one(v, &k, c, t, x0, ctrl, 2, H, dt, n_sub, &J, &m, &fl, NULL, NULL, 0, NULL, states);
    return 0;
}
