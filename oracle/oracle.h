/*
 * oracle.h - FP64 CPU oracle of the sampling MPC hot path of arxiv 2603.20525
 * ("High-Speed, All-Terrain Autonomy: Ensuring Safety at the Limits of
 * Mobility"): the single-rigid-body (SRB) vehicle rollout on a heightmap
 * (Sec. IV-A), the energy stability margin (ESM) constraint (Sec. IV-B),
 * the cost (Sec. IV-C) and the empirical argmin (Sec. IV-D).
 *
 * TEST INFRASTRUCTURE.  This library exists to check the CUDA path.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA path, and
 * the product never falls back to it.
 *
 * Everything is plain, slow FP64 C written in the order the paper states the
 * model.  Where the paper is silent or ambiguous the oracle follows one
 * documented reading (the same list is kept in the design notes):
 *   Q1  terrain normal of z = f(x, y) is proportional to (-f_x, -f_y, 1);
 *   Q2  eps_esm defaults to 10 % of the level-ground ESM;
 *   Q3  dt is the zero-order-hold interval, integrated by n_sub Euler steps;
 *   Q4  the goal test runs before every Euler step and on the final state;
 *       a candidate that reached the goal is frozen;
 *   Q5  the steering angle is clamped to +/-delta_max after every step, the
 *       steering rate to +/-delta_rate_max before use;
 *   Q6  running cost is a left Riemann sum; the margin covers every state
 *       visited, the final one included;
 *   Q7  best = lexicographic minimum of (infeasible, J, index);
 *   Q10 bilinear heights; node gradients by central differences (one-sided
 *       at the border), bilinearly interpolated; queries clamped to the map;
 *   Q11 slip angle uses atan2.
 */
#ifndef ALLTERRAIN_ORACLE_H
#define ALLTERRAIN_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Vehicle parameters, SI units (App. A notation table, App. B). */
typedef struct {
    double M, Jxx, Jyy, Jzz;       /* mass, principal inertias about b_x, b_y, b_z */
    double Lf, Lr, e, hR;          /* CoM to front / rear axle, track, h + R */
    double kf, kr, bf, br;         /* spring and damper rates, front / rear */
    double C, mu;                  /* sigmoid tire model (Sec. III-A) */
    double delta_max, delta_rate_max, g;
} orc_vehicle;

/* Cost weights (Sec. IV-C). eps_esm <= 0 selects 0.1 * U_ESM(level). */
typedef struct {
    double wt, wc, wg, sigma, eps_esm, goal_x, goal_y, goal_r;
} orc_cost;

/* Heightmap heights[j][i] = f(x0 + i cell, y0 + j cell).  gx, gy are the node
 * gradients made by orc_terrain_gradients (caller-owned).  costmap is an
 * optional summed soft-constraint cost-rate map sampled at every wheel. */
typedef struct {
    const float *heights;
    const double *gx, *gy;
    const float *costmap;
    int nx, ny;
    double cell, x0, y0;
} orc_terrain;

/* flags per candidate */
#define ORC_FEASIBLE  1u
#define ORC_DONE      2u
#define ORC_OFFMAP    4u
#define ORC_NONFINITE 8u

/* Per-wheel diagnostics written by orc_eval, ORC_WHEEL_FIELDS doubles per wheel:
 *  0-2 P (world)  3-5 v^i (body)  6 f  7 f_x  8 f_y  9 costmap  10-12 tau (body)
 *  13 chi  14 chi_dot  15 F_k  16 F_b  17 F_z  18 alpha  19 F_y  20 F_x  21 off-map */
#define ORC_WHEEL_FIELDS 22
/* Body diagnostics: 0-8 R (row-major)  9-11 g_B  12 F_y  13 F_z  14-16 M
 *  17 U_ESM  18 L (running cost rate)  19-22 F_s per wheel */
#define ORC_BODY_FIELDS 23

/* node gradients of the heightmap (Q10) */
void orc_terrain_gradients(const float *heights, int nx, int ny, double cell,
                           double *gx, double *gy);
/* bilinear f, f_x, f_y, costmap at (x, y); returns 1 if the query was off-map */
int orc_terrain_sample(const orc_terrain *t, double x, double y, double out[4]);

/* sigmoid tire model of Sec. III-A, F_y / F_z */
double orc_tire(double C, double mu, double alpha);
/* energy stability margin U_ESM at roll phi, pitch theta (Sec. IV-B) */
double orc_esm(const orc_vehicle *v, double phi, double theta);
/* 3-2-1 rotation matrix body -> world, row-major (Sec. IV-A) */
void orc_rotation(double psi, double theta, double phi, double R[9]);

/* One evaluation of the SRB state derivative xi_dot = A(xi) + B zeta (Sec. IV-A)
 * with its running cost rate; wheel/body diagnostics may be NULL. */
void orc_eval(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
              const double xi[13], const double zeta[2], double xidot[13],
              double *wheel, double *body);

/* Forward-Euler rollout of N candidates.
 *   x0    float [13] shared (x0_per_cand = 0) or [N][13] (x0_per_cand = 1)
 *   ctrl  float [H][N][2] (steering rate, longitudinal acceleration)
 *   h = dt / n_sub.
 * Outputs (NULL allowed except J, margin, flags):
 *   J[N], margin[N] (min U_ESM over the trajectory), flags[N],
 *   xf[N][13] final state, step_margin[H][N] (min U over each control step),
 *   diag[N][3] = min over the trajectory of |F_s - k chi| / F_s (contact
 *   switch), |U| / U0 (feasibility switch) and | |p - goal| - r_g | (goal). */
int orc_rollout(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                const float *x0, int x0_per_cand, const float *ctrl,
                int N, int H, double dt, int n_sub,
                double *J, double *margin, unsigned char *flags,
                double *xf, double *step_margin, double *diag, int nthreads);

/* Single candidate, every Euler state recorded: states[(H n_sub + 1)][13],
 * Jrun[H n_sub + 1] running cost before the terminal term.  Returns the
 * Euler-step index at which the goal was reached, or -1. */
int orc_trajectory(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                   const double x0[13], const float *ctrl, int H, double dt, int n_sub,
                   double *states, double *Jrun);

/* Empirical argmin (Sec. IV-D) by the lexicographic key (infeasible, J, j). */
int orc_select(const double *J, const unsigned char *flags, int N);

/* ---- Extended single-track (EST) planar model (est.c) ----------------- */
/* EST state: x, y, psi, v_By, w_Bz, delta, v_Bx (the paper's order). */
#define ORC_EST_FIELDS 19
void orc_est_rotation(double phi, double theta, double psi, double R[9]);
void orc_est_eval(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double xi[7],
                  const double zeta[2], double xidot[7], double *diag);
/* As orc_rollout with 7-component states; margin = min over the integrated
 * Euler steps of abar - |a_By - g_By|; diag[N][3] = (inf, min |margin| / abar,
 * goal-circle distance). */
int orc_est_rollout(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const float *x0,
                    int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub, double *J,
                    double *margin, unsigned char *flags, double *xf, double *step_margin, double *diag,
                    int nthreads);
int orc_est_trajectory(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                       const double x0[7], const float *ctrl, int H, double dt, int n_sub,
                       double *states);

/* ---- Terrain preprocessing (terrain_tools.c) --------------------------- */
int orc_lod_weights(double cell, double sigma, int r_max, double *w);
int orc_lod_smooth(const float *f, int nx, int ny, double cell, double sigma, double *out);
double orc_sdist(const double *xy, int n, int kind, double px, double py);
void orc_costmap(const double *xy, const int *start, const int *kind, int n_poly, int nx, int ny,
                 double cell, double x0, double y0, double eps, double sigma, double *cost,
                 double *sdist_min);

#ifdef __cplusplus
}
#endif
#endif
