/*
 * atp.h - C-ABI of the GB300 (sm_103a) all-terrain rollout planner.
 *
 * The library runs the sampling MPC hot path of arxiv 2603.20525 ("High-Speed,
 * All-Terrain Autonomy: Ensuring Safety at the Limits of Mobility"):
 * N candidate control sequences are rolled forward through the paper's
 * single-rigid-body (SRB) vehicle model on a heightmap (Sec. IV-A), scored
 * with the cost of Sec. IV-C including the energy-stability-margin (ESM) soft
 * constraint of Sec. IV-B, and reduced to the best feasible candidate, the
 * "empirical argmin" of Sec. IV-D.  Every step runs in the library's own CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions
 *   - Frames (App. A): W is world-fixed with w_z up; B is body-fixed with
 *     b_x forward, b_y left, b_z up.  SI units, angles in radians.
 *   - State (Sec. IV-A), 13 floats in this order:
 *       x, y, z, psi, theta, phi (3-2-1 yaw, pitch, roll), v_Bx, v_By, v_Bz,
 *       w_Bx, w_By, w_Bz, delta (steering angle).
 *   - Control (Sec. III-A, IV-A): zeta = (steering rate [rad/s],
 *     longitudinal velocity rate [m/s^2]), held for dt (zero-order hold,
 *     Sec. IV-C).  Candidates are float2 ctrl[H][N], time-major, so one
 *     control step of a warp's 32 candidates is 256 contiguous bytes.
 *   - Heights: heights[j][i] = f(x0 + i*cell, y0 + j*cell), row-major FP32.
 *   - Each control step runs n_sub forward-Euler steps of h = dt / n_sub
 *     (n_sub = 0 selects ceil(dt / 5 ms), the paper's 5 ms step, Sec. IV-D).
 *
 * Ownership and asynchrony
 *   All array arguments named *_dev are device pointers owned by the caller.
 *   Structs passed by pointer without _dev are host memory read during the
 *   call only.  Every compute call is enqueued on the given stream (NULL =
 *   legacy default stream) and returns before the GPU finishes; outputs are
 *   valid once the stream has been synchronized.  A context owns only small
 *   scratch buffers (the reduction key, counters and, when the caller does not
 *   supply them, per-candidate outputs), is bound to one device, and is not
 *   thread-safe: use one context per host thread or stream, because calls on
 *   one context that overlap on the GPU share its scratch.
 *
 * Errors
 *   Every int-returning call returns ATP_OK (0) or a negative ATP_ERR_* code
 *   and never throws.  atp_last_error() gives a one-line reason.  Invalid
 *   arguments are rejected before anything is enqueued.  A candidate whose
 *   rollout turns non-finite is data, not an error: its cost is +inf and it
 *   is infeasible, with ATP_FLAG_NONFINITE set.
 */
#ifndef ATP_H
#define ATP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ATP_VERSION 1

enum {
    ATP_OK = 0,
    ATP_ERR_INVALID = -1,     /* null pointer, bad size, non-finite parameter */
    ATP_ERR_UNSUPPORTED = -2, /* size or format the library does not handle */
    ATP_ERR_NOMEM = -3,       /* device allocation failed */
    ATP_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    ATP_ERR_TIMEOUT = -5      /* a bounded device wait gave up */
};

/* texel formats of a prepared terrain */
enum {
    ATP_TERRAIN_F32X4 = 0,    /* float4 (f, f_x, f_y, cost) per node, 16 B */
    ATP_TERRAIN_BF16X4 = 1    /* 4 x bf16 per node, 8 B: the height's and slopes'
                                 residuals from their 8 x 8 block's FP32 plane (through
                                 the block's first node, with its first row's and
                                 column's slopes) and the cost; then the planes */
};

/* context options (atp_set_option) */
enum {
    ATP_OPT_COST_FP64 = 1,    /* accumulate the running cost in FP64 (default 0: FP32) */
    ATP_OPT_LANES = 2,        /* threads per candidate in atp_plan / atp_rollout: 0 chooses
                                 by batch size (default), 1, 2 or 4 forces it */
    ATP_OPT_STAGE_TERRAIN = 3 /* side in nodes (2..120) of a texel window staged in shared
                                 memory by atp_plan / atp_rollout; 0 (default) off */
};

/* per-candidate flag bits */
enum {
    ATP_FLAG_FEASIBLE = 1,    /* min U_ESM over the trajectory > 0 and finite (Sec. IV-B) */
    ATP_FLAG_DONE = 2,        /* reached the goal circle and was frozen (Sec. IV-C) */
    ATP_FLAG_OFFMAP = 4,      /* a wheel queried the terrain outside the map */
    ATP_FLAG_NONFINITE = 8    /* state or cost became NaN/inf */
};

/* Vehicle parameters in SI units (App. A notation, App. B values).
 * L_f, L_r: CoM to front / rear axle; e: track; hR: h + R, the CoM height
 * above the contact patches; k, b: spring and damper rate of each front /
 * rear corner; C, mu: sigmoid tire model (Sec. III-A); delta_max: steering
 * angle limit; delta_rate_max: steering rate limit (Sec. IV-C); g: gravity. */
typedef struct {
    double M, Jxx, Jyy, Jzz;
    double Lf, Lr, e, hR;
    double kf, kr, bf, br;
    double C, mu;
    double delta_max, delta_rate_max, g;
} atp_vehicle;

/* Cost of Sec. IV-C: L = w_t + w_c delta_dot^2 + sigma max(0, 1 - U/eps)^2
 * + sum over wheels of the costmap, Phi = w_g |p_xy - goal|; the horizon is
 * truncated when |p_xy - goal| <= goal_r.  eps_esm <= 0 selects 10 % of the
 * level-ground ESM.  All weights must be >= 0. */
typedef struct {
    double wt, wc, wg, sigma, eps_esm, goal_x, goal_y, goal_r;
} atp_cost;

/* one SRB state, the 13 floats in the order given above */
typedef struct {
    float x, y, z, psi, theta, phi, vx, vy, vz, wx, wy, wz, delta;
} atp_state;

/* terrain flag bits (atp_terrain.flags) */
enum {
    ATP_TERRAIN_HAS_COSTMAP = 1   /* the texels' cost channel holds a costmap */
};

/* A prepared terrain (see atp_terrain_prepare).  texels is a device pointer
 * owned by the caller, nx * ny texels of the given format.  flags is set by
 * atp_terrain_prepare; without ATP_TERRAIN_HAS_COSTMAP the kernels skip the
 * cost channel (it is zero). */
typedef struct {
    const void *texels;
    int nx, ny;
    double cell, x0, y0;      /* node (i, j) is at (x0 + i cell, y0 + j cell) */
    int format;
    int flags;
} atp_terrain;

/* Result of a plan, written to device memory. */
typedef struct {
    uint32_t best_idx;        /* index of the best candidate (Sec. IV-D, reading Q7) */
    uint32_t n_feasible;      /* number of feasible candidates */
    float best_cost;          /* J of the best candidate */
    float best_min_margin;    /* its minimum U_ESM over the trajectory [J] */
    int32_t best_min_step;    /* control step holding that minimum */
    uint32_t reserved;
} atp_plan_out;

/* --------------------------------------------------------------------- */
int atp_version(void);

/* Create a context on `device` (made current for the call).  Allocates the
 * small reduction scratch.  Returns ATP_ERR_CUDA / ATP_ERR_NOMEM on failure,
 * with *ctx set to NULL. */
struct atp_ctx;
typedef struct atp_ctx atp_ctx;
int atp_create(atp_ctx **ctx, int device);

/* Free the context and its scratch.  Waits for the device first. */
int atp_destroy(atp_ctx *ctx);

/* One-line description of the last error on this context ("" if none). */
const char *atp_last_error(const atp_ctx *ctx);

/* Pre-size the context scratch for plans (or batches, see atp_plan_batch) of
 * up to N candidates in total and H control steps, so that later calls
 * allocate nothing.  Without it, a call grows the scratch on first use of a
 * larger size (a synchronous cudaMalloc after a device synchronize). */
int atp_reserve(atp_ctx *ctx, int N, int H);

/* Bytes of device memory a prepared terrain of nx x ny nodes needs:
 * 16 nx ny (F32X4); 8 nx ny rounded up to 256, plus 16 bytes per 8 x 8
 * block (BF16X4). */
size_t atp_terrain_bytes(int nx, int ny, int format);

/* Set a context option for the calls that follow on this context:
 * ATP_OPT_COST_FP64 (value 0 or 1) accumulates each candidate's running cost
 * (time, control effort and the soft ESM and costmap constraints, Sec. IV-C)
 * in FP64 instead of FP32; ATP_OPT_LANES (0, 1, 2 or 4) sets the threads per
 * candidate of atp_plan and atp_rollout (two split the axles and four the
 * wheels: lower latency for small batches; one: more throughput once a batch
 * fills the GPU).  One, two and four lanes give the same bits: every layout
 * forms the axle sums and the force and moment totals in one order.
 * ATP_OPT_STAGE_TERRAIN (0, or a side W from 2 to 120 nodes) stages a window
 * of the texels in shared memory (Sec. IV-D's cached terrain lookups): each
 * CTA of 512 threads first copies min(W, nx) x min(W, ny) texels (16 B each,
 * at most 225 KB), centred a quarter of its side ahead of the start along
 * the start heading and moved inside the map, then reads every lookup whose
 * four corners lie in it from shared memory and the rest from global
 * memory.  It applies to plans of one lane per candidate on F32X4 terrains
 * from a shared start state (x0 on the host); other plans, atp_plan_batch
 * and atp_plan_noalloc run unstaged.  The results are the same bits as the
 * unstaged one-lane kernel's.
 * Returns ATP_ERR_INVALID for an unknown option or value. */
int atp_set_option(atp_ctx *ctx, int option, int value);

/* Threads per candidate (1, 2 or 4) that atp_plan and atp_rollout on this
 * context use for a plan of N candidates: the ATP_OPT_LANES value if set,
 * else the library's choice by batch size.  Returns ATP_ERR_INVALID for a
 * NULL context or N < 1. */
int atp_plan_lanes(const atp_ctx *ctx, int N);

/* Build the texels of a terrain: per node the height, its slope f_x, f_y by
 * central differences (one-sided on the border) and the optional costmap
 * value, the numeric-slope heightmap of Sec. III-A and the interpolated
 * costmap of Sec. IV-D (reading Q10).
 *   heights_dev  float [ny][nx], device
 *   costmap_dev  float [ny][nx] summed soft-constraint cost rate, or NULL (0)
 *   texels_dev   atp_terrain_bytes(nx, ny, format) bytes, 16-byte aligned
 * nx, ny >= 3, cell > 0.  Fills *out (may be NULL) with the terrain handle. */
int atp_terrain_prepare(atp_ctx *ctx, const float *heights_dev, const float *costmap_dev,
                        int nx, int ny, double cell, double x0, double y0, int format,
                        void *texels_dev, atp_terrain *out, void *stream);

/* Plan: roll out N candidates over H control steps and reduce to the best.
 *
 *   x0            host state shared by every candidate, or NULL when
 *   x0_dev        float [13][N] device SoA of per-candidate initial states
 *                 (row q holds state component q of every candidate)
 *   ctrl_dev      float2 ctrl[H][N] device, 8-byte aligned
 *   dt, n_sub     zero-order-hold interval and Euler steps per interval
 *   out_dev       atp_plan_out, device
 *   best_ctrl_dev float [H][2] or NULL: the best candidate's controls with the
 *                 steering rate clamped as used
 *   best_margin_dev float [H] or NULL: the best candidate's minimum U_ESM over
 *                 each control step (the final state folded into step H-1);
 *                 only then does the plan keep every candidate's per-step
 *                 margins (4 N H bytes of scratch written), otherwise each
 *                 candidate keeps just the step of its smallest margin
 *   cand_cost_dev, cand_margin_dev  float [N] or NULL: J and min U_ESM
 *   cand_flags_dev uint8 [N] or NULL: ATP_FLAG_* bits
 *   cand_xf_dev   float [13][N] or NULL: final states, SoA
 *   stream        cudaStream_t
 * 1 <= N, H >= 1, dt > 0, 0 <= n_sub.  Validation failures return
 * ATP_ERR_INVALID; N above 2^31 - 1025 (the most candidates any call takes, so
 * that every kernel's thread index stays within 32 bits) ATP_ERR_UNSUPPORTED;
 * launch failures ATP_ERR_CUDA. */
int atp_plan(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
             const atp_terrain *terrain, const atp_state *x0, const float *x0_dev,
             const float *ctrl_dev, int N, int H, float dt, int n_sub,
             atp_plan_out *out_dev, float *best_ctrl_dev, float *best_margin_dev,
             float *cand_cost_dev, float *cand_margin_dev, uint8_t *cand_flags_dev,
             float *cand_xf_dev, void *stream);

/* Batched rollout without the reduction: the same per-candidate results as
 * atp_plan (cost, margin, flags, final states, per-step margins
 * step_margin_dev float [H][N] or NULL), nothing else. */
int atp_rollout(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
                const atp_terrain *terrain, const atp_state *x0, const float *x0_dev,
                const float *ctrl_dev, int N, int H, float dt, int n_sub,
                float *cand_cost_dev, float *cand_margin_dev, uint8_t *cand_flags_dev,
                float *cand_xf_dev, float *step_margin_dev, void *stream);

/* One plan of a batch: the arguments of atp_plan gathered in a struct.  The
 * struct pointers (veh, cost, terrain, x0) are host memory read during the
 * call; the *_dev pointers are device memory as for atp_plan. */
typedef struct {
    const atp_vehicle *veh;
    const atp_cost *cost;
    const atp_terrain *terrain;
    const atp_state *x0;
    const float *x0_dev;
    const float *ctrl_dev;
    int N, H;
    float dt;
    int n_sub;
    atp_plan_out *out_dev;
    float *best_ctrl_dev, *best_margin_dev;
    float *cand_cost_dev, *cand_margin_dev;
    uint8_t *cand_flags_dev;
    float *cand_xf_dev;
} atp_plan_request;

/* Continuous batching: n_req (1..64) independent plans, each with its own
 * vehicle, terrain, candidates, horizon and outputs, in one kernel launch.
 * Each plan's results are bit-identical to a single atp_plan of the same
 * request, alone or in any mix, since every layout gives the same bits.  The
 * batch chooses each plan's threads per candidate for the batch as a whole:
 * ATP_OPT_LANES if set; else one, raised in request order to the four (or
 * two) lanes a plan of its size would run alone while the batch's threads
 * stay within what a two-lane plan alone may use (2 x 28672), else to two if
 * those fit.  The
 * context's scratch grows to the sum of the plans' needs; atp_reserve(ctx,
 * sum of N, max H) pre-sizes it for any batch within those totals.
 * Validation failures name the offending request in atp_last_error. */
int atp_plan_batch(atp_ctx *ctx, const atp_plan_request *reqs, int n_req, void *stream);

/* Gradient of each candidate's cost with respect to its raw controls: the
 * hand-written reverse-mode adjoint of the discrete rollout (Sec. IV-A..C)
 * for K candidates, J = sum over Euler steps of h L + Phi, with the
 * branches (liftoff, clamps, off-map, goal) taken as in the forward pass.
 *   ctrl_dev  float2 [H][K] raw controls (steering rate, acceleration)
 *   cost_dev  float [K]: J of each candidate (as atp_plan computes it)
 *   grad_dev  float [H][K][2]: dJ/d(steering rate), dJ/d(acceleration);
 *             zero for a steering rate beyond its limit (the clamp)
 *   ckpt      control steps between stored states (0 selects 10); the
 *             reverse pass recomputes one such segment at a time, so memory
 *             is (H / ckpt + b ckpt n_sub) x 320 bytes per candidate, b the
 *             number of segment buffers: 2 while the grid of 16-candidate
 *             CTAs fits the device in one wave (one set of warps then
 *             recomputes the next segment while another walks this one
 *             back), else 1.  The results are the same bits either way and
 *             for every ckpt.
 * Four threads per candidate (one wheel each); K <= 2^28; F32X4 terrain
 * only. */
int atp_grad(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost, const atp_terrain *terrain,
             const atp_state *x0, const float *x0_dev, const float *ctrl_dev, int K, int H, float dt,
             int n_sub, int ckpt, float *cost_dev, float *grad_dev, void *stream);

/* Constraint gradient: the same adjoint for each candidate's ESM margin, the
 * minimum of U_ESM over every state of its trajectory (Sec. IV-B; the final
 * state and the states frozen at the goal included, as atp_plan's margin):
 * d(min U_ESM)/du, taken as the gradient of U_ESM at the state holding the
 * minimum (the first such state on ties), a subgradient of the minimum.
 *   margin_dev float [K]: each candidate's margin [J] (as atp_plan's)
 *   grad_dev   float [H][K][2]: d(margin)/d(steering rate), d(margin)/d(accel)
 * Other arguments, memory and limits as atp_grad. */
int atp_grad_margin(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
                    const atp_terrain *terrain, const atp_state *x0, const float *x0_dev,
                    const float *ctrl_dev, int K, int H, float dt, int n_sub, int ckpt,
                    float *margin_dev, float *grad_dev, void *stream);

/* Gradient refinement of K candidates by projected gradient descent on
 * their cost (atp_grad), in three calls per iteration; every array is
 * device memory, [H][K][2] ones (steering rate, acceleration) 8-byte aligned:
 *   atp_refine_init    eta[K] = step / (max over k, c of |grad[k][j][c]| + 1e-12)
 *   atp_refine_trial   trial = ctrl - eta[j] grad, the steering rate clamped
 *                      to +/- rate_max (the admissible set of Sec. IV-C)
 *   atp_refine_accept  for each candidate whose trial_cost is finite and lower
 *                      than cost: ctrl, grad and cost take the trial's and
 *                      eta grows by 1.5; for the others eta halves.
 * An iteration is trial, atp_grad on the trial, accept; the cost then never
 * increases.  K, H >= 1, K <= 2^31 - 1025; step > 0; rate_max >= 0. */
int atp_refine_init(atp_ctx *ctx, const float *grad_dev, int K, int H, float step, float *eta_dev, void *stream);
int atp_refine_trial(atp_ctx *ctx, const float *ctrl_dev, const float *grad_dev, const float *eta_dev, int K,
                     int H, float rate_max, float *trial_dev, void *stream);
int atp_refine_accept(atp_ctx *ctx, int K, int H, const float *trial_dev, const float *trial_cost_dev,
                      const float *trial_grad_dev, float *ctrl_dev, float *cost_dev, float *grad_dev,
                      float *eta_dev, void *stream);

/* Candidate sampler (the on-GPU drawing of Sec. IV-D): writes float2
 * ctrl[H][N] with ctrl[k][j] = nominal[k] + (sigma_rate n1, sigma_acc n2),
 * where (n1, n2) is a Box-Muller pair of 23-bit uniforms from Philox4x64-10
 * (Salmon et al., SC'11) under key (key0, key1): one call at counter
 * (j, kq, nonce, 0) serves steps k = 4 kq + s, s = 0..3, with the words
 * (w0, w1) for s = 0, 2 and (w2, w3) for s = 1, 3, each word's bits 63..41
 * for s < 2 and bits 31..9 for s >= 2; candidate 0 is the nominal.
 * The nominal is a warm start from the previous plan's best controls,
 * nominal[k] = prev_best[min(k + shift, H_prev - 1)] (float [H_prev][2],
 * device), or zero when H_prev = 0.  Draws depend only on (key, nonce, j, k),
 * not on the launch.  1 <= H <= 65535, 1 <= N <= 2^31 - 1025. */
int atp_sample(atp_ctx *ctx, const float *prev_best_dev, int H_prev, int shift, double sigma_rate,
               double sigma_acc, uint64_t key0, uint64_t key1, uint64_t nonce, int N, int H,
               float *ctrl_dev, void *stream);

/* Diagnostic: evaluates the library's own FP32 elementary functions next to
 * CUDA's on n input pairs (a_i, b_i), writing 14 floats per pair to out_dev:
 * [sin a, cos a] (library), [sinf a, cosf a] (CUDA), atan2(a, b) (library),
 * atan2f(a, b) (CUDA), 1/b (library reciprocal), 1.0f/b (IEEE division),
 * 1/sqrt(b) (library), rsqrtf(b) (CUDA), then a b + b by the packed
 * two-wide FMA and by the scalar one, and b - a by the packed two-wide
 * subtraction and by the scalar one.  All pointers are device memory of n
 * (a, b) and 14 n (out) floats. */
int atp_math_check(const float *a_dev, const float *b_dev, int n, float *out_dev, void *stream);

/* ---- The planar model (App. "Extended Single-Track Vehicle Dynamics
 * Model"): the formulation the paper sets beside the SRB model. ---------- */

/* one EST state: position, yaw, lateral velocity, yaw rate, steering angle,
 * longitudinal velocity (the paper's order) */
typedef struct {
    float x, y, psi, vy, wz, delta, vx;
} atp_est_state;

/* Plan with the extended single-track model instead of the SRB model: per
 * Euler step the terrain's normal under the CoM sets pitch and roll (1-2-3
 * convention, normal ~ (-f_x, -f_y, 1)), the virtual front and rear tires'
 * normal forces follow from the load-transfer coefficients, their lateral
 * forces from the sigmoid tire, and the lateral-acceleration constraint
 * |a_By - g_By| < abar = g e / (2 (h+R)) replaces the ESM: its soft cost
 * sigma max(0, 1 - margin / eps)^2 with eps = cost->eps_esm if > 0, else
 * 0.1 abar, and a candidate is feasible when its minimum margin over the
 * integrated Euler steps is > 0.  The costmap is read at the four wheel
 * contact points.  Arguments, outputs and results are those of atp_plan,
 * with 7-component states: x0 (host) or x0_dev float [7][N]; cand_xf_dev
 * float [7][N]; margins in m/s^2.  Uses Jzz, Lf, Lr, e, hR, C, mu, the
 * steering limits and g of the vehicle. */
int atp_plan_est(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
                 const atp_terrain *terrain, const atp_est_state *x0, const float *x0_dev,
                 const float *ctrl_dev, int N, int H, float dt, int n_sub,
                 atp_plan_out *out_dev, float *best_ctrl_dev, float *best_margin_dev,
                 float *cand_cost_dev, float *cand_margin_dev, uint8_t *cand_flags_dev,
                 float *cand_xf_dev, void *stream);

/* ---- Terrain preprocessing ---------------------------------------------- */

/* Model-specific level of detail (Sec. V-B): out = the heightmap smoothed by a
 * Gaussian of standard deviation sigma metres (0.3 m for the SRB model, 1.5 m
 * for the planar model in the paper), cut at r = floor(4 sigma / cell + 1/2)
 * cells, with the map extended by its nearest border node.  sigma = 0 copies.
 *   heights_dev, out_dev  float [ny][nx], device (out may equal heights)
 *   tmp_dev               float [ny][nx], device scratch, aliasing neither
 * r <= 512 cells, else ATP_ERR_UNSUPPORTED. */
int atp_lod_smooth(atp_ctx *ctx, const float *heights_dev, int nx, int ny, double cell,
                   double sigma, float *tmp_dev, float *out_dev, void *stream);

/* Costmap of the distance constraints (Sec. IV-C, IV-D): at every node
 * (x0 + i cell, y0 + j cell) the sum over perimeters p of
 * sigma max(0, 1 - sdist_p / eps)^2, where sdist_p is the distance to p's
 * edges, negative inside an obstacle (kind 0) and outside a path boundary
 * (kind 1), inside by the even-odd rule.  The paper uses eps = 0.25 m and
 * sigma = 1e6.  The result is the costmap_dev input of atp_terrain_prepare.
 *   xy_dev      double [n_vert][2] perimeter vertices in world metres, device
 *   start       int [n_poly + 1], host: perimeter p is vertices start[p] ..
 *               start[p+1]-1, start[0] = 0, start[n_poly] = n_vert, each >= 2
 *   kind        int [n_poly], host: 0 obstacle, 1 path boundary
 *   cost_dev    float [ny][nx], device
 *   sdist_dev   float [ny][nx] or NULL: the smallest signed distance
 * 1 <= n_poly <= 256.  Without sdist_dev, each 16 x 16 tile of nodes skips the
 * obstacles whose bounding box lies more than 2 eps away from it (their rate
 * there is exactly zero), which gives the same costmap bits as evaluating
 * every perimeter; with sdist_dev every perimeter is evaluated at every node. */
int atp_costmap(atp_ctx *ctx, const double *xy_dev, const int *start, const int *kind, int n_poly,
                int nx, int ny, double cell, double x0, double y0, double eps, double sigma,
                float *cost_dev, float *sdist_dev, void *stream);

/* Plan without allocating: atp_plan for callers that cannot allocate device
 * memory once running, such as a planner in a hard real-time control loop
 * whose latency budget or certification forbids cudaMalloc after start-up, or
 * a plugin host that gives its plugins no allocator.  The paper has no
 * counterpart; it exists for such callers only.
 *
 * Arguments, outputs and results are those of atp_plan on a context with the
 * default options (running cost accumulated in FP32, threads per candidate
 * chosen by batch size), without a context.  Its scratch is one file-scope
 * device array of 8 MiB in this library, which every GPU that loads the
 * library holds until the process exits.  It supports plans whose scratch
 * fits in 8 MiB: 256 B + 13 N bytes, plus 4 N H bytes when best_margin_dev
 * is given, each of the five parts rounded up to 256 B (N up to about
 * 645,000 without per-step margins; N = 16384 with H <= 124 with them);
 * larger plans return ATP_ERR_UNSUPPORTED before anything is enqueued.  The call
 * runs on the calling thread's current device (at most device 63), calls no
 * cudaMalloc or cudaFree, and enqueues two small memsets that reset the
 * reduction state before the kernel.  Its first call on a device looks up the
 * array's device address with that device current (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: a caller that resets a device (cudaDeviceReset)
 * must not call this function on that device afterwards.  Every call shares the one
 * array, so calls that overlap on the GPU (other streams, other host threads)
 * race and corrupt each other's results: serialise them. */
int atp_plan_noalloc(const atp_vehicle *veh, const atp_cost *cost, const atp_terrain *terrain,
                     const atp_state *x0, const float *x0_dev, const float *ctrl_dev, int N,
                     int H, float dt, int n_sub, atp_plan_out *out_dev, float *best_ctrl_dev,
                     float *best_margin_dev, float *cand_cost_dev, float *cand_margin_dev,
                     uint8_t *cand_flags_dev, float *cand_xf_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ATP_H */
