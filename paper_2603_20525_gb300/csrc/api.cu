// api.cu - the C-ABI of include/atp.h: argument validation, the context and
// its scratch, FP64 -> FP32 parameter derivation and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "atp.h"
#include "adjoint.cuh"
#include "est_kernel.cuh"
#include "plan_kernel.cuh"
#include "refine.cuh"
#include "sampler.cuh"
#include "terrain_tools.cuh"

struct atp_ctx {
    int device;
    int acc64;                // ATP_OPT_COST_FP64
    int lanes;                // ATP_OPT_LANES
    int stage;                // ATP_OPT_STAGE_TERRAIN: window side in nodes, 0 off
    char err[256];
    void *scratch;            // reduction headers + per-plan candidate buffers
    size_t scratch_bytes;
    atp::BatchParams *batch;  // host staging of one batch's descriptors
    float4 *cm_box;           // the costmap's per-perimeter reach boxes (device)
    int grad_ctas;            // resident CTAs of the split adjoint layout, -1 until queried
};

namespace {

int fail(atp_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(atp_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, e == cudaErrorMemoryAllocation ? ATP_ERR_NOMEM : ATP_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// Selects ctx->device for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
        else if (err == cudaSuccess) prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool fin(double v) { return std::isfinite(v); }

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Per-plan scratch: the candidates' cost, margin, flags and minimum-margin
// step, and, only when the best candidate's per-step margins are asked for,
// every candidate's per-step margins [H][N].
struct RegionLayout {
    size_t cost, margin, flags, min_step, step_margin, total;
};

RegionLayout region_layout(size_t N, size_t H, bool steps, size_t o = 0)
{
    RegionLayout L;
    L.cost = o;        o = align_up(o + N * sizeof(float));
    L.margin = o;      o = align_up(o + N * sizeof(float));
    L.flags = o;       o = align_up(o + N);
    L.min_step = o;    o = align_up(o + N * sizeof(int));
    L.step_margin = o; o = align_up(o + (steps ? N * H * sizeof(float) : 0));
    L.total = o;
    return L;
}

// Scratch of atp_plan_noalloc: one reduction header, then one plan's region.
RegionLayout layout(size_t N, size_t H, bool steps)
{
    return region_layout(N, H, steps, align_up(sizeof(atp::Scratch)));
}

// Context scratch: kMaxBatch reduction headers at fixed offsets (each plan's
// last CTA restores its header, so they stay valid across calls), then one
// region per plan of the call.
constexpr size_t kHeaderBytes = (atp::kMaxBatch * sizeof(atp::Scratch) + kAlign - 1) / kAlign * kAlign;

int ensure_scratch_bytes(atp_ctx *ctx, size_t need)
{
    need += kHeaderBytes;
    if (ctx->scratch && need <= ctx->scratch_bytes) return ATP_OK;
    if (ctx->scratch) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize before growing scratch");
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch allocation");
    atp::Scratch init[atp::kMaxBatch];
    for (auto &h : init) h = atp::Scratch{~0ull, 0u, 0u};
    e = cudaMemcpy(p, init, sizeof init, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_fail(ctx, e, "scratch initialisation");
    }
    ctx->scratch = p;
    ctx->scratch_bytes = need;
    return ATP_OK;
}

int ensure_scratch(atp_ctx *ctx, int N, int H, bool steps)
{
    return ensure_scratch_bytes(ctx, region_layout((size_t)N, (size_t)H, steps).total);
}

int check_vehicle(atp_ctx *ctx, const atp_vehicle *v)
{
    if (!v) return fail(ctx, ATP_ERR_INVALID, "vehicle is NULL");
    const double a[] = {v->M, v->Jxx, v->Jyy, v->Jzz, v->Lf, v->Lr, v->e, v->hR, v->kf, v->kr,
                        v->bf, v->br, v->C, v->mu, v->delta_max, v->delta_rate_max, v->g};
    for (double x : a)
        if (!fin(x)) return fail(ctx, ATP_ERR_INVALID, "vehicle parameter is not finite");
    if (!(v->M > 0 && v->Jxx > 0 && v->Jyy > 0 && v->Jzz > 0))
        return fail(ctx, ATP_ERR_INVALID, "mass and inertias must be > 0");
    if (!(v->Lf > 0 && v->Lr > 0 && v->e > 0 && v->hR > 0))
        return fail(ctx, ATP_ERR_INVALID, "Lf, Lr, e, h+R must be > 0");
    if (!(v->kf >= 0 && v->kr >= 0 && v->bf >= 0 && v->br >= 0 && v->C >= 0 && v->mu > 0 &&
          v->delta_max >= 0 && v->delta_rate_max >= 0 && v->g >= 0))
        return fail(ctx, ATP_ERR_INVALID, "k, b, C, delta limits, g must be >= 0 and mu > 0");
    return ATP_OK;
}

int check_cost(atp_ctx *ctx, const atp_cost *c)
{
    if (!c) return fail(ctx, ATP_ERR_INVALID, "cost is NULL");
    const double a[] = {c->wt, c->wc, c->wg, c->sigma, c->eps_esm, c->goal_x, c->goal_y, c->goal_r};
    for (double x : a)
        if (!fin(x)) return fail(ctx, ATP_ERR_INVALID, "cost parameter is not finite");
    if (!(c->wt >= 0 && c->wc >= 0 && c->wg >= 0 && c->sigma >= 0 && c->goal_r >= 0))
        return fail(ctx, ATP_ERR_INVALID, "cost weights and goal radius must be >= 0");
    return ATP_OK;
}

int check_terrain(atp_ctx *ctx, const atp_terrain *t)
{
    if (!t || !t->texels) return fail(ctx, ATP_ERR_INVALID, "terrain or its texels is NULL");
    if (t->format != ATP_TERRAIN_F32X4 && t->format != ATP_TERRAIN_BF16X4)
        return fail(ctx, ATP_ERR_UNSUPPORTED, "terrain format %d not supported", t->format);
    if (t->nx < 3 || t->ny < 3 || t->nx > 65536 || t->ny > 65536)
        return fail(ctx, ATP_ERR_INVALID, "terrain must be between 3 and 65536 nodes per side");
    if (!(t->cell > 0.0) || !std::isfinite(t->cell) || !std::isfinite(t->x0) || !std::isfinite(t->y0))
        return fail(ctx, ATP_ERR_INVALID, "terrain cell must be > 0 and origin finite");
    if ((uintptr_t)t->texels % 16 != 0) return fail(ctx, ATP_ERR_INVALID, "texels must be 16-byte aligned");
    return ATP_OK;
}

// v = hi + lo with hi = fl(v), lo = fl(v - hi)
void split(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// FP64 derivation of the kernel constants (Sec. III-A load transfer, Sec.
// IV-A preload, Sec. IV-B ESM geometry, Sec. IV-C cost).
void derive(const atp_vehicle &v, const atp_cost &c, const atp_terrain &t, atp::PlanParams &p)
{
    const double L = v.Lf + v.Lr;
    const double Kzzf = v.M * v.Lr / L, Kzzr = v.M * v.Lf / L;
    const double Rbar = std::sqrt(v.hR * v.hR + 0.25 * v.e * v.e);
    const double phibar = std::atan(2.0 * v.hR / v.e);
    atp::Veh &V = p.V;
    V.M = (float)v.M;
    V.halfM = (float)(0.5 * v.M);
    V.invM = (float)(1.0 / v.M);
    V.dJyz = (float)(v.Jyy - v.Jzz);
    V.dJxz = (float)(v.Jxx - v.Jzz);
    V.dJxy = (float)(v.Jxx - v.Jyy);
    V.invJxx = (float)(1.0 / v.Jxx);
    V.invJyy = (float)(1.0 / v.Jyy);
    V.invJzz = (float)(1.0 / v.Jzz);
    V.Lf = (float)v.Lf;
    V.Lr = (float)v.Lr;
    V.he = (float)(0.5 * v.e);
    V.hR = (float)v.hR;
    V.kf = (float)v.kf;
    V.kr = (float)v.kr;
    V.bf = (float)v.bf;
    V.br = (float)v.br;
    V.Fsf = (float)(0.5 * v.g * Kzzf);
    V.Fsr = (float)(0.5 * v.g * Kzzr);
    V.C = (float)v.C;
    V.mu = (float)v.mu;
    V.mu2 = (float)(v.mu * v.mu);
    V.dmax = (float)v.delta_max;
    V.ddmax = (float)v.delta_rate_max;
    V.g = (float)v.g;
    V.MgRbar = (float)(v.M * v.g * Rbar);
    V.cpb = (float)std::cos(phibar);
    V.spb = (float)std::sin(phibar);
    V.tip = (float)(0.5 * M_PI - phibar);
    V.Kzzf = (float)Kzzf;
    V.Kzzr = (float)Kzzr;
    V.Kzx = (float)(v.M * v.hR / L);
    V.abar = (float)(v.g * v.e / (2.0 * v.hR));      // M g / (2 K_zy), K_zy = M (h+R) / e
    const double U0 = v.M * v.g * Rbar * (1.0 - std::sin(phibar));
    const double eps = c.eps_esm > 0 ? c.eps_esm : 0.1 * U0;
    atp::Cost &C = p.C;
    C.wt = (float)c.wt;
    C.wc = (float)c.wc;
    C.wg = (float)c.wg;
    C.sigma = (float)c.sigma;
    C.inv_eps = (float)(1.0 / eps);
    split(c.goal_x - t.x0, C.gx_hi, C.gx_lo);
    split(c.goal_y - t.y0, C.gy_hi, C.gy_lo);
    C.goal_r2 = (float)(c.goal_r * c.goal_r);
    atp::Terrain &T = p.T;
    p.tex_format = t.format == ATP_TERRAIN_BF16X4 ? atp::TEX_BF16 : atp::TEX_F32;
    T.tex = (const float4 *)t.texels;
    T.tex16 = (const uint2 *)t.texels;
    T.plane16 = (const float4 *)((const char *)t.texels + atp::bf16_base_offset(t.nx, t.ny));
    T.nbx = (t.nx + 7) / 8;
    T.nx = t.nx;
    T.ny = t.ny;
    T.has_cm = (t.flags & ATP_TERRAIN_HAS_COSTMAP) != 0;
    T.inv_cell = (float)(1.0 / t.cell);
    split(t.x0, T.x0_hi, T.x0_lo);
    split(t.y0, T.y0_hi, T.y0_lo);
}

// The most candidates of one call: every kernel's 32-bit thread index over
// one-thread-per-candidate grids, rounded up to its block, stays below 2^31.
constexpr int kMaxN = INT_MAX - 1024;

int common_checks(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost, const atp_terrain *ter,
                  const float *x0, int n_state, const float *x0_dev, const float *ctrl_dev, int N,
                  int H, float dt, int n_sub, int *n_sub_out)
{
    int rc;
    if ((rc = check_vehicle(ctx, veh)) != ATP_OK) return rc;
    if ((rc = check_cost(ctx, cost)) != ATP_OK) return rc;
    if ((rc = check_terrain(ctx, ter)) != ATP_OK) return rc;
    if (!x0 && !x0_dev) return fail(ctx, ATP_ERR_INVALID, "need x0 or x0_dev");
    if (x0) {
        for (int q = 0; q < n_state; ++q)
            if (!std::isfinite(x0[q])) return fail(ctx, ATP_ERR_INVALID, "x0 is not finite");
    }
    if (!ctrl_dev) return fail(ctx, ATP_ERR_INVALID, "ctrl_dev is NULL");
    if ((uintptr_t)ctrl_dev % 8 != 0) return fail(ctx, ATP_ERR_INVALID, "ctrl_dev must be 8-byte aligned");
    if (N < 1) return fail(ctx, ATP_ERR_INVALID, "N must be >= 1");
    if (N > kMaxN) return fail(ctx, ATP_ERR_UNSUPPORTED, "N above %d", kMaxN);
    if (H < 1) return fail(ctx, ATP_ERR_INVALID, "H must be >= 1");
    if (!(dt > 0.f) || !std::isfinite(dt)) return fail(ctx, ATP_ERR_INVALID, "dt must be finite and > 0");
    if (n_sub < 0 || n_sub > 1000000) return fail(ctx, ATP_ERR_INVALID, "n_sub must be in [0, 1e6]");
    if (n_sub == 0) {
        // ceil(dt / 5 ms), with a dt within FP32 rounding of a multiple of
        // 5 ms taken as that multiple (0.025f is 0.0250000004)
        double q = std::ceil((double)dt / 0.005 - 1e-5);
        n_sub = q < 1.0 ? 1 : (int)q;
    }
    *n_sub_out = n_sub;
    return ATP_OK;
}

void fill_problem(atp::PlanParams &p, const atp_state *x0, const float *x0_dev, const float *ctrl,
                  int N, int H, float dt, int n_sub)
{
    if (x0) {
        std::memcpy(p.x0, &x0->x, sizeof p.x0);
        p.x0_soa = nullptr;
    } else {
        std::memset(p.x0, 0, sizeof p.x0);
        p.x0_soa = x0_dev;
    }
    p.ctrl = (const float2 *)ctrl;
    p.N = N;
    p.H = H;
    p.n_sub = n_sub;
    p.h = (float)((double)dt / (double)n_sub);
}

// The plan's kernel: staged (ATP_OPT_STAGE_TERRAIN) where the option
// applies, i.e. a one-lane plan on F32 texels from a shared start state,
// else the plain kernel.  The window of side min(stage, map side) nodes is
// centred a quarter of its side ahead of the start along the heading, and
// moved inside the map.
cudaError_t launch_plan_for(const atp_ctx *ctx, atp::PlanParams &p, const atp_terrain &t, bool reduce,
                            cudaStream_t stream)
{
    if (ctx->stage == 0 || p.tex_format != atp::TEX_F32 || p.x0_soa || atp::plan_lanes(p.lanes, p.N) != 1)
        return atp::launch_plan(p, reduce, stream);
    const int ww = std::min(ctx->stage, t.nx), wh = std::min(ctx->stage, t.ny);
    const double cx = ((double)p.x0[0] - t.x0) / t.cell, cy = ((double)p.x0[1] - t.y0) / t.cell;
    const double psi = p.x0[3];
    const double ox = cx + 0.25 * ww * std::cos(psi) - 0.5 * ww, oy = cy + 0.25 * wh * std::sin(psi) - 0.5 * wh;
    p.T.wx0 = (int)std::lround(std::min(std::max(ox, 0.0), (double)(t.nx - ww)));
    p.T.wy0 = (int)std::lround(std::min(std::max(oy, 0.0), (double)(t.ny - wh)));
    p.T.ww = ww;
    p.T.wh = wh;
    p.tex_format = atp::TEX_F32W;
    return atp::launch_plan_staged(p, reduce, stream);
}

}  // namespace

extern "C" {

int atp_version(void) { return ATP_VERSION; }

int atp_create(atp_ctx **out, int device)
{
    if (!out) return ATP_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return ATP_ERR_INVALID;
    atp_ctx *ctx = new (std::nothrow) atp_ctx();
    if (!ctx) return ATP_ERR_NOMEM;
    ctx->device = device;
    ctx->acc64 = 0;
    ctx->lanes = 0;
    ctx->stage = 0;
    ctx->grad_ctas = -1;
    ctx->err[0] = 0;
    ctx->batch = new (std::nothrow) atp::BatchParams;
    if (!ctx->batch) {
        delete ctx;
        return ATP_ERR_NOMEM;
    }
    DeviceGuard g(device);
    if (g.err != cudaSuccess) {
        delete ctx->batch;
        delete ctx;
        return ATP_ERR_CUDA;
    }
    if (cudaMalloc(&ctx->cm_box, sizeof(float4) * atp::kCostmapMaxPolys) != cudaSuccess) {
        delete ctx->batch;
        delete ctx;
        return ATP_ERR_NOMEM;
    }
    int rc = ensure_scratch(ctx, 1, 1, true);
    if (rc != ATP_OK) {
        cudaFree(ctx->cm_box);
        delete ctx->batch;
        delete ctx;
        return rc;
    }
    *out = ctx;
    return ATP_OK;
}

int atp_destroy(atp_ctx *ctx)
{
    if (!ctx) return ATP_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->cm_box) cudaFree(ctx->cm_box);
    delete ctx->batch;
    delete ctx;
    return ATP_OK;
}

const char *atp_last_error(const atp_ctx *ctx) { return ctx ? ctx->err : "no context"; }

int atp_reserve(atp_ctx *ctx, int N, int H)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (N < 1 || H < 1) return fail(ctx, ATP_ERR_INVALID, "reserve needs N, H >= 1");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    // room for any batch of up to kMaxBatch plans within these totals: each
    // plan's four arrays round up to kAlign at most once
    return ensure_scratch_bytes(ctx, region_layout((size_t)N, (size_t)H, true).total +
                                         (size_t)atp::kMaxBatch * 5 * kAlign);
}

size_t atp_terrain_bytes(int nx, int ny, int format)
{
    if (nx < 1 || ny < 1) return 0;
    if (format == ATP_TERRAIN_BF16X4)
        return atp::bf16_base_offset(nx, ny) + (size_t)((nx + 7) / 8) * ((ny + 7) / 8) * 16;
    return (size_t)nx * (size_t)ny * 16;
}

int atp_set_option(atp_ctx *ctx, int option, int value)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (option == ATP_OPT_COST_FP64) {
        ctx->acc64 = value != 0;
        return ATP_OK;
    }
    if (option == ATP_OPT_LANES) {
        if (value != 0 && value != 1 && value != 2 && value != 4)
            return fail(ctx, ATP_ERR_INVALID, "ATP_OPT_LANES takes 0, 1, 2 or 4");
        ctx->lanes = value;
        return ATP_OK;
    }
    if (option == ATP_OPT_STAGE_TERRAIN) {
        if (value != 0 && (value < 2 || value > atp::kStageMaxSide))
            return fail(ctx, ATP_ERR_INVALID, "ATP_OPT_STAGE_TERRAIN takes 0 or 2..%d", atp::kStageMaxSide);
        ctx->stage = value;
        return ATP_OK;
    }
    return fail(ctx, ATP_ERR_INVALID, "unknown option %d", option);
}

int atp_terrain_prepare(atp_ctx *ctx, const float *heights_dev, const float *costmap_dev, int nx,
                        int ny, double cell, double x0, double y0, int format, void *texels_dev,
                        atp_terrain *out, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (!heights_dev || !texels_dev) return fail(ctx, ATP_ERR_INVALID, "heights or texels is NULL");
    if (nx < 3 || ny < 3 || nx > 65536 || ny > 65536)
        return fail(ctx, ATP_ERR_INVALID, "terrain must be between 3 and 65536 nodes per side");
    if (!(cell > 0.0) || !std::isfinite(cell) || !std::isfinite(x0) || !std::isfinite(y0))
        return fail(ctx, ATP_ERR_INVALID, "cell must be > 0 and origin finite");
    if (format != ATP_TERRAIN_F32X4 && format != ATP_TERRAIN_BF16X4)
        return fail(ctx, ATP_ERR_UNSUPPORTED, "terrain format %d not supported", format);
    if ((uintptr_t)texels_dev % 16 != 0) return fail(ctx, ATP_ERR_INVALID, "texels must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    cudaError_t e;
    if (format == ATP_TERRAIN_F32X4)
        e = atp::launch_terrain_prepare_f32(heights_dev, costmap_dev, nx, ny, (float)(1.0 / cell),
                                            (float4 *)texels_dev, (cudaStream_t)stream);
    else
        e = atp::launch_terrain_prepare_bf16(heights_dev, costmap_dev, nx, ny, (float)(1.0 / cell),
                                             (uint2 *)texels_dev,
                                             (float4 *)((char *)texels_dev + atp::bf16_base_offset(nx, ny)),
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "terrain prepare launch");
    if (out) {
        out->texels = texels_dev;
        out->nx = nx;
        out->ny = ny;
        out->cell = cell;
        out->x0 = x0;
        out->y0 = y0;
        out->format = format;
        out->flags = costmap_dev ? ATP_TERRAIN_HAS_COSTMAP : 0;
    }
    return ATP_OK;
}

int atp_plan(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost, const atp_terrain *terrain,
             const atp_state *x0, const float *x0_dev, const float *ctrl_dev, int N, int H, float dt,
             int n_sub, atp_plan_out *out_dev, float *best_ctrl_dev, float *best_margin_dev,
             float *cand_cost_dev, float *cand_margin_dev, uint8_t *cand_flags_dev,
             float *cand_xf_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int ns = 0;
    int rc = common_checks(ctx, veh, cost, terrain, x0 ? &x0->x : nullptr, 13, x0_dev, ctrl_dev, N, H, dt,
                           n_sub, &ns);
    if (rc != ATP_OK) return rc;
    if (!out_dev) return fail(ctx, ATP_ERR_INVALID, "out_dev is NULL");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    const bool steps = best_margin_dev != nullptr;
    if ((rc = ensure_scratch(ctx, N, H, steps)) != ATP_OK) return rc;
    const RegionLayout L = region_layout((size_t)N, (size_t)H, steps);
    char *base = (char *)ctx->scratch + kHeaderBytes;
    atp::PlanParams p;
    std::memset(&p, 0, sizeof p);
    derive(*veh, *cost, *terrain, p);
    fill_problem(p, x0, x0_dev, ctrl_dev, N, H, dt, ns);
    p.cost = cand_cost_dev ? cand_cost_dev : (float *)(base + L.cost);
    p.margin = cand_margin_dev ? cand_margin_dev : (float *)(base + L.margin);
    p.flags = cand_flags_dev ? cand_flags_dev : (uint8_t *)(base + L.flags);
    p.xf = cand_xf_dev;
    p.min_step = (int *)(base + L.min_step);
    p.step_margin = steps ? (float *)(base + L.step_margin) : nullptr;
    p.out = out_dev;
    p.best_ctrl = best_ctrl_dev;
    p.best_margin = best_margin_dev;
    p.scratch = (atp::Scratch *)ctx->scratch;
    p.acc64 = ctx->acc64;
    p.lanes = ctx->lanes;
    cudaError_t e = launch_plan_for(ctx, p, *terrain, true, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plan launch");
    return ATP_OK;
}

int atp_rollout(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost, const atp_terrain *terrain,
                const atp_state *x0, const float *x0_dev, const float *ctrl_dev, int N, int H,
                float dt, int n_sub, float *cand_cost_dev, float *cand_margin_dev,
                uint8_t *cand_flags_dev, float *cand_xf_dev, float *step_margin_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int ns = 0;
    int rc = common_checks(ctx, veh, cost, terrain, x0 ? &x0->x : nullptr, 13, x0_dev, ctrl_dev, N, H, dt,
                           n_sub, &ns);
    if (rc != ATP_OK) return rc;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    atp::PlanParams p;
    std::memset(&p, 0, sizeof p);
    derive(*veh, *cost, *terrain, p);
    fill_problem(p, x0, x0_dev, ctrl_dev, N, H, dt, ns);
    p.cost = cand_cost_dev;
    p.margin = cand_margin_dev;
    p.flags = cand_flags_dev;
    p.xf = cand_xf_dev;
    p.step_margin = step_margin_dev;
    p.acc64 = ctx->acc64;
    p.lanes = ctx->lanes;
    cudaError_t e = launch_plan_for(ctx, p, *terrain, false, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rollout launch");
    return ATP_OK;
}

}  // extern "C"

extern "C" int atp_plan_lanes(const atp_ctx *ctx, int N)
{
    if (!ctx || N < 1) return ATP_ERR_INVALID;
    return atp::plan_lanes(ctx->lanes, N);
}

extern "C" int atp_plan_batch(atp_ctx *ctx, const atp_plan_request *reqs, int n_req, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (!reqs || n_req < 1 || n_req > atp::kMaxBatch)
        return fail(ctx, ATP_ERR_INVALID, "need 1 <= n_req <= %d requests", atp::kMaxBatch);
    size_t need = 0;
    long long ctas = 0, threads = 0;
    int ns[atp::kMaxBatch], lanes[atp::kMaxBatch];
    for (int r = 0; r < n_req; ++r) {
        const atp_plan_request &q = reqs[r];
        int rc = common_checks(ctx, q.veh, q.cost, q.terrain, q.x0 ? &q.x0->x : nullptr, 13, q.x0_dev,
                               q.ctrl_dev, q.N, q.H,
                               q.dt, q.n_sub, &ns[r]);
        if (rc != ATP_OK) {
            char why[sizeof ctx->err];
            std::memcpy(why, ctx->err, sizeof why);
            return fail(ctx, rc, "request %d: %s", r, why);
        }
        if (!q.out_dev) return fail(ctx, ATP_ERR_INVALID, "request %d: out_dev is NULL", r);
        if (q.N > (1 << 29)) return fail(ctx, ATP_ERR_UNSUPPORTED, "request %d: N too large for a batch", r);
        need += region_layout((size_t)q.N, (size_t)q.H, q.best_margin_dev != nullptr).total;
        lanes[r] = ctx->lanes ? ctx->lanes : 1;
        threads += (long long)q.N * lanes[r];
    }
    // Several lanes per candidate pay only while the GPU is mostly empty, and
    // every layout gives the same bits, so the batch chooses each plan's
    // lanes for the batch as a whole (unless ATP_OPT_LANES forces them):
    // every plan starts at one lane, and in request order a plan that would
    // run four (or two) lanes alone gets them while the batch's threads stay
    // within what a two-lane plan alone may use, else two if those fit.
    // Measured on the GB300 on the 32-vehicle serving mix: at 80 requests/s
    // per vehicle p99 fell from 55 to 32 ms, unchanged at 20 to 40.
    if (!ctx->lanes) {
        const long long budget = 2LL * atp::kLanes2MaxN;
        for (int r = 0; r < n_req; ++r) {
            const long long N = reqs[r].N;
            const int alone = atp::plan_lanes(0, reqs[r].N);
            if (alone == 4 && threads + 3 * N <= budget) {
                lanes[r] = 4;
                threads += 3 * N;
            } else if (alone >= 2 && threads + N <= budget) {
                lanes[r] = 2;
                threads += N;
            }
        }
    }
    for (int r = 0; r < n_req; ++r)
        ctas += ((long long)reqs[r].N * lanes[r] + atp::kPlanBlock - 1) / atp::kPlanBlock;
    if (ctas > 0x7fffffffLL) return fail(ctx, ATP_ERR_UNSUPPORTED, "batch too large");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    int rc = ensure_scratch_bytes(ctx, need);
    if (rc != ATP_OK) return rc;
    atp::BatchParams &b = *ctx->batch;
    b.n = n_req;
    b.cta_begin[0] = 0;
    char *region = (char *)ctx->scratch + kHeaderBytes;
    for (int r = 0; r < n_req; ++r) {
        const atp_plan_request &q = reqs[r];
        const bool steps = q.best_margin_dev != nullptr;
        const RegionLayout L = region_layout((size_t)q.N, (size_t)q.H, steps);
        atp::PlanParams &p = b.req[r];
        std::memset(&p, 0, sizeof p);
        derive(*q.veh, *q.cost, *q.terrain, p);
        fill_problem(p, q.x0, q.x0_dev, q.ctrl_dev, q.N, q.H, q.dt, ns[r]);
        p.cost = q.cand_cost_dev ? q.cand_cost_dev : (float *)(region + L.cost);
        p.margin = q.cand_margin_dev ? q.cand_margin_dev : (float *)(region + L.margin);
        p.flags = q.cand_flags_dev ? q.cand_flags_dev : (uint8_t *)(region + L.flags);
        p.xf = q.cand_xf_dev;
        p.min_step = (int *)(region + L.min_step);
        p.step_margin = steps ? (float *)(region + L.step_margin) : nullptr;
        p.out = q.out_dev;
        p.best_ctrl = q.best_ctrl_dev;
        p.best_margin = q.best_margin_dev;
        p.scratch = (atp::Scratch *)ctx->scratch + r;
        p.acc64 = ctx->acc64;
        p.lanes = lanes[r];
        region += L.total;
        b.cta_begin[r + 1] = b.cta_begin[r] + (int)(((long long)q.N * p.lanes + atp::kPlanBlock - 1) / atp::kPlanBlock);
    }
    cudaError_t e = atp::launch_plan_batch(b, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch launch");
    return ATP_OK;
}

extern "C" int atp_plan_est(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
                            const atp_terrain *terrain, const atp_est_state *x0, const float *x0_dev,
                            const float *ctrl_dev, int N, int H, float dt, int n_sub,
                            atp_plan_out *out_dev, float *best_ctrl_dev, float *best_margin_dev,
                            float *cand_cost_dev, float *cand_margin_dev, uint8_t *cand_flags_dev,
                            float *cand_xf_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int ns = 0;
    int rc = common_checks(ctx, veh, cost, terrain, x0 ? &x0->x : nullptr, 7, x0_dev, ctrl_dev, N, H, dt,
                           n_sub, &ns);
    if (rc != ATP_OK) return rc;
    if (!out_dev) return fail(ctx, ATP_ERR_INVALID, "out_dev is NULL");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    const bool steps = best_margin_dev != nullptr;
    if ((rc = ensure_scratch(ctx, N, H, steps)) != ATP_OK) return rc;
    const RegionLayout L = region_layout((size_t)N, (size_t)H, steps);
    char *base = (char *)ctx->scratch + kHeaderBytes;
    atp::PlanParams p;
    std::memset(&p, 0, sizeof p);
    derive(*veh, *cost, *terrain, p);
    // the lateral-acceleration constraint's normaliser (reading Q2)
    const double abar = veh->g * veh->e / (2.0 * veh->hR);
    p.C.inv_eps = (float)(1.0 / (cost->eps_esm > 0 ? cost->eps_esm : 0.1 * abar));
    if (x0) {
        std::memcpy(p.x0, &x0->x, 7 * sizeof(float));
        p.x0_soa = nullptr;
    } else {
        p.x0_soa = x0_dev;
    }
    p.ctrl = (const float2 *)ctrl_dev;
    p.N = N;
    p.H = H;
    p.n_sub = ns;
    p.h = (float)((double)dt / (double)ns);
    p.cost = cand_cost_dev ? cand_cost_dev : (float *)(base + L.cost);
    p.margin = cand_margin_dev ? cand_margin_dev : (float *)(base + L.margin);
    p.flags = cand_flags_dev ? cand_flags_dev : (uint8_t *)(base + L.flags);
    p.xf = cand_xf_dev;
    p.min_step = (int *)(base + L.min_step);
    p.step_margin = steps ? (float *)(base + L.step_margin) : nullptr;
    p.out = out_dev;
    p.best_ctrl = best_ctrl_dev;
    p.best_margin = best_margin_dev;
    p.scratch = (atp::Scratch *)ctx->scratch;
    p.acc64 = ctx->acc64;
    cudaError_t e = atp::launch_est(p, true, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "planar plan launch");
    return ATP_OK;
}

extern "C" int atp_lod_smooth(atp_ctx *ctx, const float *heights_dev, int nx, int ny, double cell,
                              double sigma, float *tmp_dev, float *out_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (!heights_dev || !tmp_dev || !out_dev) return fail(ctx, ATP_ERR_INVALID, "a buffer is NULL");
    if (tmp_dev == heights_dev || tmp_dev == out_dev)
        return fail(ctx, ATP_ERR_INVALID, "tmp_dev must alias neither heights_dev nor out_dev");
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536)
        return fail(ctx, ATP_ERR_INVALID, "map must be between 1 and 65536 nodes per side");
    if (!(cell > 0.0) || !std::isfinite(cell) || !(sigma >= 0.0) || !std::isfinite(sigma))
        return fail(ctx, ATP_ERR_INVALID, "cell must be > 0 and sigma >= 0, both finite");
    const double s = sigma / cell;                      // standard deviation in cells
    const double rr = 4.0 * s + 0.5;
    if (rr >= (double)atp::kLodMaxRadius + 1.0)
        return fail(ctx, ATP_ERR_UNSUPPORTED, "Gaussian radius above %d cells", atp::kLodMaxRadius);
    const int r = sigma > 0.0 ? (int)rr : 0;
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    const float inv2s2 = r > 0 ? (float)(0.5 / (s * s)) : 0.f;
    cudaError_t e = atp::launch_lod_smooth(heights_dev, tmp_dev, out_dev, nx, ny, r, inv2s2,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "level-of-detail launch");
    return ATP_OK;
}

extern "C" int atp_costmap(atp_ctx *ctx, const double *xy_dev, const int *start, const int *kind,
                           int n_poly, int nx, int ny, double cell, double x0, double y0, double eps,
                           double sigma, float *cost_dev, float *sdist_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (!xy_dev || !start || !kind || !cost_dev) return fail(ctx, ATP_ERR_INVALID, "a buffer is NULL");
    if (n_poly < 1 || n_poly > atp::kCostmapMaxPolys)
        return fail(ctx, ATP_ERR_INVALID, "need 1 <= n_poly <= %d", atp::kCostmapMaxPolys);
    if (start[0] != 0) return fail(ctx, ATP_ERR_INVALID, "start[0] must be 0");
    for (int q = 0; q < n_poly; ++q) {
        if (start[q + 1] - start[q] < 2)
            return fail(ctx, ATP_ERR_INVALID, "perimeter %d has fewer than 2 vertices", q);
        if (kind[q] != 0 && kind[q] != 1) return fail(ctx, ATP_ERR_INVALID, "kind[%d] must be 0 or 1", q);
    }
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536)
        return fail(ctx, ATP_ERR_INVALID, "map must be between 1 and 65536 nodes per side");
    if (!(cell > 0.0) || !std::isfinite(cell) || !std::isfinite(x0) || !std::isfinite(y0) || !(eps > 0.0) ||
        !std::isfinite(eps) || !(sigma >= 0.0) || !std::isfinite(sigma))
        return fail(ctx, ATP_ERR_INVALID, "cell, eps must be > 0, sigma >= 0, all finite");
    if ((uintptr_t)xy_dev % 8 != 0) return fail(ctx, ATP_ERR_INVALID, "xy_dev must be 8-byte aligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    atp::CostmapParams p;
    std::memset(&p, 0, sizeof p);
    p.xy = xy_dev;
    p.n_poly = n_poly;
    p.n_vert = start[n_poly];
    for (int q = 0; q <= n_poly; ++q) p.start[q] = start[q];
    for (int q = 0; q < n_poly; ++q) p.kind[q] = kind[q];
    p.nx = nx;
    p.ny = ny;
    p.cell = cell;
    p.x0 = x0;
    p.y0 = y0;
    p.inv_eps = (float)(1.0 / eps);
    p.sigma = (float)sigma;
    p.cost = cost_dev;
    p.sdist = sdist_dev;
    // An obstacle farther than eps from a node adds nothing there; the boxes
    // are grown by twice that plus a margin for the FP32 distance arithmetic
    // (a few ulps of the map's extent), so a skipped obstacle's rate is
    // exactly zero at every node of a tile it misses.
    const double ext = std::max((double)(nx - 1), (double)(ny - 1)) * cell;
    const float reach = (float)(2.0 * eps + 1e-3 + 1e-5 * ext);
    cudaError_t e = atp::launch_costmap(p, ctx->cm_box, reach, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "costmap launch");
    return ATP_OK;
}

namespace {

int grad_impl(atp_ctx *ctx, int objective, const atp_vehicle *veh, const atp_cost *cost,
              const atp_terrain *terrain, const atp_state *x0, const float *x0_dev, const float *ctrl_dev,
              int K, int H, float dt, int n_sub, int ckpt, float *cost_dev, float *grad_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int ns = 0;
    int rc = common_checks(ctx, veh, cost, terrain, x0 ? &x0->x : nullptr, 13, x0_dev, ctrl_dev, K, H, dt,
                           n_sub, &ns);
    if (rc != ATP_OK) return rc;
    if (terrain->format != ATP_TERRAIN_F32X4)
        return fail(ctx, ATP_ERR_UNSUPPORTED, "the adjoint takes F32X4 terrain only");
    // four lanes per candidate, up to twice in a CTA: the lane slot stays within 32 bits
    if (K > (1 << 28)) return fail(ctx, ATP_ERR_UNSUPPORTED, "the adjoint takes at most 2^28 candidates");
    if (!cost_dev || !grad_dev) return fail(ctx, ATP_ERR_INVALID, "cost_dev and grad_dev are required");
    if (ckpt == 0) ckpt = 10;
    if (ckpt < 1) return fail(ctx, ATP_ERR_INVALID, "ckpt must be >= 1 (0 selects 10)");
    if (ckpt > H) ckpt = H;
    const size_t n_seg = (size_t)(H + ckpt - 1) / ckpt;
    const size_t KL = (size_t)K * atp::kGradLanes;      // every lane keeps its own states
    const size_t ck_bytes = align_up(n_seg * 20 * KL * sizeof(float));
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    if (ctx->grad_ctas < 0) ctx->grad_ctas = atp::grad_split_ctas(ctx->device);
    // walking and recomputing on separate warps pays while one wave holds the grid
    const bool split = ((size_t)K + atp::kGradCands - 1) / atp::kGradCands <= (size_t)ctx->grad_ctas;
    const size_t seg_bytes = align_up((split ? 2 : 1) * (size_t)ckpt * ns * 20 * KL * sizeof(float));
    if ((rc = ensure_scratch_bytes(ctx, ck_bytes + seg_bytes)) != ATP_OK) return rc;
    char *base = (char *)ctx->scratch + kHeaderBytes;
    atp::PlanParams pp;
    std::memset(&pp, 0, sizeof pp);
    derive(*veh, *cost, *terrain, pp);
    fill_problem(pp, x0, x0_dev, ctrl_dev, K, H, dt, ns);
    atp::GradParams p;
    std::memset(&p, 0, sizeof p);
    p.V = pp.V;
    p.C = pp.C;
    p.T = pp.T;
    std::memcpy(p.x0, pp.x0, sizeof p.x0);
    p.x0_soa = pp.x0_soa;
    p.ctrl = pp.ctrl;
    p.K = K;
    p.H = H;
    p.n_sub = ns;
    p.ckpt = ckpt;
    p.h = pp.h;
    p.objective = objective;
    p.split = split;
    p.cost = cost_dev;
    p.grad = grad_dev;
    p.ckpt_buf = (float *)base;
    p.seg_buf = (float *)(base + ck_bytes);
    cudaError_t e = atp::launch_grad(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "grad launch");
    return ATP_OK;
}

}  // namespace

extern "C" int atp_grad(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
                        const atp_terrain *terrain, const atp_state *x0, const float *x0_dev,
                        const float *ctrl_dev, int K, int H, float dt, int n_sub, int ckpt,
                        float *cost_dev, float *grad_dev, void *stream)
{
    return grad_impl(ctx, atp::kGradCost, veh, cost, terrain, x0, x0_dev, ctrl_dev, K, H, dt, n_sub, ckpt,
                     cost_dev, grad_dev, stream);
}

extern "C" int atp_grad_margin(atp_ctx *ctx, const atp_vehicle *veh, const atp_cost *cost,
                               const atp_terrain *terrain, const atp_state *x0, const float *x0_dev,
                               const float *ctrl_dev, int K, int H, float dt, int n_sub, int ckpt,
                               float *margin_dev, float *grad_dev, void *stream)
{
    return grad_impl(ctx, atp::kGradMargin, veh, cost, terrain, x0, x0_dev, ctrl_dev, K, H, dt, n_sub, ckpt,
                     margin_dev, grad_dev, stream);
}

namespace {

bool al8(const void *p) { return (uintptr_t)p % 8 == 0; }

int refine_checks(atp_ctx *ctx, int K, int H)
{
    if (K < 1 || H < 1) return fail(ctx, ATP_ERR_INVALID, "need K >= 1 and H >= 1");
    if (K > kMaxN) return fail(ctx, ATP_ERR_UNSUPPORTED, "K above %d", kMaxN);
    return ATP_OK;
}

}  // namespace

extern "C" int atp_refine_init(atp_ctx *ctx, const float *grad_dev, int K, int H, float step, float *eta_dev,
                               void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int rc = refine_checks(ctx, K, H);
    if (rc != ATP_OK) return rc;
    if (!grad_dev || !eta_dev || !al8(grad_dev)) return fail(ctx, ATP_ERR_INVALID, "grad_dev (8-byte aligned) and eta_dev are required");
    if (!(step > 0.f) || !std::isfinite(step)) return fail(ctx, ATP_ERR_INVALID, "step must be finite and > 0");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    cudaError_t e = atp::launch_refine_init(grad_dev, K, H, step, eta_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refine launch");
    return ATP_OK;
}

extern "C" int atp_refine_trial(atp_ctx *ctx, const float *ctrl_dev, const float *grad_dev, const float *eta_dev,
                                int K, int H, float rate_max, float *trial_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int rc = refine_checks(ctx, K, H);
    if (rc != ATP_OK) return rc;
    if (!ctrl_dev || !grad_dev || !eta_dev || !trial_dev || !al8(ctrl_dev) || !al8(grad_dev) || !al8(trial_dev))
        return fail(ctx, ATP_ERR_INVALID, "a buffer is NULL or a [H][K][2] buffer not 8-byte aligned");
    if (!(rate_max >= 0.f) || !std::isfinite(rate_max))
        return fail(ctx, ATP_ERR_INVALID, "rate_max must be finite and >= 0");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    cudaError_t e = atp::launch_refine_trial(ctrl_dev, grad_dev, eta_dev, K, H, rate_max, trial_dev,
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refine launch");
    return ATP_OK;
}

extern "C" int atp_refine_accept(atp_ctx *ctx, int K, int H, const float *trial_dev, const float *trial_cost_dev,
                                 const float *trial_grad_dev, float *ctrl_dev, float *cost_dev, float *grad_dev,
                                 float *eta_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    int rc = refine_checks(ctx, K, H);
    if (rc != ATP_OK) return rc;
    if (!trial_dev || !trial_cost_dev || !trial_grad_dev || !ctrl_dev || !cost_dev || !grad_dev || !eta_dev ||
        !al8(trial_dev) || !al8(trial_grad_dev) || !al8(ctrl_dev) || !al8(grad_dev))
        return fail(ctx, ATP_ERR_INVALID, "a buffer is NULL or a [H][K][2] buffer not 8-byte aligned");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    cudaError_t e = atp::launch_refine_accept(K, H, trial_dev, trial_cost_dev, trial_grad_dev, ctrl_dev, cost_dev,
                                              grad_dev, eta_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "refine launch");
    return ATP_OK;
}

extern "C" int atp_sample(atp_ctx *ctx, const float *prev_best_dev, int H_prev, int shift,
                          double sigma_rate, double sigma_acc, uint64_t key0, uint64_t key1,
                          uint64_t nonce, int N, int H, float *ctrl_dev, void *stream)
{
    if (!ctx) return ATP_ERR_INVALID;
    if (!ctrl_dev || (uintptr_t)ctrl_dev % 8 != 0)
        return fail(ctx, ATP_ERR_INVALID, "ctrl_dev must be non-NULL and 8-byte aligned");
    if (N < 1 || H < 1 || H > 65535) return fail(ctx, ATP_ERR_INVALID, "need N >= 1 and 1 <= H <= 65535");
    if (N > kMaxN) return fail(ctx, ATP_ERR_UNSUPPORTED, "N above %d", kMaxN);
    if (H_prev < 0 || shift < 0) return fail(ctx, ATP_ERR_INVALID, "H_prev and shift must be >= 0");
    if (H_prev > 0 && (!prev_best_dev || (uintptr_t)prev_best_dev % 8 != 0))
        return fail(ctx, ATP_ERR_INVALID, "prev_best_dev must be non-NULL and 8-byte aligned");
    if (!(sigma_rate >= 0.0) || !(sigma_acc >= 0.0) || !std::isfinite(sigma_rate) || !std::isfinite(sigma_acc))
        return fail(ctx, ATP_ERR_INVALID, "sigmas must be finite and >= 0");
    DeviceGuard g(ctx->device);
    if (g.err != cudaSuccess) return cuda_fail(ctx, g.err, "set device");
    atp::SampleParams p;
    p.prev = H_prev > 0 ? (const float2 *)prev_best_dev : nullptr;
    p.H_prev = H_prev;
    p.shift = shift;
    p.sigma_rate = (float)sigma_rate;
    p.sigma_acc = (float)sigma_acc;
    p.key0 = key0;
    p.key1 = key1;
    p.nonce = nonce;
    p.N = N;
    p.H = H;
    p.ctrl = (float2 *)ctrl_dev;
    cudaError_t e = atp::launch_sample(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sample launch");
    return ATP_OK;
}

// ---------------------------------------------------------------------------
// Plan without allocation.  Some callers cannot allocate device memory once
// they are running, for example a planner in a hard real-time control loop
// whose latency budget or certification forbids cudaMalloc after start-up,
// or a plugin host that gives its plugins no allocator.  atp_plan_noalloc
// runs the same kernel as atp_plan, but its scratch is the file-scope array
// below, which every GPU that loads this library holds until the process ends.

namespace {

constexpr size_t kNoallocScratchBytes = 8u << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_plan_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];

// Device address of g_plan_scratch on the current device.  Host code only
// sees a host-side stand-in for the array's name, so the address is looked up
// once per device with that device current.
int noalloc_scratch(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_plan_scratch) != cudaSuccess || !p) return ATP_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return ATP_OK;
}

}  // namespace

extern "C" int atp_plan_noalloc(const atp_vehicle *veh, const atp_cost *cost,
                                const atp_terrain *terrain, const atp_state *x0,
                                const float *x0_dev, const float *ctrl_dev, int N, int H,
                                float dt, int n_sub, atp_plan_out *out_dev, float *best_ctrl_dev,
                                float *best_margin_dev, float *cand_cost_dev,
                                float *cand_margin_dev, uint8_t *cand_flags_dev,
                                float *cand_xf_dev, void *stream)
{
    int ns = 0;
    int rc = common_checks(nullptr, veh, cost, terrain, x0 ? &x0->x : nullptr, 13, x0_dev, ctrl_dev, N, H, dt,
                           n_sub, &ns);
    if (rc != ATP_OK) return rc;
    if (!out_dev) return ATP_ERR_INVALID;
    const bool steps = best_margin_dev != nullptr;
    const RegionLayout L = layout((size_t)N, (size_t)H, steps);
    if (L.total > kNoallocScratchBytes) return ATP_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return ATP_ERR_CUDA;
    if (dev >= kMaxDevices) return ATP_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    if ((rc = noalloc_scratch(dev, &scratch)) != ATP_OK) return rc;
    char *base = (char *)scratch;
    // the reduction key starts at all ones, the count and ticket at zero; the
    // kernel's last CTA leaves them so, but a fresh process or an earlier
    // failed launch may not have
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(base, 0xff, sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemsetAsync(base + sizeof(unsigned long long), 0,
                        sizeof(atp::Scratch) - sizeof(unsigned long long), s) != cudaSuccess)
        return ATP_ERR_CUDA;
    atp::PlanParams p;
    std::memset(&p, 0, sizeof p);
    derive(*veh, *cost, *terrain, p);
    fill_problem(p, x0, x0_dev, ctrl_dev, N, H, dt, ns);
    p.cost = cand_cost_dev ? cand_cost_dev : (float *)(base + L.cost);
    p.margin = cand_margin_dev ? cand_margin_dev : (float *)(base + L.margin);
    p.flags = cand_flags_dev ? cand_flags_dev : (uint8_t *)(base + L.flags);
    p.xf = cand_xf_dev;
    p.min_step = (int *)(base + L.min_step);
    p.step_margin = steps ? (float *)(base + L.step_margin) : nullptr;
    p.out = out_dev;
    p.best_ctrl = best_ctrl_dev;
    p.best_margin = best_margin_dev;
    p.scratch = (atp::Scratch *)base;
    if (atp::launch_plan(p, true, s) != cudaSuccess) return ATP_ERR_CUDA;
    return ATP_OK;
}
