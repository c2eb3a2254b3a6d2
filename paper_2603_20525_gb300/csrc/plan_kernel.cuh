// plan_kernel.cuh - parameters and launchers of the fused rollout + argmin
// kernel (arxiv 2603.20525, Sec. IV-A..IV-D).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "atp.h"
#include "srb_model.cuh"

namespace atp {

// Reduction scratch of one plan: the packed argmin key, the feasible count and
// the ticket that elects the last CTA.  The last CTA restores the initial
// values, so consecutive plans on one stream need no memset.
struct Scratch {
    unsigned long long key;   // initial ~0ull
    unsigned int count;       // initial 0
    unsigned int ticket;      // initial 0
};

struct PlanParams {
    Veh V;
    Cost C;
    Terrain T;
    float x0[13];             // shared initial state (x0_soa == nullptr)
    const float *x0_soa;      // [13][N] per-candidate initial states, or nullptr
    const float2 *ctrl;       // [H][N]
    int N, H, n_sub;
    float h;                  // Euler step dt / n_sub
    float *cost;              // [N] or nullptr
    float *margin;            // [N] or nullptr
    uint8_t *flags;           // [N] or nullptr
    float *xf;                // [13][N] or nullptr
    float *step_margin;       // [H][N] or nullptr: each control step's minimum U_ESM
    int *min_step;            // [N] or nullptr: control step of each candidate's smallest
                              // per-step margin (the final state folded into step H-1)
    int tex_format;           // TEX_F32 or TEX_BF16
    int acc64;                // accumulate the running cost in FP64
    int lanes;                // 0: by batch size; else 1, 2 or 4 lanes per candidate
    // plan only
    atp_plan_out *out;
    float *best_ctrl;         // [H][2] or nullptr
    float *best_margin;       // [H] or nullptr
    Scratch *scratch;
};

constexpr int kPlanBlock = 64;
// Threads per candidate by batch size, from a sweep of the three layouts on
// a GB300 (scaled workload, H = 100, 4 Euler steps per control step, L2
// flushed before each plan): four lanes (one wheel each) are fastest up to
// 12288 candidates, two (one axle each) at 16384 and 24576, one from 32768 on.
constexpr int kLanes4MaxN = 12288;
constexpr int kLanes2MaxN = 28672;

// threads per candidate: `forced` (1, 2 or 4) if set, else by batch size
inline int plan_lanes(int forced, int N)
{
    return forced ? forced : (N <= kLanes4MaxN ? 4 : N <= kLanes2MaxN ? 2 : 1);
}
cudaError_t launch_plan(const PlanParams &p, bool reduce, cudaStream_t stream);

// Terrain staging (one lane per candidate, F32 texels, a shared start
// state): CTAs of kStageBlock threads, each of which first copies the window
// p.T.(wx0, wy0, ww, wh) of the texel array into its shared memory.
constexpr int kStageBlock = 512;
constexpr int kStageMaxSide = 120;     // 120 x 120 texels = 225 KB
cudaError_t launch_plan_staged(const PlanParams &p, bool reduce, cudaStream_t stream);

// A ragged batch of plans in one launch.  The descriptors travel in the
// kernel's parameter block (at most 32 KB), so a batch needs no device copy.
constexpr int kMaxBatch = 64;
struct BatchParams {
    int n;
    int cta_begin[kMaxBatch + 1];   // CTA prefix: plan r owns [cta_begin[r], cta_begin[r+1])
    PlanParams req[kMaxBatch];
};
static_assert(sizeof(BatchParams) <= 32764, "batch descriptors exceed the kernel parameter limit");

cudaError_t launch_plan_batch(const BatchParams &b, cudaStream_t stream);
cudaError_t launch_terrain_prepare_f32(const float *heights, const float *costmap, int nx, int ny,
                                       float inv_cell, float4 *out, cudaStream_t stream);
cudaError_t launch_terrain_prepare_bf16(const float *heights, const float *costmap, int nx, int ny,
                                        float inv_cell, uint2 *texels, float4 *plane, cudaStream_t stream);

// byte offset of the BF16 block planes after the texels
inline size_t bf16_base_offset(int nx, int ny) { return ((size_t)nx * ny * 8 + 255) / 256 * 256; }

}  // namespace atp
