// adjoint.cuh - parameters of the rollout-cost adjoint kernel.
#pragma once

#include <cuda_runtime.h>

#include "srb_model.cuh"

namespace atp {

// threads per candidate in the adjoint (one wheel each)
constexpr int kGradLanes = 4;
// candidates per CTA; the CTA holds them twice (walking and recomputing)
constexpr int kGradCands = 16;
constexpr int kGradHalf = kGradCands * kGradLanes;
// what the adjoint differentiates
constexpr int kGradCost = 0, kGradMargin = 1;

struct GradParams {
    Veh V;
    Cost C;
    Terrain T;
    float x0[13];             // shared initial state (x0_soa == nullptr)
    const float *x0_soa;      // [13][K] or nullptr
    const float2 *ctrl;       // [H][K]
    int K, H, n_sub, ckpt;
    float h;
    int objective;            // kGradCost: J; kGradMargin: min U_ESM over the trajectory
    int split;                // walk and recompute on separate warps (two buffers), else one
                              // quad per candidate does both (one buffer)
    float *cost;              // [K] the objective's value
    float *grad;              // [H][K][2]
    float *ckpt_buf;          // [ceil(H / ckpt)][20][K * kGradLanes]
    float *seg_buf;           // [1 or 2][ckpt * n_sub][20][K * kGradLanes]
};

// CTAs of the split layout (kGradCands candidates each) resident at once on
// `device`, 0 if the query fails; the split layout pays while one wave holds
// the grid
int grad_split_ctas(int device);
cudaError_t launch_grad(const GradParams &p, cudaStream_t stream);

}  // namespace atp
