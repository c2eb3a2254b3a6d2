// refine.cuh - launchers of the gradient-refinement step kernels.
#pragma once

#include <cuda_runtime.h>

namespace atp {

cudaError_t launch_refine_init(const float *grad, int K, int H, float step, float *eta, cudaStream_t stream);
cudaError_t launch_refine_trial(const float *ctrl, const float *grad, const float *eta, int K, int H,
                                float rate_max, float *trial, cudaStream_t stream);
cudaError_t launch_refine_accept(int K, int H, const float *trial, const float *trial_cost, const float *trial_grad,
                                 float *ctrl, float *cost, float *grad, float *eta, cudaStream_t stream);

}  // namespace atp
