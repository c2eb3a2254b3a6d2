// sampler.cuh - parameters of the on-device candidate sampler.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace atp {

struct SampleParams {
    const float2 *prev;       // warm start [H_prev] or nullptr
    int H_prev, shift;
    float sigma_rate, sigma_acc;
    uint64_t key0, key1, nonce;
    int N, H;
    float2 *ctrl;             // [H][N]
};

cudaError_t launch_sample(const SampleParams &p, cudaStream_t stream);

}  // namespace atp
