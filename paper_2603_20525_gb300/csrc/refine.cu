// refine.cu - projected-gradient refinement of candidate control sequences
// with the adjoint's gradient (atp_grad): the step arithmetic of one
// iteration, one thread per candidate (K is small: the refined candidates are
// the best few of a plan).  Layouts as the plan kernel's: ctrl, grad [H][K][2]
// (steering rate, acceleration), cost and step size [K].
#include <cuda_runtime.h>

#include "refine.cuh"

namespace atp {

namespace {

// eta[j] = step / (max over k, c of |grad[k][j][c]| + 1e-12)
__global__ void refine_init_kernel(const float *__restrict__ grad, int K, int H, float step, float *__restrict__ eta)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    float m = 0.f;
    for (int k = 0; k < H; ++k) {
        const float2 g = reinterpret_cast<const float2 *>(grad)[(size_t)k * K + j];
        m = fmaxf(m, fmaxf(fabsf(g.x), fabsf(g.y)));
    }
    eta[j] = step / (m + 1e-12f);
}

// trial = ctrl - eta[j] grad, the steering rate projected onto its limit
// (the admissible set of Sec. IV-C)
__global__ void refine_trial_kernel(const float2 *__restrict__ ctrl, const float2 *__restrict__ grad,
                                    const float *__restrict__ eta, int K, int H, float rate_max,
                                    float2 *__restrict__ trial)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const float e = eta[j];
    for (int k = 0; k < H; ++k) {
        const size_t i = (size_t)k * K + j;
        const float2 u = ctrl[i], g = grad[i];
        float r = fmaf(-e, g.x, u.x);
        r = fminf(fmaxf(r, -rate_max), rate_max);
        trial[i] = make_float2(r, fmaf(-e, g.y, u.y));
    }
}

// accept the trial of candidate j where its cost is finite and lower: the
// controls, gradient and cost become the trial's and the step grows by 1.5;
// otherwise the step halves
__global__ void refine_accept_kernel(int K, int H, const float2 *__restrict__ trial,
                                     const float *__restrict__ trial_cost, const float2 *__restrict__ trial_grad,
                                     float2 *__restrict__ ctrl, float *__restrict__ cost, float2 *__restrict__ grad,
                                     float *__restrict__ eta)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const float Jt = trial_cost[j];
    const bool ok = isfinite(Jt) && Jt < cost[j];
    if (ok) {
        for (int k = 0; k < H; ++k) {
            const size_t i = (size_t)k * K + j;
            ctrl[i] = trial[i];
            grad[i] = trial_grad[i];
        }
        cost[j] = Jt;
    }
    eta[j] *= ok ? 1.5f : 0.5f;
}

constexpr int kBlock = 128;

unsigned blocks(int K) { return (unsigned)((K + kBlock - 1) / kBlock); }

}  // namespace

cudaError_t launch_refine_init(const float *grad, int K, int H, float step, float *eta, cudaStream_t stream)
{
    refine_init_kernel<<<blocks(K), kBlock, 0, stream>>>(grad, K, H, step, eta);
    return cudaGetLastError();
}

cudaError_t launch_refine_trial(const float *ctrl, const float *grad, const float *eta, int K, int H,
                                float rate_max, float *trial, cudaStream_t stream)
{
    refine_trial_kernel<<<blocks(K), kBlock, 0, stream>>>((const float2 *)ctrl, (const float2 *)grad, eta, K, H,
                                                          rate_max, (float2 *)trial);
    return cudaGetLastError();
}

cudaError_t launch_refine_accept(int K, int H, const float *trial, const float *trial_cost, const float *trial_grad,
                                 float *ctrl, float *cost, float *grad, float *eta, cudaStream_t stream)
{
    refine_accept_kernel<<<blocks(K), kBlock, 0, stream>>>(K, H, (const float2 *)trial, trial_cost,
                                                           (const float2 *)trial_grad, (float2 *)ctrl, cost,
                                                           (float2 *)grad, eta);
    return cudaGetLastError();
}

}  // namespace atp
