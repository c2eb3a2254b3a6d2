// math_check.cu - evaluates the rollout's own elementary functions
// (fastmath.cuh) next to CUDA's library functions on the same inputs, so that
// their error can be bounded on the GPU itself, and the packed two-wide FP32
// operations next to their scalar forms.
#include "atp.h"
#include "fastmath.cuh"

namespace atp {

__global__ void math_check_kernel(const float *__restrict__ a, const float *__restrict__ b, int n,
                                  float *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = a[i], y = b[i];
    float s, c, s_ref, c_ref;
    sincos_r(x, s, c);
    sincosf(x, &s_ref, &c_ref);
    float *o = out + (size_t)14 * i;
    o[0] = s;
    o[1] = c;
    o[2] = s_ref;
    o[3] = c_ref;
    o[4] = atan2_r(x, y);
    o[5] = atan2f(x, y);
    o[6] = rcp(y);
    o[7] = 1.0f / y;
    o[8] = rsq(y);
    o[9] = rsqrtf(y);
    // packed two-wide forms next to their scalar forms
    o[10] = fma2(make_float2(x, y), make_float2(y, x), make_float2(y, x)).x;
    o[11] = fmaf(x, y, y);
    o[12] = sub2(make_float2(x, y), make_float2(y, x)).y;
    o[13] = __fsub_rn(y, x);
}

}  // namespace atp

extern "C" int atp_math_check(const float *a_dev, const float *b_dev, int n, float *out_dev,
                              void *stream)
{
    if (!a_dev || !b_dev || !out_dev || n < 0) return ATP_ERR_INVALID;
    if (n == 0) return ATP_OK;
    atp::math_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a_dev, b_dev, n,
                                                                                          out_dev);
    return cudaGetLastError() == cudaSuccess ? ATP_OK : ATP_ERR_CUDA;
}
