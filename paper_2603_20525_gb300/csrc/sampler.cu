// sampler.cu - on-device candidate sampler.  The paper draws every plan's
// candidate controls on the GPU (Sec. IV-D); here candidate j's control at
// step k is a Gaussian perturbation of a warm-start nominal, from the
// counter-based generator Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// at counter (j, floor(k / 4), nonce, 0) and the Box-Muller transform, so any
// (j, k) is drawn independently of the launch shape.
#include <cuda_runtime.h>
#include <stdint.h>

#include "atp.h"
#include "sampler.cuh"

namespace atp {

// Philox4x64 multipliers and Weyl key increments (Salmon et al. 2011)
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * c[0];
        const uint64_t hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        const uint64_t lo1 = 0xCA5A826395121157ull * c[2];
        const uint64_t hi1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0;
        const uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// One Philox call gives four 64-bit words, eight 23-bit uniforms (bits
// 63..41 and 31..9 of each word), so four Box-Muller pairs: the controls of
// four consecutive steps k = 4 kq .. 4 kq + 3 of candidate j, from counter
// (j, kq, nonce, 0).  Step 4 kq + s pairs the words (w0, w1) for s = 0, 2
// and (w2, w3) for s = 1, 3, the high uniforms for s < 2 and the low ones
// for s >= 2.
__device__ __forceinline__ float unif23(uint64_t w, bool low)
{
    const uint32_t b = low ? (uint32_t)((w >> 9) & 0x7FFFFFull) : (uint32_t)(w >> 41);
    return ((float)b + 0.5f) * (1.0f / 8388608.0f);      // on (0, 1), exact in FP32
}

__global__ void sample_kernel(SampleParams p)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int kq = blockIdx.y;
    if (j >= p.N) return;
    uint64_t c[4] = {(uint64_t)j, (uint64_t)kq, p.nonce, 0ull};
    if (j > 0) philox4x64_10(c, p.key0, p.key1);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int k = 4 * kq + s;
        if (k >= p.H) break;
        float2 nom = make_float2(0.f, 0.f);
        if (p.H_prev > 0) nom = p.prev[min(k + p.shift, p.H_prev - 1)];
        float2 o = nom;
        if (j > 0) {
            const bool low = s >= 2;
            const uint64_t wa = (s & 1) ? c[2] : c[0], wb = (s & 1) ? c[3] : c[1];
            const float u1 = unif23(wa, low), u2 = unif23(wb, low);
            const float r = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            o.x = fmaf(p.sigma_rate, r * cs, nom.x);
            o.y = fmaf(p.sigma_acc, r * sn, nom.y);
        }
        p.ctrl[(size_t)k * p.N + j] = o;
    }
}

cudaError_t launch_sample(const SampleParams &p, cudaStream_t stream)
{
    const dim3 block(256);
    const dim3 grid((unsigned)((p.N + 255) / 256), (unsigned)((p.H + 3) / 4));
    sample_kernel<<<grid, block, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace atp
