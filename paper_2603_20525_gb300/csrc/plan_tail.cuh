// plan_tail.cuh - the fused end of every planning kernel: the empirical
// argmin over the per-candidate results (Sec. IV-D) and the best candidate's
// outputs, shared by the SRB and planar kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "atp.h"
#include "plan_kernel.cuh"

namespace atp {

__device__ __forceinline__ uint32_t order_u32(float f)
{
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float clamp_keep_nan(float v, float lo, float hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

// Empirical argmin of one plan (Sec. IV-D, reading Q7): the lexicographic
// minimum of (infeasible, J, j) over the plan's n_ctas CTAs, then the last of
// them writes the result.
// BLOCK is the launch's threads per CTA.
template <int BLOCK = kPlanBlock>
__device__ __forceinline__ void plan_tail(const PlanParams &p, int j, bool leader, float J,
                                          bool feasible, unsigned n_ctas)
{
    __shared__ unsigned long long s_key[BLOCK / 32];
    __shared__ unsigned int s_cnt[BLOCK / 32];
    __shared__ bool s_last;
    unsigned long long key = ~0ull;
    if (leader)
        key = ((unsigned long long)(feasible ? 0u : 1u) << 63) |
              ((unsigned long long)order_u32(J) << 31) | (unsigned long long)j;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other < key ? other : key;
    }
    const unsigned int nf = __popc(__ballot_sync(0xffffffffu, leader && feasible));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_key[warp] = key;
        s_cnt[warp] = nf;
    }
    __threadfence();          // per-candidate outputs visible before the ticket
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bk = s_key[0];
        unsigned int bc = s_cnt[0];
        for (int w = 1; w < BLOCK / 32; ++w) {
            bk = s_key[w] < bk ? s_key[w] : bk;
            bc += s_cnt[w];
        }
        atomicMin(&p.scratch->key, bk);
        atomicAdd(&p.scratch->count, bc);
        __threadfence();
        const unsigned int t = atomicAdd(&p.scratch->ticket, 1u);
        s_last = (t == n_ctas - 1);
    }
    __syncthreads();
    if (!s_last) return;

    // ---- last CTA: result, best controls (and per-step margins), reset scratch
    __shared__ unsigned long long s_best;
    __shared__ unsigned int s_nf;
    if (threadIdx.x == 0) {
        s_best = atomicAdd(&p.scratch->key, 0ull);
        s_nf = atomicAdd(&p.scratch->count, 0u);
    }
    __syncthreads();
    const uint32_t best = (uint32_t)(s_best & 0x7fffffffull);
    const size_t N = (size_t)p.N;
    for (int k = threadIdx.x; k < p.H; k += blockDim.x) {
        if (p.best_ctrl) {
            const float2 u = __ldcg(p.ctrl + (size_t)k * N + best);
            p.best_ctrl[2 * k] = clamp_keep_nan(u.x, -p.V.ddmax, p.V.ddmax);
            p.best_ctrl[2 * k + 1] = u.y;
        }
        if (p.best_margin && p.step_margin) p.best_margin[k] = __ldcg(p.step_margin + (size_t)k * N + best);
    }
    if (threadIdx.x == 0) {
        atp_plan_out o;
        o.best_idx = best;
        o.n_feasible = s_nf;
        o.best_cost = __ldcg(p.cost + best);
        o.best_min_margin = __ldcg(p.margin + best);
        o.best_min_step = p.min_step ? __ldcg(p.min_step + best) : 0;
        o.reserved = 0;
        *p.out = o;
        // restore the scratch for the next plan on this stream
        p.scratch->key = ~0ull;
        p.scratch->count = 0u;
        p.scratch->ticket = 0u;
    }
}

}  // namespace atp
