// terrain_tools.cu - terrain preprocessing for the planner (arxiv 2603.20525):
//
//   * Level of detail (Sec. V-B).  Each model gets its own Gaussian-smoothed
//     copy of the heightmap (0.3 m standard deviation for the SRB model, the
//     length scale of a wheel; 1.5 m for the planar model, that of the
//     chassis).  The two-dimensional Gaussian is a product of one-dimensional
//     ones, so it runs as a row pass and a column pass, each through a
//     shared-memory tile with its halo; the map is extended by its nearest
//     border node and the kernel is cut at four standard deviations.
//   * Costmap of the distance constraints (Sec. IV-C, IV-D).  At every node
//     the signed distance to each obstacle or path-boundary perimeter is turned
//     into the normalised quadratic soft-constraint cost rate and summed over
//     the perimeters, so that the rollout only interpolates it.  One thread per
//     node; each 16 x 16 tile streams the edges of the perimeters that can
//     reach it through shared memory in chunks.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "terrain_tools.cuh"

namespace atp {

namespace {

constexpr int kRowThreads = 256;  // row-pass CTA
// Outputs per thread: 4 row and 8 column outputs below this radius, 8 and 16
// from it on.  Small radii are bound by each CTA's set-up, and more outputs
// per thread only halve the CTAs; large radii by the taps, where the wider
// windows load fewer values per output (measured on the GB300: the narrow
// form 4 % faster at 12 cells, the wide one 5 % at 24 and 10 to 16 % at 36
// to 200 cells; the same bits).
constexpr int kLodWideMinR = 16;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Normalised weights w[k], k = 0..2r, of exp(-(k - r)^2 / (2 s^2)), made by
// every CTA the same way: the terms, then their sum in a fixed order (per
// thread a strided run, then a fixed shuffle tree and a fixed pass over the
// warps), so every CTA holds the same bits.  Needs blockDim.x * blockDim.y a
// multiple of 32 and at most 1024 threads.
__device__ void gauss_weights_cta(float *w, int r, float inv2s2)
{
    __shared__ float s_part[32];
    __shared__ float s_total;
    const int n = 2 * r + 1;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    float part = 0.f;
    for (int k = t; k < n; k += nt) {
        const float d = (float)(k - r);
        const float e = expf(-(d * d) * inv2s2);
        w[k] = e;
        part += e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((t & 31) == 0) s_part[t >> 5] = part;
    __syncthreads();
    if (t == 0) {
        float z = 0.f;
        for (int i = 0; i < nt / 32; ++i) z += s_part[i];
        s_total = z;
    }
    __syncthreads();
    const float z = s_total;
    for (int k = t; k < n; k += nt) w[k] = w[k] / z;
    __syncthreads();
}

// The same weights for 2r + 1 <= 32, made by the CTA's first warp alone: one
// term per lane and the lanes' sum through the same shuffle tree, every lane
// dividing by lane 0's total.  The CTA-wide form adds only the other warps'
// zero sums to that total, so the bits are the same.  The other warps go
// straight on to their tile loads, and the caller's next barrier publishes
// the weights: at a radius of 12 cells this took 6 % off the two passes,
// where the set-up's barriers bound them.
__device__ __forceinline__ void gauss_weights_warp(float *w, int r, float inv2s2)
{
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if (t >= 32) return;
    const int n = 2 * r + 1;
    float e = 0.f;
    if (t < n) {
        const float d = (float)(t - r);
        e = expf(-(d * d) * inv2s2);
    }
    float z = e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    z = __shfl_sync(0xffffffffu, z, 0);
    if (t < n) w[t] = e / z;
}

// The weights of a pass: the first warp alone for the narrow windows (r below
// kLodWideMinR, so 2r + 1 <= 31), the whole CTA otherwise.
static_assert(2 * (kLodWideMinR - 1) + 1 <= 32, "the narrow windows' weights fit one warp");
template <bool NARROW>
__device__ __forceinline__ void gauss_weights(float *w, int r, float inv2s2)
{
    if (NARROW)
        gauss_weights_warp(w, r, inv2s2);
    else
        gauss_weights_cta(w, r, inv2s2);
}

// out[j][i] = sum_k w[k] in[j][clamp(i + k - r)], each sum over k in order.
// Thread t makes outputs OUT t .. OUT t + OUT - 1 of the CTA's 256 OUT from a
// window of OUT + 4 tile values refilled by one 16-byte shared load per four
// taps.
template <int OUT>
__global__ void __launch_bounds__(kRowThreads) lod_rows_kernel(LodParams p)
{
    static_assert(OUT % 4 == 0, "whole float4 windows");
    constexpr int kRowOut = OUT, kRowVec = OUT / 4, kRowTile = kRowThreads * OUT;
    extern __shared__ __align__(16) float sm[];         // the tile is read as float4
    float *w = sm;                                      // 2r + 1, padded to 4
    float *tile = sm + ((2 * p.r + 1 + 3) & ~3);        // kRowTile + 2r + 8
    gauss_weights<OUT == 4>(w, p.r, p.inv2s2);
    const int j = blockIdx.y;
    const int i0 = blockIdx.x * kRowTile;
    const float *row = p.in + (size_t)j * p.nx;
    const int n_tile = kRowTile + 2 * p.r + 8;
    for (int t = threadIdx.x; t < n_tile; t += kRowThreads)
        tile[t] = __ldg(row + clampi(i0 - p.r + t, 0, p.nx - 1));
    __syncthreads();
    const int ib = i0 + kRowOut * threadIdx.x;
    if (ib >= p.nx) return;
    const float4 *t4 = reinterpret_cast<const float4 *>(tile) + kRowVec * threadIdx.x;
    float acc[kRowOut];
    float4 win[kRowVec + 1];
#pragma unroll
    for (int q = 0; q < kRowOut; ++q) acc[q] = 0.f;
#pragma unroll
    for (int c = 0; c < kRowVec; ++c) win[c] = t4[c];
    const int n = 2 * p.r + 1;
    for (int k0 = 0; k0 < n; k0 += 4) {
        win[kRowVec] = t4[(k0 >> 2) + kRowVec];
        float v[kRowOut + 4];
#pragma unroll
        for (int c = 0; c <= kRowVec; ++c) {
            v[4 * c] = win[c].x;
            v[4 * c + 1] = win[c].y;
            v[4 * c + 2] = win[c].z;
            v[4 * c + 3] = win[c].w;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (k0 + e < n) {
                const float wk = w[k0 + e];
#pragma unroll
                for (int q = 0; q < kRowOut; ++q) acc[q] = fmaf(wk, v[e + q], acc[q]);
            }
        }
#pragma unroll
        for (int c = 0; c < kRowVec; ++c) win[c] = win[c + 1];
    }
    float *o = p.out + (size_t)j * p.nx + ib;
#pragma unroll
    for (int q = 0; q < kRowOut; ++q)
        if (ib + q < p.nx) o[q] = acc[q];
}

// out[j][i] = sum_k w[k] in[clamp(j + k - r)][i], each sum over k in order; a
// CTA of 32 x 8 threads covers 32 columns and 8 OUT rows, thread (x, y) rows
// OUT y .. OUT y + OUT - 1 of column x from a window of 2 OUT tile rows
// refilled with OUT loads per OUT taps.
template <int OUT>
__global__ void __launch_bounds__(256) lod_cols_kernel(LodParams p)
{
    constexpr int kColOut = OUT, kColTile = 8 * OUT;
    extern __shared__ float sm[];
    float *w = sm;                           // 2r + 1, padded to a multiple of 32
    float *tile = sm + ((2 * p.r + 1 + 31) & ~31);   // [kColTile + 2r + 8][32]
    gauss_weights<OUT == 8>(w, p.r, p.inv2s2);
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j0 = blockIdx.y * kColTile;
    const int ic = min(i, p.nx - 1);
    const int n_rows = kColTile + 2 * p.r + kColOut;
    for (int t = threadIdx.y; t < n_rows; t += 8)
        tile[t * 32 + threadIdx.x] = __ldg(p.in + (size_t)clampi(j0 - p.r + t, 0, p.ny - 1) * p.nx + ic);
    __syncthreads();
    const int jb = kColOut * threadIdx.y;    // first of this thread's rows in the tile
    if (i >= p.nx || j0 + jb >= p.ny) return;
    const float *col = tile + jb * 32 + threadIdx.x;
    float acc[kColOut];
    float v[2 * kColOut];
#pragma unroll
    for (int q = 0; q < kColOut; ++q) {
        acc[q] = 0.f;
        v[q] = col[q * 32];
    }
    const int n = 2 * p.r + 1;
    for (int k0 = 0; k0 < n; k0 += kColOut) {
#pragma unroll
        for (int q = 0; q < kColOut; ++q) v[kColOut + q] = col[(k0 + kColOut + q) * 32];
#pragma unroll
        for (int e = 0; e < kColOut; ++e) {
            if (k0 + e < n) {
                const float wk = w[k0 + e];
#pragma unroll
                for (int q = 0; q < kColOut; ++q) acc[q] = fmaf(wk, v[e + q], acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kColOut; ++q) v[q] = v[kColOut + q];
    }
#pragma unroll
    for (int q = 0; q < kColOut; ++q) {
        const int j = j0 + jb + q;
        if (j < p.ny) p.out[(size_t)j * p.nx + i] = acc[q];
    }
}

size_t rows_smem(int r, int out)
{
    return sizeof(float) * (size_t)(((2 * r + 1 + 3) & ~3) + kRowThreads * out + 2 * r + 8);
}
size_t cols_smem(int r, int out)
{
    return sizeof(float) * (size_t)(((2 * r + 1 + 31) & ~31) + (8 * out + 2 * r + out) * 32);
}

template <int ROW_OUT, int COL_OUT>
cudaError_t lod_passes(LodParams p, float *tmp, float *out, cudaStream_t stream)
{
    const int r = p.r;
    cudaError_t e = cudaFuncSetAttribute(lod_rows_kernel<ROW_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rows_smem(kLodMaxRadius, ROW_OUT));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lod_cols_kernel<COL_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cols_smem(kLodMaxRadius, COL_OUT));
    if (e != cudaSuccess) return e;
    p.out = tmp;
    const int row_tile = kRowThreads * ROW_OUT;
    lod_rows_kernel<ROW_OUT><<<dim3((unsigned)((p.nx + row_tile - 1) / row_tile), (unsigned)p.ny), kRowThreads,
                               rows_smem(r, ROW_OUT), stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    p.in = tmp;
    p.out = out;
    const int col_tile = 8 * COL_OUT;
    lod_cols_kernel<COL_OUT><<<dim3((unsigned)((p.nx + 31) / 32), (unsigned)((p.ny + col_tile - 1) / col_tile)),
                               dim3(32, 8), cols_smem(r, COL_OUT), stream>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lod_smooth(const float *in, float *tmp, float *out, int nx, int ny, int r,
                              float inv2s2, cudaStream_t stream)
{
    if (r < 0 || r > kLodMaxRadius) return cudaErrorInvalidValue;
    LodParams p;
    p.nx = nx;
    p.ny = ny;
    p.r = r;
    p.inv2s2 = inv2s2;
    p.in = in;
    return r < kLodWideMinR ? lod_passes<4, 8>(p, tmp, out, stream) : lod_passes<8, 16>(p, tmp, out, stream);
}

// ---------------------------------------------------------------------------
// Costmap.  Coordinates are taken relative to the terrain origin (in FP64 once
// per vertex and node, then FP32), so that the FP32 distance arithmetic works
// on metres from the map corner rather than on large world coordinates.

namespace {

constexpr int kChunk = 256;       // vertices staged per pass, one per thread
// the tile's perimeter scan takes one thread of the 16 x 16 CTA per perimeter
static_assert(kCostmapMaxPolys <= 256, "one costmap thread per perimeter");

// Bounding box of perimeter blockIdx.x in the costmap kernel's coordinates,
// grown by `reach`; one warp per perimeter.
__global__ void __launch_bounds__(32) costmap_boxes_kernel(const __grid_constant__ CostmapParams p,
                                                           float4 *box, float reach)
{
    const int q = blockIdx.x;
    float x0 = CUDART_INF_F, y0 = CUDART_INF_F, x1 = -CUDART_INF_F, y1 = -CUDART_INF_F;
    for (int v = p.start[q] + (int)threadIdx.x; v < p.start[q + 1]; v += 32) {
        const float x = (float)(p.xy[2 * v] - p.x0), y = (float)(p.xy[2 * v + 1] - p.y0);
        x0 = fminf(x0, x);
        y0 = fminf(y0, y);
        x1 = fmaxf(x1, x);
        y1 = fmaxf(y1, y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if (threadIdx.x == 0) box[q] = make_float4(x0 - reach, y0 - reach, x1 + reach, y1 + reach);
}

__global__ void __launch_bounds__(256) costmap_kernel(const __grid_constant__ CostmapParams p)
{
    __shared__ float2 s_a[kChunk], s_b[kChunk];
    __shared__ int s_poly[kChunk];
    __shared__ int s_id[kCostmapMaxPolys];        // the tile's perimeters, in order
    __shared__ int s_off[kCostmapMaxPolys + 1];   // prefix of their vertex counts
    __shared__ int s_wn[8], s_wv[8];
    const int i = blockIdx.x * 16 + threadIdx.x;
    const int j = blockIdx.y * 16 + threadIdx.y;
    const int t = threadIdx.y * 16 + threadIdx.x;
    const bool live = i < p.nx && j < p.ny;
    const float px = (float)((double)i * p.cell), py = (float)((double)j * p.cell);
    // the perimeters that can reach this tile (all of them without boxes),
    // kept in their order by a block-wide scan over one thread per perimeter
    bool keep = false;
    int nv = 0;
    if (t < p.n_poly) {
        keep = true;
        if (p.box && p.kind[t] == 0) {
            const float tx0 = (float)((double)(blockIdx.x * 16) * p.cell);
            const float tx1 = (float)((double)(blockIdx.x * 16 + 15) * p.cell);
            const float ty0 = (float)((double)(blockIdx.y * 16) * p.cell);
            const float ty1 = (float)((double)(blockIdx.y * 16 + 15) * p.cell);
            const float4 b = p.box[t];
            keep = !(b.z < tx0 || b.x > tx1 || b.w < ty0 || b.y > ty1);
        }
        nv = keep ? p.start[t + 1] - p.start[t] : 0;
    }
    const int lane = t & 31, wid = t >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    int inc = nv;                                  // inclusive scan of vertex counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) {
        s_wn[wid] = __popc(bal);
        s_wv[wid] = inc;
    }
    __syncthreads();
    int bn = 0, bv = 0, n_keep = 0, n_vert = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        if (w < wid) {
            bn += s_wn[w];
            bv += s_wv[w];
        }
        n_keep += s_wn[w];
        n_vert += s_wv[w];
    }
    if (keep) {
        const int k = bn + __popc(bal & ((1u << lane) - 1u));
        s_id[k] = t;
        s_off[k] = bv + inc - nv;
    }
    if (t == 0) s_off[n_keep] = n_vert;
    float c = 0.f, smin = CUDART_INF_F;
    int cur = -1;
    float d2 = CUDART_INF_F;
    bool inside = false;
    // the signed distance of the polygon just finished and its cost
    auto finish = [&](int q) {
        const float d = sqrtf(d2);
        const bool neg = p.kind[q] == 0 ? inside : !inside;
        const float s = neg ? -d : d;
        const float v = 1.f - s * p.inv_eps;
        if (v > 0.f) c = fmaf(p.sigma * v, v, c);
        smin = fminf(smin, s);
    };
    for (int c0 = 0; c0 < n_vert; c0 += kChunk) {
        __syncthreads();
        const int vc = c0 + t;
        if (vc < n_vert) {
            int lo = 0, hi = n_keep;               // s_off[lo] <= vc < s_off[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] <= vc) lo = mid;
                else hi = mid;
            }
            const int q = s_id[lo];
            const int v = p.start[q] + (vc - s_off[lo]);
            const int nxt = v + 1 < p.start[q + 1] ? v + 1 : p.start[q];
            s_a[t] = make_float2((float)(p.xy[2 * v] - p.x0), (float)(p.xy[2 * v + 1] - p.y0));
            s_b[t] = make_float2((float)(p.xy[2 * nxt] - p.x0), (float)(p.xy[2 * nxt + 1] - p.y0));
            s_poly[t] = q;
        }
        __syncthreads();
        const int m = min(kChunk, n_vert - c0);
        for (int e = 0; e < m; ++e) {
            const int q = s_poly[e];
            if (q != cur) {
                if (cur >= 0) finish(cur);
                cur = q;
                d2 = CUDART_INF_F;
                inside = false;
            }
            const float2 a = s_a[e], b = s_b[e];
            // distance to the segment a-b
            const float ex = b.x - a.x, ey = b.y - a.y;
            const float rx = px - a.x, ry = py - a.y;
            const float l2 = fmaf(ex, ex, ey * ey);
            float u = l2 > 0.f ? fmaf(rx, ex, ry * ey) / l2 : 0.f;
            u = fminf(fmaxf(u, 0.f), 1.f);
            const float dx = px - fmaf(u, ex, a.x), dy = py - fmaf(u, ey, a.y);
            d2 = fminf(d2, fmaf(dx, dx, dy * dy));
            // even-odd rule, ray towards +x
            if ((a.y > py) != (b.y > py)) {
                const float xc = fmaf((py - a.y) / (b.y - a.y), ex, a.x);
                if (px < xc) inside = !inside;
            }
        }
    }
    if (cur >= 0) finish(cur);
    if (!live) return;
    const size_t o = (size_t)j * p.nx + i;
    p.cost[o] = c;
    if (p.sdist) p.sdist[o] = smin;
}

}  // namespace

cudaError_t launch_costmap(CostmapParams p, float4 *box_buf, float reach, cudaStream_t stream)
{
    if (p.n_poly < 1 || p.n_poly > kCostmapMaxPolys) return cudaErrorInvalidValue;
    p.box = nullptr;
    if (box_buf && !p.sdist) {
        costmap_boxes_kernel<<<(unsigned)p.n_poly, 32, 0, stream>>>(p, box_buf, reach);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        p.box = box_buf;
    }
    const dim3 grid((unsigned)((p.nx + 15) / 16), (unsigned)((p.ny + 15) / 16));
    costmap_kernel<<<grid, dim3(16, 16), 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace atp
