// terrain_tools.cuh - the terrain preprocessing kernels: the model-specific
// Gaussian level of detail of a heightmap (Sec. V-B) and the costmap of the
// distance constraints (Sec. IV-C, IV-D).
#pragma once

#include <cuda_runtime.h>

namespace atp {

// largest Gaussian radius (cells) the level-of-detail kernels take
constexpr int kLodMaxRadius = 512;

struct LodParams {
    const float *in;          // [ny][nx]
    float *out;               // [ny][nx]
    int nx, ny;
    int r;                    // kernel radius in cells, 0..kLodMaxRadius
    float inv2s2;             // 1 / (2 s^2), s = sigma / cell
};

// Two separable passes (rows into tmp, columns into out); tmp must not alias
// in or out.
cudaError_t launch_lod_smooth(const float *in, float *tmp, float *out, int nx, int ny, int r,
                              float inv2s2, cudaStream_t stream);

constexpr int kCostmapMaxPolys = 256;

struct CostmapParams {
    const double *xy;         // vertices [n_vert][2], world metres
    int n_poly, n_vert;
    int start[kCostmapMaxPolys + 1];   // polygon p: vertices start[p] .. start[p+1]-1
    int kind[kCostmapMaxPolys];        // 0 obstacle, 1 path boundary
    int nx, ny;
    double cell, x0, y0;
    float inv_eps, sigma;
    float *cost;              // [ny][nx]
    float *sdist;             // [ny][nx] or nullptr: smallest signed distance
    const float4 *box;        // [n_poly] reach boxes (set by launch_costmap) or nullptr
};

// With box_buf (device, kCostmapMaxPolys float4) and no sdist output, a first
// kernel writes each perimeter's bounding box grown by `reach` metres and the
// costmap kernel skips, per 16 x 16 tile of nodes, every obstacle whose grown
// box misses the tile: beyond `reach` (at least twice eps) its cost rate is
// exactly zero, so the costmap keeps its bits.  Path boundaries are never
// skipped (their cost lies outside them), nor is anything when sdist is
// wanted (the smallest distance needs every perimeter).
cudaError_t launch_costmap(CostmapParams p, float4 *box_buf, float reach, cudaStream_t stream);

}  // namespace atp
