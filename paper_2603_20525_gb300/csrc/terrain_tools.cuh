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
};

cudaError_t launch_costmap(const CostmapParams &p, cudaStream_t stream);

}  // namespace atp
