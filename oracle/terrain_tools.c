/*
 * terrain_tools.c - FP64 oracle of the two terrain preprocessing steps of
 * arxiv 2603.20525:
 *   - the model-specific level of detail (Sec. V-B): a Gaussian smoothing of
 *     the heightmap whose standard deviation is set by the model's length
 *     scale (0.3 m for the SRB model, 1.5 m for the planar model);
 *   - the costmap of the distance constraints (Sec. IV-C, IV-D): the signed
 *     distance to every obstacle and path-boundary perimeter, turned into the
 *     normalised quadratic soft-constraint cost rate and summed over the
 *     perimeters, precomputed per heightmap node.
 *
 * TEST INFRASTRUCTURE: only the test suite may call this.  Plain loops, in
 * the order the definitions are stated; no blocking, no separable shortcut.
 */
#include <math.h>
#include <stddef.h>

#include "oracle.h"

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Gaussian weights w_k proportional to exp(-(k cell)^2 / (2 sigma^2)) for
 * |k| <= r, r = floor(4 sigma / cell + 1/2) (the kernel is cut at four
 * standard deviations), normalised to sum 1.  Returns r; sigma <= 0 gives the
 * identity (r = 0, w_0 = 1). */
int orc_lod_weights(double cell, double sigma, int r_max, double *w)
{
    if (!(sigma > 0.0)) {
        w[0] = 1.0;
        return 0;
    }
    const double s = sigma / cell;                 /* standard deviation in cells */
    int r = (int)(4.0 * s + 0.5);
    if (r > r_max) return -1;
    double z = 0.0;
    for (int k = -r; k <= r; ++k) {
        w[k + r] = exp(-0.5 * (double)k * (double)k / (s * s));
        z += w[k + r];
    }
    for (int k = 0; k <= 2 * r; ++k) w[k] /= z;
    return r;
}

/* out[j][i] = sum over |a|, |b| <= r of w_a w_b f[clamp(j + b)][clamp(i + a)]:
 * the two-dimensional Gaussian (a product of the one-dimensional weights),
 * with the map extended by its nearest border node.  Returns 0, or -1 if the
 * kernel radius exceeds 4096 cells. */
int orc_lod_smooth(const float *f, int nx, int ny, double cell, double sigma, double *out)
{
    static const int R_MAX = 4096;
    double w[2 * 4096 + 1];
    const int r = orc_lod_weights(cell, sigma, R_MAX, w);
    if (r < 0) return -1;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double acc = 0.0;
            for (int b = -r; b <= r; ++b) {
                const int jj = clampi(j + b, 0, ny - 1);
                for (int a = -r; a <= r; ++a) {
                    const int ii = clampi(i + a, 0, nx - 1);
                    acc += w[a + r] * w[b + r] * (double)f[(size_t)jj * nx + ii];
                }
            }
            out[(size_t)j * nx + i] = acc;
        }
    }
    return 0;
}

/* Euclidean distance from (px, py) to the segment from a to b. */
static double seg_dist(double px, double py, double ax, double ay, double bx, double by)
{
    const double ex = bx - ax, ey = by - ay;
    const double l2 = ex * ex + ey * ey;
    double t = 0.0;
    if (l2 > 0.0) {
        t = ((px - ax) * ex + (py - ay) * ey) / l2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    const double dx = px - (ax + t * ex), dy = py - (ay + t * ey);
    return sqrt(dx * dx + dy * dy);
}

/* Signed distance of (px, py) to the closed perimeter with vertices
 * xy[2k], xy[2k+1], k < n: the minimum distance to its edges, negative
 * inside an obstacle (kind 0) and outside a path boundary (kind 1); inside
 * is the even-odd rule of a ray cast towards +x. */
double orc_sdist(const double *xy, int n, int kind, double px, double py)
{
    double d = INFINITY;
    int inside = 0;
    for (int k = 0; k < n; ++k) {
        const int m = (k + 1) % n;
        const double ax = xy[2 * k], ay = xy[2 * k + 1];
        const double bx = xy[2 * m], by = xy[2 * m + 1];
        const double dk = seg_dist(px, py, ax, ay, bx, by);
        if (dk < d) d = dk;
        if ((ay > py) != (by > py)) {
            const double xc = ax + (py - ay) * (bx - ax) / (by - ay);
            if (px < xc) inside = !inside;
        }
    }
    const int negative = kind == 0 ? inside : !inside;
    return negative ? -d : d;
}

/* Costmap of the distance constraints at every node (x0 + i cell,
 * y0 + j cell): c = sum over perimeters p of sigma max(0, 1 - sdist_p / eps)^2,
 * the soft-constraint cost rate with violation measure -sdist (Sec. IV-C).
 * Perimeter p has vertices start[p] .. start[p+1]-1 of xy and kind kind[p].
 * sdist_min (optional) receives the smallest signed distance over p. */
void orc_costmap(const double *xy, const int *start, const int *kind, int n_poly, int nx, int ny,
                 double cell, double x0, double y0, double eps, double sigma, double *cost,
                 double *sdist_min)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const double px = x0 + i * cell, py = y0 + j * cell;
            double c = 0.0, smin = INFINITY;
            for (int p = 0; p < n_poly; ++p) {
                const double s = orc_sdist(xy + 2 * start[p], start[p + 1] - start[p], kind[p], px, py);
                const double v = 1.0 - s / eps;
                if (v > 0.0) c += sigma * v * v;
                if (s < smin) smin = s;
            }
            cost[(size_t)j * nx + i] = c;
            if (sdist_min) sdist_min[(size_t)j * nx + i] = smin;
        }
    }
}
