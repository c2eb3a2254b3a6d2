// emul32.cpp - two more instantiations of the templated model (model.hpp).
//
// TEST INFRASTRUCTURE.  Only the test suite calls these; they share no code
// with the CUDA path.
//
// 1. The FP32 arithmetic reference.  Every model quantity is an FP32 value
//    and every operation rounds to FP32 (separate roundings, no fused
//    multiply-add; the C library's sinf, cosf, atan2f, asinf and sqrtf).  The
//    state is kept the way a compensated FP32 implementation keeps it:
//    position, heading and linear velocity accumulate exactly (FP64 storage)
//    and the terrain is read at the exactly accumulated position, while the
//    other components are rounded to FP32 after every Euler step.  Node
//    slopes are stored in FP32.  Its difference from the FP64 oracle is the
//    error that FP32 arithmetic itself leaves on a rollout; the CUDA path is
//    compared against it.
//
// 2. The operation count.  A scalar that counts each addition, subtraction,
//    multiplication and division, and each elementary function, run over
//    the FP64 model: the algorithmic work per Euler step.
#include <cmath>
#include <vector>

#include "model.hpp"

namespace orcm {

// ---- FP32 arithmetic with FP64 storage ------------------------------------------
struct P64;

struct F32 {
    float v;
    F32() : v(0.f) {}
    F32(double x) : v((float)x) {}
    explicit F32(const P64 &p);
};

// a stored state component (FP64)
struct P64 {
    double v;
    P64() : v(0.0) {}
    P64(double x) : v(x) {}
    P64(const F32 &f) : v((double)f.v) {}
};

inline F32::F32(const P64 &p) : v((float)p.v) {}

inline F32 mkf(float x)
{
    F32 r;
    r.v = x;
    return r;
}
inline F32 operator+(const F32 &a, const F32 &b) { return mkf(a.v + b.v); }
inline F32 operator-(const F32 &a, const F32 &b) { return mkf(a.v - b.v); }
inline F32 operator*(const F32 &a, const F32 &b) { return mkf(a.v * b.v); }
inline F32 operator/(const F32 &a, const F32 &b) { return mkf(a.v / b.v); }
inline F32 operator-(const F32 &a) { return mkf(-a.v); }
inline F32 &operator+=(F32 &a, const F32 &b) { a.v = a.v + b.v; return a; }
inline double value(const F32 &a) { return (double)a.v; }
inline F32 sin(const F32 &a) { return mkf(sinf(a.v)); }
inline F32 cos(const F32 &a) { return mkf(cosf(a.v)); }
inline F32 sqrt(const F32 &a) { return mkf(sqrtf(a.v)); }
inline F32 fabs(const F32 &a) { return mkf(fabsf(a.v)); }
inline F32 asin(const F32 &a) { return mkf(asinf(a.v)); }
inline F32 atan2(const F32 &y, const F32 &x) { return mkf(atan2f(y.v, x.v)); }

inline P64 operator+(const P64 &a, const P64 &b) { return P64(a.v + b.v); }
inline P64 operator-(const P64 &a, const P64 &b) { return P64(a.v - b.v); }
inline P64 operator/(const P64 &a, const P64 &b) { return P64(a.v / b.v); }
inline double value(const P64 &a) { return a.v; }
// sin and cos at the stored argument, correctly rounded to FP32 by the caller
inline P64 sin(const P64 &a) { return P64(std::sin(a.v)); }
inline P64 cos(const P64 &a) { return P64(std::cos(a.v)); }

// ---- operation counting ---------------------------------------------------------
struct Counts {
    long add, mul, div, sqrt_, sin_, cos_, atan2_, asin_;
};
thread_local Counts g_cnt;

struct Cnt {
    double v;
    Cnt() : v(0.0) {}
    Cnt(double x) : v(x) {}
};
inline Cnt operator+(const Cnt &a, const Cnt &b) { ++g_cnt.add; return Cnt(a.v + b.v); }
inline Cnt operator-(const Cnt &a, const Cnt &b) { ++g_cnt.add; return Cnt(a.v - b.v); }
inline Cnt operator*(const Cnt &a, const Cnt &b) { ++g_cnt.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(const Cnt &a, const Cnt &b) { ++g_cnt.div; return Cnt(a.v / b.v); }
inline Cnt operator-(const Cnt &a) { return Cnt(-a.v); }
inline Cnt &operator+=(Cnt &a, const Cnt &b) { ++g_cnt.add; a.v += b.v; return a; }
inline double value(const Cnt &a) { return a.v; }
inline Cnt sin(const Cnt &a) { ++g_cnt.sin_; return Cnt(std::sin(a.v)); }
inline Cnt cos(const Cnt &a) { ++g_cnt.cos_; return Cnt(std::cos(a.v)); }
inline Cnt sqrt(const Cnt &a) { ++g_cnt.sqrt_; return Cnt(std::sqrt(a.v)); }
inline Cnt fabs(const Cnt &a) { return Cnt(std::fabs(a.v)); }
inline Cnt asin(const Cnt &a) { ++g_cnt.asin_; return Cnt(std::asin(a.v)); }
inline Cnt atan2(const Cnt &y, const Cnt &x) { ++g_cnt.atan2_; return Cnt(std::atan2(y.v, x.v)); }

// node slopes of the FP32 reference: the terrain's node slopes (central
// differences of the heights, reading Q10, or the slopes of a stored format)
// rounded to FP32
void slopes32(const orc_terrain *t, std::vector<double> &gx, std::vector<double> &gy)
{
    const size_t n = (size_t)t->nx * t->ny;
    gx.resize(n);
    gy.resize(n);
    for (size_t i = 0; i < n; ++i) {
        gx[i] = (double)(float)t->gx[i];
        gy[i] = (double)(float)t->gy[i];
    }
}

template <class T>
void controls(const float *ctrl, int N, int j, int H, std::vector<T> &u)
{
    u.resize(2 * (size_t)H);
    for (int k = 0; k < H; ++k) {
        u[2 * k] = T((double)ctrl[((size_t)k * N + j) * 2]);
        u[2 * k + 1] = T((double)ctrl[((size_t)k * N + j) * 2 + 1]);
    }
}

template <class R>
void store(const R &r, int j, int nstate, double *J, double *margin, unsigned char *flags, double *xf,
           int *min_step)
{
    J[j] = value(r.J);
    margin[j] = value(r.margin);
    flags[j] = r.flags;
    if (xf)
        for (int q = 0; q < nstate; ++q) xf[(size_t)j * nstate + q] = r.xf[q];
    if (min_step) min_step[j] = r.min_step;
}

}  // namespace orcm

using namespace orcm;

extern "C" {

// The FP32 arithmetic reference of N SRB (model = 0) or EST (model = 1)
// candidates: ctrl [H][N][2], x0 [N][n] or a shared [n] (n = 13 or 7).
int orc_rollout_f32(int model, const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                    const float *x0, int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub,
                    double *J, double *margin, unsigned char *flags, double *xf, int *min_step)
{
    if (N <= 0 || H <= 0 || n_sub <= 0 || !(dt > 0.0) || (model != 0 && model != 1)) return -1;
    std::vector<double> gx, gy;
    slopes32(t, gx, gy);
    orc_terrain t32 = *t;
    t32.gx = gx.data();
    t32.gy = gy.data();
    const int n = model == 0 ? 13 : 7;
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = 0; j < N; ++j) {
        double xs[13];
        const float *src = x0 + (x0_per_cand ? (size_t)j * n : 0);
        for (int q = 0; q < n; ++q) xs[q] = src[q];
        std::vector<F32> u;
        controls(ctrl, N, j, H, u);
        if (model == 0)
            store(rolloutT<F32, P64>(v, c, &t32, xs, u.data(), H, dt, n_sub), j, 13, J, margin, flags, xf,
                  min_step);
        else
            store(est_rolloutT<F32, P64>(v, c, &t32, xs, u.data(), H, dt, n_sub), j, 7, J, margin, flags, xf,
                  min_step);
    }
    return 0;
}

// The templated model in plain FP64 (T = S = double): the same results as
// srb.c (model = 0) or est.c (model = 1), which checks the restatement.
int orc_rollout_templated(int model, const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                          const float *x0, int x0_per_cand, const float *ctrl, int N, int H, double dt,
                          int n_sub, double *J, double *margin, unsigned char *flags, double *xf,
                          int *min_step)
{
    if (N <= 0 || H <= 0 || n_sub <= 0 || !(dt > 0.0) || (model != 0 && model != 1)) return -1;
    const int n = model == 0 ? 13 : 7;
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = 0; j < N; ++j) {
        double xs[13];
        const float *src = x0 + (x0_per_cand ? (size_t)j * n : 0);
        for (int q = 0; q < n; ++q) xs[q] = src[q];
        std::vector<double> u;
        controls(ctrl, N, j, H, u);
        if (model == 0)
            store(rolloutT<double, double>(v, c, t, xs, u.data(), H, dt, n_sub), j, 13, J, margin, flags, xf,
                  min_step);
        else
            store(est_rolloutT<double, double>(v, c, t, xs, u.data(), H, dt, n_sub), j, 7, J, margin, flags,
                  xf, min_step);
    }
    return 0;
}

// Operations of the SRB (model = 0) or EST (model = 1) rollout over N
// candidates, summed: out = {Euler steps, additions and subtractions,
// multiplications, divisions, sqrt, sin, cos, atan2, asin}.
int orc_count_ops(int model, const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const float *x0,
                  int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub, long out[9])
{
    if (N <= 0 || H <= 0 || n_sub <= 0 || !(dt > 0.0) || (model != 0 && model != 1)) return -1;
    const int n = model == 0 ? 13 : 7;
    long steps = 0;
    g_cnt = Counts{0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < N; ++j) {
        double xs[13];
        const float *src = x0 + (x0_per_cand ? (size_t)j * n : 0);
        for (int q = 0; q < n; ++q) xs[q] = src[q];
        std::vector<Cnt> u;
        controls(ctrl, N, j, H, u);
        if (model == 0) rolloutT<Cnt, Cnt>(v, c, t, xs, u.data(), H, dt, n_sub, &steps);
        else est_rolloutT<Cnt, Cnt>(v, c, t, xs, u.data(), H, dt, n_sub, &steps);
    }
    const long r[9] = {steps, g_cnt.add, g_cnt.mul, g_cnt.div, g_cnt.sqrt_, g_cnt.sin_, g_cnt.cos_,
                       g_cnt.atan2_, g_cnt.asin_};
    for (int q = 0; q < 9; ++q) out[q] = r[q];
    return 0;
}

}  // extern "C"
