// adjoint.cpp - FP64 CPU adjoint of the discrete SRB rollout cost (arxiv
// 2603.20525, Sec. IV-A..IV-C): the gradient of J = sum h L + Phi with respect
// to the raw control sequence, by generic reverse-mode automatic
// differentiation on a tape (every elementary operation records its local
// partial derivatives; one backward sweep accumulates the adjoints).  Nothing
// here is derived by hand, so it checks the CUDA path's hand-written adjoint
// independently.
//
// TEST INFRASTRUCTURE.  Only the test suite may load it; it shares no code
// with the CUDA path.  The model is restated once more, templated on the
// scalar type, in the paper's order and with the readings of oracle.h; for
// T = double it reproduces srb.c's rollout (checked by the tests).
#include <cmath>
#include <cstring>
#include <vector>

extern "C" {
#include "oracle.h"
}

namespace {

// ---- tape -----------------------------------------------------------------
struct Tape {
    std::vector<double> val;
    std::vector<int> pa, pb;        // parents (-1: none)
    std::vector<double> da, db;     // local partials
    int node(double v, int a = -1, double dav = 0.0, int b = -1, double dbv = 0.0)
    {
        val.push_back(v);
        pa.push_back(a);
        pb.push_back(b);
        da.push_back(dav);
        db.push_back(dbv);
        return (int)val.size() - 1;
    }
};

thread_local Tape *g_tape = nullptr;

struct AD {
    double v;
    int i;    // tape index, -1 for a constant
    AD() : v(0.0), i(-1) {}
    AD(double x) : v(x), i(-1) {}
    AD(double x, int idx) : v(x), i(idx) {}
};

inline AD mk(double v, const AD &a, double da)
{
    if (a.i < 0) return AD(v);
    return AD(v, g_tape->node(v, a.i, da));
}
inline AD mk2(double v, const AD &a, double da, const AD &b, double db)
{
    if (a.i < 0 && b.i < 0) return AD(v);
    if (a.i < 0) return AD(v, g_tape->node(v, b.i, db));
    if (b.i < 0) return AD(v, g_tape->node(v, a.i, da));
    return AD(v, g_tape->node(v, a.i, da, b.i, db));
}

inline AD operator+(const AD &a, const AD &b) { return mk2(a.v + b.v, a, 1.0, b, 1.0); }
inline AD operator-(const AD &a, const AD &b) { return mk2(a.v - b.v, a, 1.0, b, -1.0); }
inline AD operator*(const AD &a, const AD &b) { return mk2(a.v * b.v, a, b.v, b, a.v); }
inline AD operator/(const AD &a, const AD &b) { return mk2(a.v / b.v, a, 1.0 / b.v, b, -a.v / (b.v * b.v)); }
inline AD operator-(const AD &a) { return mk(-a.v, a, -1.0); }
inline AD operator+(const AD &a, double b) { return mk(a.v + b, a, 1.0); }
inline AD operator+(double a, const AD &b) { return mk(a + b.v, b, 1.0); }
inline AD operator-(const AD &a, double b) { return mk(a.v - b, a, 1.0); }
inline AD operator-(double a, const AD &b) { return mk(a - b.v, b, -1.0); }
inline AD operator*(const AD &a, double b) { return mk(a.v * b, a, b); }
inline AD operator*(double a, const AD &b) { return mk(a * b.v, b, a); }
inline AD operator/(const AD &a, double b) { return mk(a.v / b, a, 1.0 / b); }
inline AD &operator+=(AD &a, const AD &b) { a = a + b; return a; }
inline bool operator<(const AD &a, const AD &b) { return a.v < b.v; }
inline bool operator>(const AD &a, const AD &b) { return a.v > b.v; }
inline bool operator<=(const AD &a, const AD &b) { return a.v <= b.v; }

inline AD sin(const AD &a) { return mk(std::sin(a.v), a, std::cos(a.v)); }
inline AD cos(const AD &a) { return mk(std::cos(a.v), a, -std::sin(a.v)); }
inline AD sqrt(const AD &a) { double r = std::sqrt(a.v); return mk(r, a, r > 0 ? 0.5 / r : 0.0); }
inline AD fabs(const AD &a) { return mk(std::fabs(a.v), a, a.v < 0 ? -1.0 : 1.0); }
inline AD atan(const AD &a) { return mk(std::atan(a.v), a, 1.0 / (1.0 + a.v * a.v)); }
inline AD atan2(const AD &y, const AD &x)
{
    double r2 = x.v * x.v + y.v * y.v;
    if (r2 == 0.0) return AD(std::atan2(y.v, x.v));
    return mk2(std::atan2(y.v, x.v), y, x.v / r2, x, -y.v / r2);
}
inline double value(const AD &a) { return a.v; }
inline double value(double a) { return a; }

// ---- the model, templated ------------------------------------------------
template <class T> T Tsin(const T &a) { using std::sin; return sin(a); }
template <class T> T Tcos(const T &a) { using std::cos; return cos(a); }
template <class T> T Tsqrt(const T &a) { using std::sqrt; return sqrt(a); }
template <class T> T Tfabs(const T &a) { using std::fabs; return fabs(a); }
template <class T> T Tatan2(const T &y, const T &x) { using std::atan2; return atan2(y, x); }

template <class T> T clampT(const T &v, double lo, double hi)
{
    if (value(v) < lo) return T(lo);
    if (value(v) > hi) return T(hi);
    return v;
}

struct K {
    double Fs[4], k[4], b[4], rho[4][3], U0, eps;
};

void consts(const orc_vehicle *v, const orc_cost *c, K &k)
{
    double L = v->Lf + v->Lr, he = 0.5 * v->e;
    double Kzz[4] = {v->M * v->Lr / L, v->M * v->Lr / L, v->M * v->Lf / L, v->M * v->Lf / L};
    double rx[4] = {v->Lf, v->Lf, -v->Lr, -v->Lr}, ry[4] = {he, -he, he, -he};
    for (int i = 0; i < 4; ++i) {
        k.Fs[i] = 0.5 * v->g * Kzz[i];
        k.k[i] = i < 2 ? v->kf : v->kr;
        k.b[i] = i < 2 ? v->bf : v->br;
        k.rho[i][0] = rx[i];
        k.rho[i][1] = ry[i];
        k.rho[i][2] = -v->hR;
    }
    k.U0 = orc_esm(v, 0.0, 0.0);
    k.eps = c->eps_esm > 0 ? c->eps_esm : 0.1 * k.U0;
}

// ESM (Sec. IV-B)
template <class T> T esmT(const orc_vehicle *v, const T &phi, const T &theta)
{
    double Rbar = std::sqrt(v->hR * v->hR + 0.25 * v->e * v->e);
    double phibar = std::atan(2.0 * v->hR / v->e);
    T a = Tfabs(phi) + phibar;
    T dh = Rbar * (1.0 - Tsin(a)) * Tcos(theta);
    double s = value(a) < 0.5 * M_PI ? 1.0 : -1.0;
    return s * v->M * v->g * dh;
}

// bilinear lookup of heights, slopes and costmap (reading Q10)
template <class T> void sampleT(const orc_terrain *t, const T &x, const T &y, T out[4])
{
    T u = (x - t->x0) / t->cell, w = (y - t->y0) / t->cell;
    double umax = t->nx - 1, wmax = t->ny - 1;
    u = clampT(u, 0.0, umax);
    w = clampT(w, 0.0, wmax);
    int i = (int)std::floor(value(u)), j = (int)std::floor(value(w));
    if (i > t->nx - 2) i = t->nx - 2;
    if (j > t->ny - 2) j = t->ny - 2;
    T a = u - (double)i, b = w - (double)j;
    T w00 = (1.0 - a) * (1.0 - b), w10 = a * (1.0 - b), w01 = (1.0 - a) * b, w11 = a * b;
    const int i00 = j * t->nx + i, i10 = i00 + 1, i01 = i00 + t->nx, i11 = i01 + 1;
    out[0] = w00 * (double)t->heights[i00] + w10 * (double)t->heights[i10] +
             w01 * (double)t->heights[i01] + w11 * (double)t->heights[i11];
    out[1] = w00 * t->gx[i00] + w10 * t->gx[i10] + w01 * t->gx[i01] + w11 * t->gx[i11];
    out[2] = w00 * t->gy[i00] + w10 * t->gy[i10] + w01 * t->gy[i01] + w11 * t->gy[i11];
    if (t->costmap)
        out[3] = w00 * (double)t->costmap[i00] + w10 * (double)t->costmap[i10] +
                 w01 * (double)t->costmap[i01] + w11 * (double)t->costmap[i11];
    else
        out[3] = T(0.0);
}

// xi_dot = A(xi) + B zeta and the running cost rate (Sec. IV-A, IV-C)
template <class T>
void derivT(const orc_vehicle *v, const K &k, const orc_cost *c, const orc_terrain *t, const T xi[13],
            const T zeta[2], T xd[13], T &L)
{
    T cps = Tcos(xi[3]), sps = Tsin(xi[3]), cth = Tcos(xi[4]), sth = Tsin(xi[4]);
    T cph = Tcos(xi[5]), sph = Tsin(xi[5]);
    T R[9];
    R[0] = cps * cth;
    R[1] = cps * sph * sth - cph * sps;
    R[2] = sph * sps + cph * cps * sth;
    R[3] = cth * sps;
    R[4] = cph * cps + sph * sps * sth;
    R[5] = cph * sps * sth - cps * sph;
    R[6] = -sth;
    R[7] = cth * sph;
    R[8] = cph * cth;
    T gB[3] = {-v->g * R[6], -v->g * R[7], -v->g * R[8]};
    T vB[3] = {xi[6], xi[7], xi[8]}, w[3] = {xi[9], xi[10], xi[11]};
    T wxbz[3] = {w[1], -w[0], T(0.0)};
    T Fy_sum(0.0), Fz_sum(0.0), M[3] = {T(0.0), T(0.0), T(0.0)}, cmap(0.0);
    for (int i = 0; i < 4; ++i) {
        const double *rho = k.rho[i];
        T P[3], vi[3], ter[4], tauB[3];
        P[0] = xi[0] + R[0] * rho[0] + R[1] * rho[1] + R[2] * rho[2];
        P[1] = xi[1] + R[3] * rho[0] + R[4] * rho[1] + R[5] * rho[2];
        P[2] = xi[2] + R[6] * rho[0] + R[7] * rho[1] + R[8] * rho[2];
        vi[0] = vB[0] + (w[1] * rho[2] - w[2] * rho[1]);
        vi[1] = vB[1] + (w[2] * rho[0] - w[0] * rho[2]);
        vi[2] = vB[2] + (w[0] * rho[1] - w[1] * rho[0]);
        sampleT(t, P[0], P[1], ter);
        T tW[3] = {-ter[1], -ter[2], T(1.0)};
        tauB[0] = R[0] * tW[0] + R[3] * tW[1] + R[6] * tW[2];
        tauB[1] = R[1] * tW[0] + R[4] * tW[1] + R[7] * tW[2];
        tauB[2] = R[2] * tW[0] + R[5] * tW[1] + R[8] * tW[2];
        T chi = (P[2] - ter[0]) / tauB[2];
        T rel[3] = {vi[0] - chi * wxbz[0], vi[1] - chi * wxbz[1], vi[2] - chi * wxbz[2]};
        T chid = (tauB[0] * rel[0] + tauB[1] * rel[1] + tauB[2] * rel[2]) / tauB[2];
        T Fk = k.Fs[i] - k.k[i] * chi;
        if (value(Fk) < 0.0) Fk = T(0.0);
        T Fb(0.0);
        if (value(Fk) > 0.0) {
            Fb = -k.b[i] * chid;
            if (value(Fb) < -value(Fk)) Fb = -Fk;
        }
        T Fz = Fk + Fb;
        T di = i < 2 ? xi[12] : T(0.0);
        T alpha = Tatan2(vi[1], vi[0]) - di;
        T Ca = v->C * alpha;
        T den = Tsqrt(v->mu * v->mu + Ca * Ca);
        T Fy = (value(den) == 0.0) ? T(0.0) : Fz * (-Ca * v->mu / den);
        T Fx = (i >= 2) ? 0.5 * v->M * (zeta[1] - gB[0] + w[1] * vB[2] - w[2] * vB[1]) : T(0.0);
        T cdi = Tcos(di);
        Fy_sum += Fy * cdi;
        Fz_sum += Fz;
        T F[3] = {Fx, Fy * cdi, Fz};
        M[0] += rho[1] * F[2] - rho[2] * F[1];
        M[1] += rho[2] * F[0] - rho[0] * F[2];
        M[2] += rho[0] * F[1] - rho[1] * F[0];
        cmap += ter[3];
    }
    xd[0] = R[0] * vB[0] + R[1] * vB[1] + R[2] * vB[2];
    xd[1] = R[3] * vB[0] + R[4] * vB[1] + R[5] * vB[2];
    xd[2] = R[6] * vB[0] + R[7] * vB[1] + R[8] * vB[2];
    xd[3] = (sph / cth) * w[1] + (cph / cth) * w[2];
    xd[4] = cph * w[1] - sph * w[2];
    xd[5] = w[0] + (sph * sth / cth) * w[1] + (cph * sth / cth) * w[2];
    xd[6] = zeta[1];
    xd[7] = Fy_sum / v->M + gB[1] + w[0] * vB[2] - w[2] * vB[0];
    xd[8] = Fz_sum / v->M + gB[2] - w[0] * vB[1] + w[1] * vB[0];
    xd[9] = (M[0] + (v->Jyy - v->Jzz) * w[1] * w[2]) / v->Jxx;
    xd[10] = (M[1] - (v->Jxx - v->Jzz) * w[0] * w[2]) / v->Jyy;
    xd[11] = (M[2] + (v->Jxx - v->Jyy) * w[0] * w[1]) / v->Jzz;
    xd[12] = zeta[0];
    T U = esmT(v, xi[5], xi[4]);
    T s = 1.0 - U / k.eps;
    if (value(s) < 0.0) s = T(0.0);
    L = (c->wt + c->wc * zeta[0] * zeta[0]) + (c->sigma * s * s + cmap);
}

// J of one candidate: Euler with zero-order hold, goal truncation, terminal
// distance (Sec. IV-C, IV-D); u[H][2] are the raw controls
template <class T>
T costT(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13], const T *u,
        int H, double dt, int n_sub)
{
    K k;
    consts(v, c, k);
    const double h = dt / n_sub;
    T xi[13], xd[13], L;
    for (int q = 0; q < 13; ++q) xi[q] = T(x0[q]);
    T J(0.0);
    bool done = false;
    for (int kk = 0; kk < H && !done; ++kk) {
        T zeta[2] = {clampT(u[2 * kk], -v->delta_rate_max, v->delta_rate_max), u[2 * kk + 1]};
        for (int s = 0; s < n_sub; ++s) {
            double dx = value(xi[0]) - c->goal_x, dy = value(xi[1]) - c->goal_y;
            if (std::sqrt(dx * dx + dy * dy) <= c->goal_r) {
                done = true;
                break;
            }
            derivT(v, k, c, t, xi, zeta, xd, L);
            J += h * L;
            for (int q = 0; q < 13; ++q) xi[q] = xi[q] + h * xd[q];
            xi[12] = clampT(xi[12], -v->delta_max, v->delta_max);
        }
    }
    T gx = xi[0] - c->goal_x, gy = xi[1] - c->goal_y;
    J += c->wg * Tsqrt(gx * gx + gy * gy);
    return J;
}

}  // namespace

extern "C" {

// J in plain FP64 through the templated restatement (checks it against srb.c)
double orc_cost_templated(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13],
                          const float *ctrl, int H, double dt, int n_sub)
{
    std::vector<double> u(2 * (size_t)H);
    for (int i = 0; i < 2 * H; ++i) u[i] = ctrl[i];
    return costT<double>(v, c, t, x0, u.data(), H, dt, n_sub);
}

// J in plain FP64 with FP64 controls u[H][2] (central finite differences)
double orc_cost_f64(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13],
                    const double *u, int H, double dt, int n_sub)
{
    return costT<double>(v, c, t, x0, u, H, dt, n_sub);
}

// J and dJ/du (grad[H][2]) of one candidate by reverse-mode AD on a tape
double orc_grad(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13],
                const float *ctrl, int H, double dt, int n_sub, double *grad)
{
    Tape tape;
    tape.val.reserve(1 << 20);
    g_tape = &tape;
    std::vector<AD> u(2 * (size_t)H);
    for (int i = 0; i < 2 * H; ++i) u[i] = AD((double)ctrl[i], tape.node((double)ctrl[i]));
    AD J = costT<AD>(v, c, t, x0, u.data(), H, dt, n_sub);
    std::vector<double> adj(tape.val.size(), 0.0);
    if (J.i >= 0) {
        adj[J.i] = 1.0;
        for (int n = J.i; n >= 0; --n) {
            if (adj[n] == 0.0) continue;
            if (tape.pa[n] >= 0) adj[tape.pa[n]] += adj[n] * tape.da[n];
            if (tape.pb[n] >= 0) adj[tape.pb[n]] += adj[n] * tape.db[n];
        }
    }
    for (int i = 0; i < 2 * H; ++i) grad[i] = adj[u[i].i];
    g_tape = nullptr;
    return J.v;
}

// J and gradients of N candidates (ctrl [H][N][2], x0 [N][13] or shared [13]), OpenMP over candidates
int orc_grad_batch(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const float *x0,
                   int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub, double *J,
                   double *grad)
{
    if (N <= 0 || H <= 0 || n_sub <= 0 || !(dt > 0.0)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < N; ++j) {
        double xs[13];
        std::vector<float> uj(2 * (size_t)H);
        std::vector<double> gj(2 * (size_t)H);
        const float *src = x0 + (x0_per_cand ? (size_t)j * 13 : 0);
        for (int q = 0; q < 13; ++q) xs[q] = src[q];
        for (int k = 0; k < H; ++k) {
            uj[2 * k] = ctrl[((size_t)k * N + j) * 2];
            uj[2 * k + 1] = ctrl[((size_t)k * N + j) * 2 + 1];
        }
        J[j] = orc_grad(v, c, t, xs, uj.data(), H, dt, n_sub, gj.data());
        for (int k = 0; k < H; ++k) {
            grad[((size_t)k * N + j) * 2] = gj[2 * k];
            grad[((size_t)k * N + j) * 2 + 1] = gj[2 * k + 1];
        }
    }
    return 0;
}

}  // extern "C"
