// adjoint.cpp - FP64 CPU adjoint of the discrete SRB rollout cost (arxiv
// 2603.20525, Sec. IV-A..IV-C): the gradient of J = sum h L + Phi with respect
// to the raw control sequence, by generic reverse-mode automatic
// differentiation on a tape (every elementary operation records its local
// partial derivatives; one backward sweep accumulates the adjoints).  Nothing
// here is derived by hand, so it checks the CUDA path's hand-written adjoint
// independently.
//
// TEST INFRASTRUCTURE.  Only the test suite may load it; it shares no code
// with the CUDA path.  The model is the templated restatement of model.hpp
// (for T = double it reproduces srb.c's rollout, checked by the tests),
// instantiated on the tape scalar below.
#include <cmath>
#include <cstring>
#include <vector>

#include "model.hpp"

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
inline AD asin(const AD &a) { return mk(std::asin(a.v), a, 1.0 / std::sqrt(1.0 - a.v * a.v)); }
inline double value(const AD &a) { return a.v; }

// J of one candidate through the templated model (model.hpp): Euler with
// zero-order hold, goal truncation, terminal distance (Sec. IV-C, IV-D);
// u[H][2] are the raw controls
template <class T>
T costT(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13], const T *u,
        int H, double dt, int n_sub)
{
    return orcm::rolloutT<T, T>(v, c, t, x0, u, H, dt, n_sub).J;
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

// The objective (0: J; 1: the ESM margin, min U_ESM over the trajectory) of
// one candidate and its gradient grad[H][2] by reverse-mode AD on a tape.  The
// margin's minimum is taken by value (the first state holding it), so the tape
// records the subgradient through that state.
static double tape_grad(int objective, const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                        const double x0[13], const float *ctrl, int H, double dt, int n_sub, double *grad)
{
    Tape tape;
    tape.val.reserve(1 << 20);
    g_tape = &tape;
    std::vector<AD> u(2 * (size_t)H);
    for (int i = 0; i < 2 * H; ++i) u[i] = AD((double)ctrl[i], tape.node((double)ctrl[i]));
    const orcm::Result<AD> r = orcm::rolloutT<AD, AD>(v, c, t, x0, u.data(), H, dt, n_sub);
    const AD f = objective == 0 ? r.J : r.margin;
    std::vector<double> adj(tape.val.size(), 0.0);
    if (f.i >= 0) {
        adj[f.i] = 1.0;
        for (int n = f.i; n >= 0; --n) {
            if (adj[n] == 0.0) continue;
            if (tape.pa[n] >= 0) adj[tape.pa[n]] += adj[n] * tape.da[n];
            if (tape.pb[n] >= 0) adj[tape.pb[n]] += adj[n] * tape.db[n];
        }
    }
    for (int i = 0; i < 2 * H; ++i) grad[i] = adj[u[i].i];
    g_tape = nullptr;
    return f.v;
}

// J and dJ/du (grad[H][2]) of one candidate by reverse-mode AD on a tape
double orc_grad(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13],
                const float *ctrl, int H, double dt, int n_sub, double *grad)
{
    return tape_grad(0, v, c, t, x0, ctrl, H, dt, n_sub, grad);
}

// The objective (0: J; 1: the margin) and its gradient for N candidates
// (ctrl [H][N][2], x0 [N][13] or shared [13]), OpenMP over candidates.
static int grad_batch(int objective, const orc_vehicle *v, const orc_cost *c, const orc_terrain *t,
                      const float *x0, int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub,
                      double *F, double *grad)
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
        F[j] = tape_grad(objective, v, c, t, xs, uj.data(), H, dt, n_sub, gj.data());
        for (int k = 0; k < H; ++k) {
            grad[((size_t)k * N + j) * 2] = gj[2 * k];
            grad[((size_t)k * N + j) * 2 + 1] = gj[2 * k + 1];
        }
    }
    return 0;
}

int orc_grad_batch(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const float *x0,
                   int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub, double *J,
                   double *grad)
{
    return grad_batch(0, v, c, t, x0, x0_per_cand, ctrl, N, H, dt, n_sub, J, grad);
}

// the ESM margin (min U_ESM over the trajectory) and d(margin)/du
int orc_grad_margin_batch(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const float *x0,
                          int x0_per_cand, const float *ctrl, int N, int H, double dt, int n_sub,
                          double *margin, double *grad)
{
    return grad_batch(1, v, c, t, x0, x0_per_cand, ctrl, N, H, dt, n_sub, margin, grad);
}

// the margin of one candidate in plain FP64 with FP64 controls u[H][2]
// (central finite differences)
double orc_margin_f64(const orc_vehicle *v, const orc_cost *c, const orc_terrain *t, const double x0[13],
                      const double *u, int H, double dt, int n_sub)
{
    return orcm::rolloutT<double, double>(v, c, t, x0, u, H, dt, n_sub).margin;
}

}  // extern "C"
