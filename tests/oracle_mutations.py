"""Mutation check of the oracle's pins: each plausible mistake below
(a wrong sign, a swapped index, a dropped term, a transposed rotation, a
changed clamp, threshold or boundary rule) is planted, one at a time, in a
copy of the oracle, and the pin tests of that file must fail.

Run by hand (a few minutes, CPU only; pytest does not collect this file):

    python tests/oracle_mutations.py

Each run copies oracle/, gen/ and tests/ into a temporary tree, plants the
mistake there and runs the pins of that tree, so the repository's own
oracle is never touched.  Two planted changes leave the model's behaviour
unchanged and are expected to survive: moving the rear longitudinal
constraint force to the front wheels (the moments about the CoM are the
same), and casting the inside test's ray towards -x (the even-odd parity of
a closed polygon is the same).
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in the source, replacement)
SRB = [
 ("Q1 sign", "tauW[0] = -ter[1];", "tauW[0] = ter[1];"),
 ("Kzz swap", "double Kzzf = v->M * v->Lr / L;", "double Kzzf = v->M * v->Lf / L;"),
 ("vy wx*vz sign", "w[0] * vB[2] - w[2] * vB[0];", "- w[0] * vB[2] - w[2] * vB[0];"),
 ("wy gyro sign", "(Msum[1] - (v->Jxx - v->Jzz)", "(Msum[1] + (v->Jxx - v->Jzz)"),
 ("R[1] sign", "R[1] = cps * sph * sth - cph * sps;", "R[1] = cps * sph * sth + cph * sps;"),
 ("damper clamp", "if (Fb < -Fk) Fb = -Fk;", "if (Fb < -2*Fk) Fb = -2*Fk;"),
 ("alpha +delta", "alpha = atan2(vi[1], vi[0]) - di;", "alpha = atan2(vi[1], vi[0]) + di;"),
 ("no cos delta", "Fy_sum += Fy * cos(di);", "Fy_sum += Fy;"),
 ("chidot wxbz sign", "rel[0] = vi[0] - chi * wxbz[0];", "rel[0] = vi[0] + chi * wxbz[0];"),
 ("esm no abs", "double a = fabs(phi) + phibar;", "double a = phi + phibar;"),
 ("esm no cos", "double dh = Rbar * (1.0 - sin(a)) * cos(theta);", "double dh = Rbar * (1.0 - sin(a));"),
 ("cost linear", "L0 = c->wt + c->wc * zeta[0] * zeta[0];", "L0 = c->wt + c->wc * fabs(zeta[0]);"),
 ("no delta clamp", "xi[DELTA] = clampd(xi[DELTA], -v->delta_max, v->delta_max);", ""),
 ("theta rate sign", "xidot[THETA] = cphi * w[1] - sphi * w[2];", "xidot[THETA] = cphi * w[1] + sphi * w[2];"),
 ("Fx gB sign", "Fx = 0.5 * v->M * (zeta[1] - gB[0]", "Fx = 0.5 * v->M * (zeta[1] + gB[0]"),
 ("no final margin", "if (U < margin) margin = U;\n        if (fabs(U) / k->U0 < d_esm) d_esm = fabs(U) / k->U0;\n        if (step_margin && H > 0)", "if (fabs(U) / k->U0 < d_esm) d_esm = fabs(U) / k->U0;\n        if (step_margin && H > 0)"),
 ("select ties high", "(inf_j == inf_b && J[j] < J[best])", "(inf_j == inf_b && J[j] <= J[best])"),
 ("gy halfcell", "gy[j * nx + i] = (a - b) / (2.0 * cell); }", "gy[j * nx + i] = (a - b) / cell; }"),
 ("bilinear swap", "w10 = a * (1.0 - b);\n    w01 = (1.0 - a) * b;", "w10 = (1.0 - a) * b;\n    w01 = a * (1.0 - b);"),
 ("damper sign", "Fb = -k->b[i] * chidot;", "Fb = k->b[i] * chidot;"),
 ("Fx on front", "if (i == RL || i == RR)\n            Fx", "if (i == FL || i == FR)\n            Fx"),
 ("vz wx vy sign", "gB[2] - w[0] * vB[1]", "gB[2] + w[0] * vB[1]"),
 ("wz gyro", "(v->Jxx - v->Jyy) * w[0] * w[1]", "(v->Jyy - v->Jxx) * w[0] * w[1]"),
 ("pos R^T", "xidot[X] = R[0] * vB[0] + R[1] * vB[1] + R[2] * vB[2];", "xidot[X] = R[0] * vB[0] + R[3] * vB[1] + R[6] * vB[2];"),
 ("goal strict", "if (gd <= c->goal_r) {\n                    done = 1;", "if (gd < c->goal_r - 0.001) {\n                    done = 1;"),
 ("Fs half missing", "k->Fs[i] = 0.5 * v->g * k->Kzz[i];", "k->Fs[i] = v->g * k->Kzz[i];"),
]

EST = [
 ("normal sign", "const double tau[3] = {-ter[1] / n, -ter[2] / n, 1.0 / n};", "const double tau[3] = {ter[1] / n, -ter[2] / n, 1.0 / n};"),
 ("phi sign", "const double phi = atan2(-tau[1], tau[2]);", "const double phi = atan2(tau[1], tau[2]);"),
 ("theta sign", "const double theta = asin(tau[0]);", "const double theta = asin(-tau[0]);"),
 ("R[3] sign", "R[3] = cf * sp + cp * sf * st;", "R[3] = cf * sp - cp * sf * st;"),
 ("gB column", "const double gB[3] = {-v->g * R[6], -v->g * R[7], -v->g * R[8]};", "const double gB[3] = {-v->g * R[2], -v->g * R[5], -v->g * R[8]};"),
 ("aBx sign", "const double aBx = zeta[1] - wz * vy;", "const double aBx = zeta[1] + wz * vy;"),
 ("Kzx sign front", "const double Fzf = -k->Kzzf * gB[2] - k->Kzx * aBx;", "const double Fzf = -k->Kzzf * gB[2] + k->Kzx * aBx;"),
 ("Kzz swap", "k->Kzzf = v->M * v->Lr / L;", "k->Kzzf = v->M * v->Lf / L;"),
 ("alpha_f +delta", "const double af = atan2(vy + wz * v->Lf, vx) - delta;", "const double af = atan2(vy + wz * v->Lf, vx) + delta;"),
 ("alpha_r sign", "const double ar = atan2(vy - wz * v->Lr, vx);", "const double ar = atan2(vy + wz * v->Lr, vx);"),
 ("dvy centripetal sign", "xidot[EVY] = (Fyf + Fyr) / v->M + gB[1] - wz * vx;", "xidot[EVY] = (Fyf + Fyr) / v->M + gB[1] + wz * vx;"),
 ("dvy no gravity", "xidot[EVY] = (Fyf + Fyr) / v->M + gB[1] - wz * vx;", "xidot[EVY] = (Fyf + Fyr) / v->M - wz * vx;"),
 ("dwz no cos", "xidot[EWZ] = (Fyf * v->Lf * cos(delta) - Fyr * v->Lr) / v->Jzz;", "xidot[EWZ] = (Fyf * v->Lf - Fyr * v->Lr) / v->Jzz;"),
 ("dwz rear sign", "xidot[EWZ] = (Fyf * v->Lf * cos(delta) - Fyr * v->Lr) / v->Jzz;", "xidot[EWZ] = (Fyf * v->Lf * cos(delta) + Fyr * v->Lr) / v->Jzz;"),
 ("xdot transposed", "xidot[EX] = R[0] * vx + R[1] * vy;", "xidot[EX] = R[0] * vx + R[3] * vy;"),
 ("margin no gravity", "const double margin = k->abar - fabs(aBy - gB[1]);", "const double margin = k->abar - fabs(aBy);"),
 ("abar factor 2", "k->abar = v->M * v->g / (2.0 * k->Kzy);", "k->abar = v->M * v->g / k->Kzy;"),
 ("soft sign", "const double viol = 1.0 - margin / k->eps;", "const double viol = 1.0 + margin / k->eps;"),
 ("rho z sign", "k->rho[i][2] = -v->hR;", "k->rho[i][2] = v->hR;"),
 ("rho y same side", "k->rho[i][1] = (i & 1) ? -0.5 * v->e : 0.5 * v->e;", "k->rho[i][1] = 0.5 * v->e;"),
 ("goal strict", "if (gd <= c->goal_r) done = 1;\n            }\n            if (!done) {", "if (gd < c->goal_r - 0.01) done = 1;\n            }\n            if (!done) {"),
 ("no delta clamp", "xi[EDELTA] = clampv(xi[EDELTA], -v->delta_max, v->delta_max);", ""),
 ("no rate clamp", "zeta[0] = clampv((double)ctrl[(size_t)kk * ctrl_stride], -v->delta_rate_max, v->delta_rate_max);", "zeta[0] = (double)ctrl[(size_t)kk * ctrl_stride];"),
 ("eps default", "k->eps = c->eps_esm > 0.0 ? c->eps_esm : 0.1 * k->abar;", "k->eps = c->eps_esm > 0.0 ? c->eps_esm : 0.2 * k->abar;"),
 ("feasible >=", "if (finite && margin > 0.0) fl |= ORC_FEASIBLE;", "if (finite && margin > -1.0) fl |= ORC_FEASIBLE;"),
]

TERRAIN = [
 ("gauss exponent", "w[k + r] = exp(-0.5 * (double)k * (double)k / (s * s));", "w[k + r] = exp(-(double)k * (double)k / (s * s));"),
 ("cut 3 sigma", "int r = (int)(4.0 * s + 0.5);", "int r = (int)(3.0 * s + 0.5);"),
 ("no normalisation", "for (int k = 0; k <= 2 * r; ++k) w[k] /= z;", ""),
 ("wrap border", "const int jj = clampi(j + b, 0, ny - 1);", "const int jj = (j + b + ny) % ny;"),
 ("same axis weight", "acc += w[a + r] * w[b + r] * (double)f[(size_t)jj * nx + ii];", "acc += w[a + r] * w[a + r] * (double)f[(size_t)jj * nx + ii];"),
 ("segment as line", "        if (t < 0.0) t = 0.0;\n        if (t > 1.0) t = 1.0;\n", ""),
 ("ray direction", "if (px < xc) inside = !inside;", "if (px > xc) inside = !inside;"),
 ("kind sign", "const int negative = kind == 0 ? inside : !inside;", "const int negative = kind == 0 ? !inside : inside;"),
 ("cost sign", "const double v = 1.0 - s / eps;", "const double v = 1.0 + s / eps;"),
 ("cost linear", "if (v > 0.0) c += sigma * v * v;", "if (v > 0.0) c += sigma * v;"),
 ("node half cell", "const double px = x0 + i * cell, py = y0 + j * cell;", "const double px = x0 + (i + 0.5) * cell, py = y0 + j * cell;"),
 ("open polygon", "const int m = (k + 1) % n;", "const int m = k + 1 < n ? k + 1 : k;"),
 ("crossing half-open", "if ((ay > py) != (by > py)) {", "if ((ay >= py) != (by > py)) {"),
]

SAMPLER = [
 ("rounds 9", "for (r = 0; r < 10; ++r) {", "for (r = 0; r < 9; ++r) {"),
 ("key bumped before the first round", "if (r > 0) {", "if (r >= 0) {"),
 ("word order", "n[1] = lo1;", "n[1] = lo0;"),
 ("shift ignored", "int src = k + shift;", "int src = k;"),
 ("sin for both", "sigma_rate * r * cos(2.0 * M_PI * u2)", "sigma_rate * r * sin(2.0 * M_PI * u2)"),
 ("sigmas swapped", "o[0] = nom[0] + sigma_rate", "o[0] = nom[0] + sigma_acc"),
 ("nominal at candidate 1", "if (j == 0) {", "if (j == 1) {"),
 ("one call per step", "(uint64_t)(k / 4)", "(uint64_t)k"),
 ("word pairs swapped", "u1 = unif23((s & 1) ? w[2] : w[0], low);", "u1 = unif23((s & 1) ? w[0] : w[2], low);"),
 ("low uniform from other bits", "(w >> 9) & 0x7FFFFFull", "(w >> 8) & 0x7FFFFFull"),
]

ADJOINT = [
 ("d sin sign", "inline AD sin(const AD &a) { return mk(std::sin(a.v), a, std::cos(a.v)); }",
  "inline AD sin(const AD &a) { return mk(std::sin(a.v), a, -std::cos(a.v)); }"),
 ("d cos sign", "inline AD cos(const AD &a) { return mk(std::cos(a.v), a, -std::sin(a.v)); }",
  "inline AD cos(const AD &a) { return mk(std::cos(a.v), a, std::sin(a.v)); }"),
 ("d sqrt factor", "return mk(r, a, r > 0 ? 0.5 / r : 0.0); }", "return mk(r, a, r > 0 ? 1.0 / r : 0.0); }"),
 ("d quotient sign", "b, -a.v / (b.v * b.v)); }", "b, a.v / (b.v * b.v)); }"),
 ("d product swapped", "return mk2(a.v * b.v, a, b.v, b, a.v); }", "return mk2(a.v * b.v, a, a.v, b, b.v); }"),
 ("d atan2 swapped", "return mk2(std::atan2(y.v, x.v), y, x.v / r2, x, -y.v / r2);",
  "return mk2(std::atan2(y.v, x.v), y, -y.v / r2, x, x.v / r2);"),
 ("d fabs", "return mk(std::fabs(a.v), a, a.v < 0 ? -1.0 : 1.0); }", "return mk(std::fabs(a.v), a, 1.0); }"),
]

BF16 = [
 ("round half up", "b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16", "b = (b + 0x8000) >> 16"),
 ("truncate", "b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16", "b = b >> 16"),
 ("slope over n", "f32(f32(1.0) / f32(ni - 1))) if ni > 1", "f32(f32(1.0) / f32(ni))) if ni > 1"),
 ("plane through the block centre", "c0 = H[j0, i0]", "c0 = H[j0 + nj // 2, i0 + ni // 2]"),
 ("plane slopes not removed", "w_gx = bf16_round((g.gx.astype(np.float32) - px).astype(np.float32))",
  "w_gx = bf16_round(g.gx.astype(np.float32))"),
 ("y slope from x", "py = (P[..., 2] * inv).astype(np.float32)", "py = (P[..., 1] * inv).astype(np.float32)"),
]

MODEL = [
 ("R[4] sign", "R[4] = cph * cps + sph * sps * sth;", "R[4] = cph * cps - sph * sps * sth;"),
 ("chi from the wrong corner", "T chi = T(P[2] - ter[0]) / tauB[2];", "T chi = T(P[2] - ter[1]) / tauB[2];"),
 ("minimum step last on ties", "if (value(sm) < value(best_sm)) {", "if (value(sm) <= value(best_sm)) {"),
 ("position not accumulated exactly", "constexpr bool kSrbWide[13] = {true,", "constexpr bool kSrbWide[13] = {false,"),
 ("planar aBx sign", "T aBx = zeta[1] - wz * vy;", "T aBx = zeta[1] + wz * vy;"),
 ("planar margin without gravity", "margin = k.abar - Tfabs(aBy - gB[1]);", "margin = k.abar - Tfabs(aBy);"),
]

COUNT = [
 ("multiplications not counted", "inline Cnt operator*(const Cnt &a, const Cnt &b) { ++g_cnt.mul; ",
  "inline Cnt operator*(const Cnt &a, const Cnt &b) { "),
 ("divisions counted twice", "{ ++g_cnt.div; return Cnt(a.v / b.v); }", "{ g_cnt.div += 2; return Cnt(a.v / b.v); }"),
]

EQUIVALENT = {("srb.c", "Fx on front"), ("terrain_tools.c", "ray direction")}


def run(fname, mutations, test):
    with open(os.path.join(ROOT, "oracle", fname)) as f:
        src = f.read()
    missed = []
    for name, a, b in mutations:
        assert src.count(a) >= 1, (fname, name)
        d = tempfile.mkdtemp()
        try:
            for sub in ("oracle", "gen", "tests"):
                shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                                ignore=shutil.ignore_patterns("_build", "__pycache__"))
            with open(os.path.join(d, "oracle", fname), "w") as f:
                f.write(src.replace(a, b, 1))
            env = dict(os.environ, PYTHONPATH=d)
            p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                                os.path.join(d, "tests", test)], cwd=d, env=env, capture_output=True,
                               text=True)
        finally:
            shutil.rmtree(d)
        caught = p.returncode != 0
        first = [l for l in p.stdout.splitlines() if l.startswith("FAILED")][:1]
        print(f"{fname}: {name}: {'caught' if caught else 'MISSED'} {first}", flush=True)
        if not caught and (fname, name) not in EQUIVALENT:
            missed.append((fname, name))
    return missed


if __name__ == "__main__":
    missed = (run("srb.c", SRB, "test_oracle_pins.py") + run("est.c", EST, "test_oracle_est.py") +
              run("terrain_tools.c", TERRAIN, "test_oracle_terrain_tools.py") +
              run("sampler.c", SAMPLER, "test_oracle_sampler.py") +
              run("adjoint.cpp", ADJOINT, "test_oracle_adjoint.py") +
              run("model.hpp", MODEL, "test_oracle_templated.py") +
              run("emul32.cpp", COUNT, "test_bench_host.py") +
              run("__init__.py", BF16, "test_oracle_bf16.py"))
    print("missed:", missed or "none beyond the two equivalent changes")
    sys.exit(1 if missed else 0)
