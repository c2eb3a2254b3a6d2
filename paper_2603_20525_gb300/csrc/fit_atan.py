"""Derives the coefficients of the arctangent polynomial in fastmath.cuh.

atan(r) = r * P(r^2) on r in [0, 1], P of degree 8, fitted to
atan(sqrt(s)) / sqrt(s) on s in [0, 1] by iteratively reweighted least
squares on Chebyshev-spaced nodes (Lawson's algorithm), minimising the
maximum *relative* error so that small slip angles keep FP32 relative
accuracy.  Prints the FP32 coefficients and the achieved errors.
Run: python paper_2603_20525_gb300/csrc/fit_atan.py
"""
import numpy as np

DEG = 8


def target(s):
    r = np.sqrt(s)
    out = np.ones_like(s)
    m = r > 0
    out[m] = np.arctan(r[m]) / r[m]
    return out


def fit(deg=DEG, n=4000, iters=200):
    s = 0.5 * (1 - np.cos(np.linspace(0, np.pi, n)))
    y = target(s)
    V = np.vander(s, deg + 1, increasing=True)
    w = np.ones(n)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * (w / y)[:, None], w, rcond=None)
        e = np.abs(V @ c - y) / y
        w = w * np.sqrt(e / e.max()) + 1e-12
        w /= w.max()
    return c


def main():
    c = fit().astype(np.float32)
    s = np.linspace(0, 1, 400001)
    y = target(s)
    p = np.float32(c[-1])
    s32 = s.astype(np.float32)
    for k in range(DEG - 1, -1, -1):
        p = (p * s32 + c[k]).astype(np.float32)
    rel = np.abs(p.astype(np.float64) - y) / y
    print("coefficients (c0..c8):")
    for v in c:
        print(f"    {float(v)!r}f,")
    print(f"max relative error with FP32 coefficients and evaluation: {rel.max():.3e}")


if __name__ == "__main__":
    main()
