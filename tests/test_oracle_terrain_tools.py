"""Pins of the FP64 oracle of the terrain preprocessing steps: the Gaussian
level of detail (Sec. V-B) against SciPy's Gaussian filter, the closed form
of a sampled Gaussian's response to a sinusoid, exactness on constants and
planes, and its impulse response; the distance-constraint costmap (Sec.
IV-C, IV-D) against closed-form signed distances of a square, a circle and a
concave polygon and the soft-constraint values at the onset, the boundary
and one normaliser inside."""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle


def rough(n=64, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.3, (n, n + 7)).astype(np.float32)


# SciPy's gaussian_filter with the same standard deviation (in cells), the
# same cut at four standard deviations and the nearest-node extension.
@pytest.mark.parametrize("cell,sigma", [(0.1, 0.3), (0.2, 1.5), (0.5, 0.3), (0.1, 0.05)])
def test_lod_matches_scipy_gaussian_filter(cell, sigma):
    f = rough()
    got = oracle.lod_smooth(f, cell, sigma)
    ref = ndimage.gaussian_filter(f.astype(np.float64), sigma / cell, mode="nearest", truncate=4.0)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_lod_identity_constant_and_plane():
    f = rough()
    assert np.array_equal(oracle.lod_smooth(f, 0.1, 0.0), f.astype(np.float64))
    c = np.full((40, 50), 1.75, np.float32)
    np.testing.assert_allclose(oracle.lod_smooth(c, 0.1, 0.3), 1.75, rtol=0, atol=1e-14)
    # a plane is kept wherever the kernel does not reach the border
    j, i = np.mgrid[0:60, 0:70]
    p = (0.25 * i - 0.125 * j).astype(np.float32)
    r = int(4 * 0.3 / 0.1 + 0.5)
    out = oracle.lod_smooth(p, 0.1, 0.3)
    np.testing.assert_allclose(out[r:-r, r:-r], p[r:-r, r:-r], rtol=0, atol=1e-12)


def test_lod_impulse_response_is_gaussian():
    n, cell, sigma = 61, 0.1, 0.3
    f = np.zeros((n, n), np.float32)
    f[30, 30] = 1.0
    out = oracle.lod_smooth(f, cell, sigma)
    k = np.arange(-12, 13)
    g = np.exp(-0.5 * (k * cell / sigma) ** 2)
    g /= g.sum()
    np.testing.assert_allclose(out[18:43, 18:43], np.outer(g, g), rtol=0, atol=1e-15)
    assert out.sum() == pytest.approx(1.0, abs=1e-14)


# A sinusoid of wavelength lambda is scaled by exp(-2 pi^2 sigma^2 / lambda^2),
# the Fourier transform of the Gaussian, up to the cut at 4 sigma (a relative
# 3e-4 of the kernel's mass).
@pytest.mark.parametrize("lam", [1.0, 2.0, 4.0])
def test_lod_attenuates_sinusoid_as_gaussian_transfer(lam):
    n, cell, sigma = 400, 0.05, 0.3
    x = cell * np.arange(n)
    f = np.tile(np.cos(2 * np.pi * x / lam), (9, 1)).astype(np.float32)
    out = oracle.lod_smooth(f, cell, sigma)
    r = int(4 * sigma / cell + 0.5)
    mid = out[4, r:-r]
    gain = math.exp(-2 * math.pi ** 2 * sigma ** 2 / lam ** 2)
    np.testing.assert_allclose(mid, gain * f[4, r:-r].astype(np.float64), rtol=0, atol=4e-4 + 1e-6)


SQUARE = [(0.0, 0.0), (2.0, 0.0), (2.0, 2.0), (0.0, 2.0)]


@pytest.mark.parametrize("pt,expect", [((1.0, 1.0), -1.0), ((0.5, 1.2), -0.5), ((3.0, 1.0), 1.0),
                                       ((3.0, 3.0), math.sqrt(2.0)), ((1.0, -0.25), 0.25),
                                       ((2.0, 1.0), 0.0), ((-1.0, 2.5), math.hypot(1.0, 0.5))])
def test_sdist_square_closed_form(pt, expect):
    for poly in (SQUARE, SQUARE[::-1]):                # either orientation
        assert oracle.sdist(poly, 0, *pt) == pytest.approx(expect, abs=1e-15)
        # a path boundary counts the other side as violation
        assert oracle.sdist(poly, 1, *pt) == pytest.approx(-expect, abs=1e-15)


def test_sdist_circle_polygon():
    R, n, c = 3.0, 512, (1.0, -2.0)
    t = 2 * np.pi * np.arange(n) / n
    poly = np.stack([c[0] + R * np.cos(t), c[1] + R * np.sin(t)], 1)
    sag = R * (1 - math.cos(math.pi / n))               # chord sagitta
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = np.array(c) + rng.uniform(-6, 6, 2)
        expect = math.hypot(p[0] - c[0], p[1] - c[1]) - R
        assert abs(oracle.sdist(poly, 0, *p) - expect) <= sag + 1e-12


def test_sdist_concave_polygon_inside_by_union():
    # an L: the union of [0, 4] x [0, 1] and [0, 1] x [0, 3]
    L = [(0, 0), (4, 0), (4, 1), (1, 1), (1, 3), (0, 3)]
    rng = np.random.default_rng(4)
    for _ in range(400):
        x, y = rng.uniform(-1, 5), rng.uniform(-1, 4)
        inside = (0 < x < 4 and 0 < y < 1) or (0 < x < 1 and 0 < y < 3)
        s = oracle.sdist(L, 0, x, y)
        if abs(s) > 1e-12:
            assert (s < 0) == inside


# The normalised quadratic soft constraint sigma max(0, 1 + pi / eps)^2 with
# pi = -sdist (Sec. IV-C): 0 from eps outside on, sigma on the perimeter,
# 4 sigma one eps inside; contributions of several perimeters add up.
def test_costmap_soft_constraint_values_and_sum():
    eps, sig = 0.25, 1e6
    # nodes at x = -1, -0.75, ..., along y = 1 through the square's middle
    c, s = oracle.costmap([(SQUARE, 0)], 21, 1, 0.25, -1.0, 1.0, eps, sig)
    x = -1.0 + 0.25 * np.arange(21)
    for i, xi in enumerate(x):
        sd = oracle.sdist(SQUARE, 0, xi, 1.0)
        assert s[0, i] == sd
        assert c[0, i] == pytest.approx(sig * max(0.0, 1.0 - sd / eps) ** 2, rel=1e-15)
    # x = -0.25, 0, 0.25: one eps outside, on the perimeter, one eps inside
    assert c[0, 3] == 0.0 and c[0, 4] == sig and c[0, 5] == 4 * sig
    far = [(np.array(SQUARE) + 10.0, 0)]
    c2, _ = oracle.costmap([(SQUARE, 0)] + far, 21, 1, 0.25, -1.0, 1.0, eps, sig)
    np.testing.assert_allclose(c2, c, rtol=0, atol=0)  # the far obstacle adds nothing here
    both = [(SQUARE, 0), (SQUARE, 0)]
    c3, _ = oracle.costmap(both, 21, 1, 0.25, -1.0, 1.0, eps, sig)
    np.testing.assert_allclose(c3, 2 * c, rtol=1e-15)


def _winding(poly, x, y):
    """Winding number of a closed polygon around (x, y) (Sunday's crossing
    test with orientation signs): an inside test independent of the oracle's
    even-odd ray rule."""
    wn = 0
    n = len(poly)
    for k in range(n):
        (ax, ay), (bx, by) = poly[k], poly[(k + 1) % n]
        cross = (bx - ax) * (y - ay) - (x - ax) * (by - ay)
        if ay <= y < by and cross > 0:
            wn += 1
        elif by <= y < ay and cross < 0:
            wn -= 1
    return wn


# Points exactly at the height of vertices (where a ray passes through a
# vertex), for a diamond, a star with notches and a polygon with a horizontal
# edge, against the winding number.
def test_inside_rule_at_vertex_heights():
    star = [(math.cos(a) * (2.0 if k % 2 == 0 else 0.8), math.sin(a) * (2.0 if k % 2 == 0 else 0.8))
            for k, a in enumerate(np.linspace(0, 2 * np.pi, 10, endpoint=False))]
    shapes = [[(0, 1), (1, 0), (0, -1), (-1, 0)], star, [(0, 0), (3, 0), (3, 1), (2, 1), (2, 2), (0, 2)]]
    rng = np.random.default_rng(5)
    for poly in shapes:
        ys = sorted({float(p[1]) for p in poly})
        for _ in range(300):
            y = ys[rng.integers(len(ys))]
            x = rng.uniform(-3, 4)
            s = oracle.sdist(poly, 0, x, y)
            if abs(s) < 1e-9:
                continue                      # on the perimeter
            assert (s < 0) == (_winding(poly, x, y) != 0), (poly, x, y, s)
