"""Pins of the oracle's cubic B-spline (prefilter and evaluation).

Each test checks the oracle against a fact fixed outside it: a dense direct
solve of the interpolation conditions, hand-derived coefficients, the closed
form of the inverse filter, polynomial reproduction, central differences.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import bspline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mirror(k, n):
    p = 2 * n - 2
    k = abs(k) % p
    return p - k if k >= n else k


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 17, 33, 64])
def test_prefilter_solves_mirror_interpolation_system(n):
    rng = np.random.default_rng(n)
    s = rng.normal(size=n)
    B = np.zeros((n, n))
    for k in range(n):
        B[k, k] += 4.0 / 6.0
        B[k, _mirror(k - 1, n)] += 1.0 / 6.0
        B[k, _mirror(k + 1, n)] += 1.0 / 6.0
    c_ref = np.linalg.solve(B, s)
    c = bspline.prefilter_axis(s, 0)
    np.testing.assert_allclose(c, c_ref, rtol=0, atol=1e-12 * np.abs(c_ref).max())


def test_prefilter_hand_derived_cases():
    with open(os.path.join(GOLDEN, "bspline_small.json")) as fh:
        g = json.load(fh)
    for case in g["cases"]:
        c = bspline.prefilter_axis(np.array(case["s"], float), 0)
        np.testing.assert_allclose(c, case["c"], atol=1e-13)


def test_impulse_response_closed_form():
    n = 201
    s = np.zeros(n)
    s[100] = 1.0
    c = bspline.prefilter_axis(s, 0)
    k = np.arange(-40, 41)
    expect = math.sqrt(3.0) * bspline.Z1 ** np.abs(k)
    np.testing.assert_allclose(c[100 + k], expect, atol=1e-14)


def test_interpolation_reproduces_grid_values():
    rng = np.random.default_rng(1)
    img = rng.uniform(size=(13, 17))
    coef = bspline.prefilter_2d(img)
    ys, xs = np.mgrid[0:13, 0:17].astype(float)
    val = bspline.evaluate(coef, xs, ys)
    np.testing.assert_allclose(val, img, atol=1e-12)


def test_constant_image_has_constant_coefficients():
    img = np.full((9, 6), 0.375)
    np.testing.assert_allclose(bspline.prefilter_2d(img), 0.375, atol=1e-14)
    rng = np.random.default_rng(2)
    x = rng.uniform(-20, 30, size=50)
    y = rng.uniform(-20, 30, size=50)
    np.testing.assert_allclose(bspline.evaluate(bspline.prefilter_2d(img), x, y), 0.375, atol=1e-14)


def test_cubic_polynomials_reproduced_away_from_border():
    n = 64
    ys, xs = np.mgrid[0:n, 0:n].astype(float)

    def p(x, y):
        x = (x - 30.0) / 10.0
        y = (y - 31.0) / 10.0
        return 0.3 + x - 0.5 * y + 0.2 * x * y - 0.1 * x ** 3 + 0.07 * y ** 3 + 0.05 * x * x * y

    coef = bspline.prefilter_2d(p(xs, ys))
    rng = np.random.default_rng(3)
    x = rng.uniform(20, n - 21, size=200)
    y = rng.uniform(20, n - 21, size=200)
    np.testing.assert_allclose(bspline.evaluate(coef, x, y), p(x, y), atol=1e-9)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    img = rng.uniform(size=(20, 24))
    coef = bspline.prefilter_2d(img)
    x = rng.uniform(-3, 26, size=100)
    y = rng.uniform(-3, 22, size=100)
    v, gx, gy = bspline.evaluate(coef, x, y, grad=True)
    h = 1e-6
    fx = (bspline.evaluate(coef, x + h, y) - bspline.evaluate(coef, x - h, y)) / (2 * h)
    fy = (bspline.evaluate(coef, x, y + h) - bspline.evaluate(coef, x, y - h)) / (2 * h)
    np.testing.assert_allclose(gx, fx, atol=1e-7)
    np.testing.assert_allclose(gy, fy, atol=1e-7)
    np.testing.assert_allclose(v, bspline.evaluate(coef, x, y), atol=0)


def test_mirror_extension_outside_the_image():
    rng = np.random.default_rng(5)
    img = rng.uniform(size=(11, 14))
    coef = bspline.prefilter_2d(img)
    x = rng.uniform(0, 13, size=60)
    y = rng.uniform(0, 10, size=60)
    v = bspline.evaluate(coef, x, y)
    np.testing.assert_allclose(bspline.evaluate(coef, -x, y), v, atol=1e-12)
    np.testing.assert_allclose(bspline.evaluate(coef, x, -y), v, atol=1e-12)
    np.testing.assert_allclose(bspline.evaluate(coef, 2 * 13 - x, y), v, atol=1e-12)
    np.testing.assert_allclose(bspline.evaluate(coef, x, 2 * 10 - y), v, atol=1e-12)


def test_weights_values_and_partition_of_unity():
    w = bspline.cubic_weights(np.array(0.0))
    np.testing.assert_allclose([float(a) for a in w], [1 / 6, 4 / 6, 1 / 6, 0.0], atol=1e-15)
    t = np.linspace(0, 1, 33)[:-1]
    np.testing.assert_allclose(sum(bspline.cubic_weights(t)), 1.0, atol=1e-15)
    np.testing.assert_allclose(sum(bspline.cubic_dweights(t)), 0.0, atol=1e-15)
    # first moment: sum_k w_k (k - 1) = t  (linear reproduction)
    w = bspline.cubic_weights(t)
    np.testing.assert_allclose(sum(wk * (k - 1) for k, wk in enumerate(w)), t, atol=1e-15)


def test_mirror_index():
    n = 5
    got = bspline.mirror_index(np.arange(-9, 14), n)
    expect = [_mirror(k, n) for k in range(-9, 14)]
    assert list(got) == expect
    assert set(got) <= set(range(n))
