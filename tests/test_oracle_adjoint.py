"""Pins of the oracle's warp energy and its gradient (oracle/adjoint.py).

  * FP64 central differences (h = 1e-6) of E reproduce the analytic gradient
    (a wrong lambda, a missing chain-rule factor, a sign or a swapped x/y all
    fail this);
  * identical images at u = 0 give E = 0 and a zero gradient;
  * summed over nodes the gradient equals the dense sum of r grad Te, since
    the barycentric coordinates of a pixel sum to 1;
  * E equals HW/2 times the MSD that register.Problem reports;
  * the spline Hessian matches central differences of the spline gradient;
  * the unrolled gradient dE(u_K)/du_0 matches central differences of the
    composed FP64 function (a dropped Hessian term, a transposed S or a
    wrong tau all fail it).
"""
import numpy as np
import pytest

from oracle import adjoint, bspline, register
from paper_1411_2141_gb300 import inputs


@pytest.fixture(scope="module")
def small_case():
    spec = inputs.CaseSpec(side=48, n_nodes=120, seed=11, n_blobs=8, dmax=2.0, n_iter=5)
    return inputs.make_case(spec)


def _problem(c):
    return register.Problem(c.V, c.T, c.Re, c.Te, 0.1, 1.0, "S0", "G1")


def _smooth_u(c, amp=0.7, seed=3):
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 1.5, size=4)
    x, y = c.V[:, 0].astype(np.float64), c.V[:, 1].astype(np.float64)
    s = c.spec.side
    return amp * np.stack([np.sin(2 * np.pi * k[0] * x / s + k[1]),
                           np.cos(2 * np.pi * k[2] * y / s + k[3])], axis=1)


def test_gradient_matches_central_differences(small_case):
    pb = _problem(small_case)
    u = _smooth_u(small_case)
    _, g = adjoint.warp_energy_grad(pb, u)
    rng = np.random.default_rng(0)
    h = 1e-6
    for a in rng.choice(pb.n, size=12, replace=False):
        for c in range(2):
            up = u.copy()
            um = u.copy()
            up[a, c] += h
            um[a, c] -= h
            fd = (adjoint.warp_energy(pb, up) - adjoint.warp_energy(pb, um)) / (2 * h)
            assert abs(fd - g[a, c]) <= 1e-6 * max(1.0, np.abs(g).max()), (a, c, fd, g[a, c])


def test_identical_images_give_zero(small_case):
    c = small_case
    pb = register.Problem(c.V, c.T, c.Re, c.Re, 0.1, 1.0, "S0", "G1")
    E, g = adjoint.warp_energy_grad(pb, np.zeros((pb.n, 2)))
    assert E < 1e-20 and np.abs(g).max() < 1e-10


def test_gradient_sum_is_dense_sum(small_case):
    pb = _problem(small_case)
    u = _smooth_u(small_case)
    _, g = adjoint.warp_energy_grad(pb, u)
    ud = pb.dense_displacement(u)
    ys, xs = np.mgrid[0:pb.H, 0:pb.W].astype(np.float64)
    val, gx, gy = bspline.evaluate(pb.cTe, xs + ud[..., 0], ys + ud[..., 1], grad=True)
    r = val - pb.Re
    np.testing.assert_allclose(g.sum(axis=0), [np.sum(r * gx), np.sum(r * gy)], rtol=1e-10,
                               atol=1e-10)


def test_energy_is_half_the_pixel_sum_of_the_msd(small_case):
    pb = _problem(small_case)
    u = _smooth_u(small_case)
    E, _ = adjoint.warp_energy_grad(pb, u)
    assert E == pytest.approx(0.5 * pb.H * pb.W * pb.msd(u), rel=1e-12)


def test_spline_hessian_matches_differences_of_the_gradient(small_case):
    pb = _problem(small_case)
    rng = np.random.default_rng(5)
    x = rng.uniform(-3, pb.W + 2, 40)
    y = rng.uniform(-3, pb.H + 2, 40)
    hxx, hxy, hyy = bspline.hessian(pb.cTe, x, y)
    h = 1e-5
    _, gxp, gyp = bspline.evaluate(pb.cTe, x + h, y, grad=True)
    _, gxm, gym = bspline.evaluate(pb.cTe, x - h, y, grad=True)
    _, gxq, _ = bspline.evaluate(pb.cTe, x, y + h, grad=True)
    _, gxr, _ = bspline.evaluate(pb.cTe, x, y - h, grad=True)
    _, _, gyq = bspline.evaluate(pb.cTe, x, y + h, grad=True)
    _, _, gyr = bspline.evaluate(pb.cTe, x, y - h, grad=True)
    # away from cell boundaries the second derivative is smooth
    ok = (np.abs(x - np.round(x)) > 2 * h) & (np.abs(y - np.round(y)) > 2 * h)
    sc = max(1.0, np.abs(hxx).max())
    np.testing.assert_allclose(hxx[ok], ((gxp - gxm) / (2 * h))[ok], atol=1e-6 * sc)
    np.testing.assert_allclose(hxy[ok], ((gyp - gym) / (2 * h))[ok], atol=1e-6 * sc)
    np.testing.assert_allclose(hxy[ok], ((gxq - gxr) / (2 * h))[ok], atol=1e-6 * sc)
    np.testing.assert_allclose(hyy[ok], ((gyq - gyr) / (2 * h))[ok], atol=1e-6 * sc)


@pytest.mark.parametrize("passes", [1, 3])
def test_unrolled_gradient_matches_central_differences(small_case, passes):
    c = small_case
    pb = register.Problem(c.V, c.T, c.Re, c.Te, 0.1, 1.0, "S0", "G1", smooth_passes=passes)
    u0 = _smooth_u(small_case, amp=0.5, seed=9)
    K = 5
    _, g = adjoint.unrolled_grad(pb, u0, K)
    rng = np.random.default_rng(2)
    h = 1e-6
    scale = max(1.0, np.abs(g).max())
    for a in rng.choice(pb.n, size=8, replace=False):
        for c in range(2):
            up = u0.copy()
            um = u0.copy()
            up[a, c] += h
            um[a, c] -= h
            fd = (adjoint.unrolled_energy(pb, up, K) - adjoint.unrolled_energy(pb, um, K)) / (2 * h)
            assert abs(fd - g[a, c]) <= 1e-6 * scale, (a, c, fd, g[a, c])


def test_unrolled_gradient_of_zero_iterations_is_the_warp_gradient(small_case):
    pb = _problem(small_case)
    u0 = _smooth_u(small_case, amp=0.5, seed=9)
    E0, g0 = adjoint.unrolled_grad(pb, u0, 0)
    E1, g1 = adjoint.warp_energy_grad(pb, u0)
    assert E0 == E1 and np.array_equal(g0, g1)
