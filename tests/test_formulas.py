"""Identities the CUDA path relies on where it evaluates a formula in a form
other than the printed one, checked in FP64 against the oracle's form:

* Eq. 9 in edge-normal form: for node i of a triangle whose other corners
  j, k follow counter-clockwise, with e1 = V_j - V_i, e2 = V_k - V_i,
  df1 = f_j - f_i, df2 = f_k - f_i and A2 = e1 x e2,
      A_T grad f_T = 1/2 sgn(A2) (df1 e2y - df2 e1y, df2 e1x - df1 e2x),
  which the force phase sums over the incident triangles (Eq. 10's
  numerator) without forming 1 / (4 A^2);
* the P1 interpolant of u over a triangle (a, b, c) in affine form,
      u(x) = u_a + G (x - V_a),  G = [d_b d_c] [e1 e2]^-1,
  d = u - u_a, e = V - V_a, which the one-pair warp evaluates per pixel
  instead of the barycentric sum;
* the B-spline prefilter of a line as independent windows: each segment of
  64 outputs is filtered over a window of 16 more samples on each side of
  the line's mirror-symmetric extension, both recursions starting from a
  zero state -- against the exact mirror-boundary filter;
* the Chebyshev solve of S1: the spectrum of D^-1 A lies in
  [1/(1+l), (1+2l)/(1+l)], and k steps of the semi-iteration on that
  interval bring the residual below sqrt(m_max/m_min) |r_0| / T_k(theta/delta),
  the bound the step count is taken from.
"""
import math

import numpy as np
import scipy.sparse as sp

from oracle import bspline, mesh


def _random_triangles(rng, n):
    P = rng.uniform(-20.0, 20.0, size=(3 * n, 2))
    T = np.arange(3 * n).reshape(n, 3)
    a = P[T]
    area2 = ((a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1])
             - (a[:, 1, 1] - a[:, 0, 1]) * (a[:, 2, 0] - a[:, 0, 0]))
    keep = np.abs(area2) > 1.0
    return P, T[keep]


def test_eq9_edge_normal_form_equals_the_printed_form():
    rng = np.random.default_rng(7)
    P, T = _random_triangles(rng, 400)
    f = rng.normal(size=len(P))
    grad, A = mesh.triangle_gradient_eq9(P, f, T)
    for corner in range(3):   # the node i may be any corner; j, k follow it cyclically
        i, j, k = T[:, corner], T[:, (corner + 1) % 3], T[:, (corner + 2) % 3]
        e1, e2 = P[j] - P[i], P[k] - P[i]
        df1, df2 = f[j] - f[i], f[k] - f[i]
        A2 = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
        h = np.where(A2 > 0, 0.5, -0.5)
        n = np.stack([h * (df1 * e2[:, 1] - df2 * e1[:, 1]), h * (df2 * e1[:, 0] - df1 * e2[:, 0])], 1)
        np.testing.assert_allclose(n, A[:, None] * grad, rtol=1e-9, atol=1e-9 * np.abs(n).max())
        np.testing.assert_allclose(0.5 * np.abs(A2), A, rtol=1e-12)


def test_affine_form_of_the_p1_interpolant():
    rng = np.random.default_rng(8)
    P, T = _random_triangles(rng, 300)
    u = rng.normal(scale=3.0, size=(len(P), 2))
    for t in T:
        a, b, c = t
        e1, e2 = P[b] - P[a], P[c] - P[a]
        E = np.stack([e1, e2], 1)                       # columns e1, e2
        D = np.stack([u[b] - u[a], u[c] - u[a]], 1)     # columns d_b, d_c
        G = D @ np.linalg.inv(E)
        # random points inside (and on the edges of) the triangle
        w = rng.dirichlet(np.ones(3), size=8)
        w[0] = (1.0, 0.0, 0.0)
        w[1] = (0.0, 0.5, 0.5)
        x = w @ P[t]
        bary = w @ u[t]                                  # sum_a lambda_a(x) u_a
        aff = u[a] + (x - P[a]) @ G.T
        np.testing.assert_allclose(aff, bary, rtol=1e-10, atol=1e-10)


def _windowed_prefilter_line(s, seg=64, warm=16):
    """The kernels' windowed form, restated in FP64."""
    z = math.sqrt(3.0) - 2.0
    n = len(s)
    p = 2 * n - 2

    def fold(j):
        j %= p
        return j if j < n else p - j

    out = np.empty(n)
    win = seg + 2 * warm
    for s0 in range(0, n, seg):
        v = np.array([6.0 * s[fold(s0 - warm + k)] for k in range(win)])
        for k in range(1, win):
            v[k] += z * v[k - 1]
        v[win - 1] = z * (0.0 - v[win - 1])
        for k in range(win - 2, warm - 1, -1):
            v[k] = z * (v[k + 1] - v[k])
        m = min(seg, n - s0)
        out[s0:s0 + m] = v[warm:warm + m]
    return out


def test_windowed_prefilter_equals_the_exact_mirror_boundary_filter():
    rng = np.random.default_rng(5)
    for n in (2, 3, 5, 17, 63, 64, 65, 97, 130, 300):
        s = rng.uniform(-1.0, 1.0, size=n)
        ref = bspline.prefilter_axis(s[None, :], axis=1)[0]
        got = _windowed_prefilter_line(s)
        # the zero states cost |z1|^16 ~ 7e-10 of the samples, amplified by
        # at most the recursions' gains
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(s).max(), n


def _grid_mesh(n):
    g = np.arange(n + 1, dtype=np.float64)
    V = np.array([(x, y) for y in g for x in g])
    T = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            T += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.array(T)


def test_chebyshev_interval_and_step_bound_for_the_umbrella_system():
    lam = 0.1
    V, T = _grid_mesh(7)
    rng = np.random.default_rng(8)
    V = V + rng.uniform(-0.2, 0.2, size=V.shape)
    n = len(V)
    W = mesh.adjacency(T, n).tocsr()
    m = np.asarray(W.sum(axis=1)).ravel()
    A = ((1.0 + lam) * sp.diags(m) - lam * W).tocsr()
    Dinv = 1.0 / ((1.0 + lam) * m)
    ev = np.linalg.eigvals((sp.diags(Dinv) @ A).toarray()).real
    lo, hi = 1.0 / (1.0 + lam), (1.0 + 2.0 * lam) / (1.0 + lam)
    assert ev.min() >= lo - 1e-12 and ev.max() <= hi + 1e-12
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    b = rng.normal(size=n)
    x = rng.normal(size=n)
    r0 = np.linalg.norm(b - A @ x)
    # the three-term Chebyshev semi-iteration on [lo, hi] (Saad, Sec. 12.3)
    sigma = theta / delta
    rho = 1.0 / sigma
    d = Dinv * (b - A @ x) / theta
    for k in range(1, 7):
        x = x + d
        r = b - A @ x
        bound = math.sqrt(m.max() / m.min()) * r0 / math.cosh(k * math.acosh(sigma))
        assert np.linalg.norm(r) <= bound * (1.0 + 1e-9), k
        rn = 1.0 / (2.0 * sigma - rho)
        d = rn * rho * d + 2.0 * rn / delta * (Dinv * r)
        rho = rn
