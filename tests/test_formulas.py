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
  instead of the barycentric sum.
"""
import numpy as np

from oracle import mesh


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
