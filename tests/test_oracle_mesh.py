"""Pins of the oracle's mesh operators (Eq. 9-14 and the P1 matrices)."""
import json
import os

import numpy as np
import pytest

from oracle import mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def two():
    with open(os.path.join(GOLDEN, "two_triangle.json")) as fh:
        g = json.load(fh)
    g["P"] = np.array(g["nodes"], float)
    g["T"] = np.array(g["tris"], np.int64)
    return g


def _random_mesh(seed, n=60, side=20.0):
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    pts = np.vstack([[0, 0], [side, 0], [side, side], [0, side], rng.uniform(1, side - 1, (n, 2))])
    T = Delaunay(pts).simplices.astype(np.int64)
    A = mesh.signed_area(pts, T)
    T[A < 0] = T[A < 0][:, [0, 2, 1]]
    return pts, T


def test_eq9_exact_for_linear_functions():
    rng = np.random.default_rng(0)
    P = rng.uniform(-50, 50, size=(3000, 2))
    T = np.arange(3000).reshape(1000, 3)
    a = np.array([0.7, -1.3])
    f = P @ a + 0.25
    g, A = mesh.triangle_gradient_eq9(P, f, T)
    ok = A > 1.0
    np.testing.assert_allclose(g[ok], np.broadcast_to(a, g[ok].shape), rtol=1e-8, atol=1e-8)


def test_eq9_orientation_free_and_matches_hat_gradients():
    rng = np.random.default_rng(1)
    P = rng.uniform(0, 10, size=(300, 2))
    T = np.arange(300).reshape(100, 3)
    f = rng.normal(size=300)
    g, A = mesh.triangle_gradient_eq9(P, f, T)
    g_flip, _ = mesh.triangle_gradient_eq9(P, f, T[:, [0, 2, 1]])
    np.testing.assert_allclose(g, g_flip, rtol=1e-9, atol=1e-9)
    hat, _ = mesh.p1_gradients(P, T)
    g_hat = np.einsum("ta,tad->td", f[T], hat)
    ok = A > 0.5
    np.testing.assert_allclose(g[ok], g_hat[ok], rtol=1e-7, atol=1e-7)


def test_hat_gradients_interpolate_corner_values():
    rng = np.random.default_rng(2)
    P = rng.uniform(0, 10, size=(300, 2))
    T = np.arange(300).reshape(100, 3)
    hat, A = mesh.p1_gradients(P, T)
    X = P[T]
    ok = A > 0.5
    for a in range(3):
        for b in range(3):
            # phi_a(V_b) - phi_a(V_a) = grad phi_a . (V_b - V_a) = delta_ab - 1
            d = np.sum(hat[:, a] * (X[:, b] - X[:, a]), axis=1)
            np.testing.assert_allclose(d[ok], (1.0 if a == b else 0.0) - 1.0, atol=1e-8)


def test_eq10_exact_for_linear_functions_on_deformed_mesh():
    P, T = _random_mesh(3)
    rng = np.random.default_rng(3)
    Pd = P + rng.uniform(-0.2, 0.2, P.shape)
    a = np.array([-0.4, 2.0])
    for X in (P, Pd):
        g = mesh.node_gradient_eq10(X, X @ a - 3.0, T, area_floor=1e-12)
        np.testing.assert_allclose(g, np.broadcast_to(a, g.shape), rtol=1e-9, atol=1e-9)


def test_eq10_degenerate_triangle_has_zero_weight():
    P = np.array([[0, 0], [1, 0], [0, 1], [2, 0]], float)   # (0,1,3) is collinear
    T = np.array([[0, 1, 2], [0, 1, 3]])
    f = np.array([0.0, 1.0, 2.0, 7.0])
    g = mesh.node_gradient_eq10(P, f, T, area_floor=1e-12)
    np.testing.assert_allclose(g[0], [1.0, 2.0])
    np.testing.assert_allclose(g[3], [0.0, 0.0])


def test_two_triangle_closed_forms(two):
    P, T = two["P"], two["T"]
    assert list(mesh.valence(T, 4)) == two["valence"]
    g, A = mesh.triangle_gradient_eq9(P, np.array(two["f_linear_x"], float), T)
    np.testing.assert_allclose(g, two["eq9_grad_linear_x"], atol=1e-15)
    np.testing.assert_allclose(A, [0.5, 0.5])
    g, _ = mesh.triangle_gradient_eq9(P, np.array(two["f_nonlinear"], float), T)
    np.testing.assert_allclose(g, two["eq9_grad_nonlinear"], atol=1e-15)
    gn = mesh.node_gradient_eq10(P, np.array(two["f_nonlinear"], float), T, 1e-12)
    np.testing.assert_allclose(gn, two["eq10_node_grad_nonlinear"], atol=1e-15)
    M, K = mesh.p1_mass_stiffness(P, T)
    np.testing.assert_allclose(K.toarray(), two["K"], atol=1e-14)
    np.testing.assert_allclose(24.0 * M.toarray(), two["M_times_24"], atol=1e-13)


def test_two_triangle_update_forms(two):
    from oracle import register
    P, T = two["P"], two["T"]
    lam = two["smoothing_lambda"]
    img = np.zeros((2, 2), np.float32)
    u0 = np.array(two["smoothing_u0"], float)
    zero = np.zeros_like(u0)
    pb = register.Problem(P, T, img, img, alpha=0.1, tau=1.0, mode="S0", lam=lam)
    np.testing.assert_allclose(pb.update(u0, zero), two["smoothing_u1"], atol=1e-15)
    pb = register.Problem(P, T, img, img, alpha=0.1, tau=1.0, mode="S1", lam=lam)
    np.testing.assert_allclose(pb.Asys.toarray(), two["s1_matrix_lambda_quarter"], atol=1e-15)
    u1 = pb.update(u0, zero)
    A = np.array(two["s1_matrix_lambda_quarter"])
    np.testing.assert_allclose(A @ u1, np.array(two["valence"])[:, None] * u0, atol=1e-14)


def test_operator_invariants():
    P, T = _random_mesh(4, n=80, side=30.0)
    n = len(P)
    W = mesh.adjacency(T, n)
    m = mesh.valence(T, n)
    Alap = mesh.umbrella_matrix(T, n)
    np.testing.assert_allclose(np.asarray(Alap.sum(axis=1)).ravel(), 1.0, atol=1e-14)
    assert (W != W.T).nnz == 0
    np.testing.assert_allclose(np.asarray((np.diag(m) - W.toarray()).sum(axis=1)).ravel(), 0, atol=1e-12)
    M, K = mesh.p1_mass_stiffness(P, T)
    np.testing.assert_allclose(np.asarray(K.sum(axis=1)).ravel(), 0.0, atol=1e-12)
    np.testing.assert_allclose(M.sum(), 30.0 * 30.0, rtol=1e-12)
    np.testing.assert_allclose((K - K.T).toarray(), 0, atol=1e-12)
    assert np.linalg.eigvalsh(K.toarray()).min() > -1e-10
    assert np.linalg.eigvalsh(M.toarray()).min() > 0
    np.testing.assert_allclose(mesh.lumped_area(P, T), np.asarray(M.sum(axis=1)).ravel(), rtol=1e-12)
    # S0 smoothing (Eq. 14) keeps a uniform field
    u = np.tile([[0.3, -1.2]], (n, 1))
    np.testing.assert_allclose(Alap @ u, u, atol=1e-14)


def test_incident_triangles_brute_force():
    P, T = _random_mesh(5, n=30)
    inc = mesh.incident_triangles(T, len(P))
    for v in range(len(P)):
        expect = [t for t in range(len(T)) if v in T[t]]
        assert list(inc[v]) == expect
