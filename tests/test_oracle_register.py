"""Pins of the oracle's iteration (Algorithm 1) and of its warp / MSD."""
import numpy as np
import pytest

from oracle import mesh, register
from paper_1411_2141_gb300 import inputs

MODES = [("S0", "G0", "Q0"), ("S0", "G1", "Q0"), ("S1", "G0", "Q0"), ("S1", "G1", "Q0"),
         ("S2", "G0", "Q0"), ("S2", "G1", "Q0"), ("S2", "G1", "Q1")]


@pytest.fixture(scope="module")
def small():
    return inputs.make_case(inputs.CaseSpec(side=48, n_nodes=220, seed=11, dmax=2.0))


@pytest.mark.parametrize("mode,grad,quad", MODES)
def test_zero_force_on_identical_images(small, mode, grad, quad):
    pb = register.Problem(small.V, small.T, small.Re, small.Re, 0.1, 1.0, mode, grad, quad)
    u = np.zeros((pb.n, 2))
    f, r, g = pb.sample(u)
    assert np.abs(r).max() == 0.0
    F = pb.force(u, f, r, g)
    assert np.abs(F).max() == 0.0
    u1, _ = pb.step(u)
    assert np.abs(u1).max() < 1e-14


@pytest.mark.parametrize("mode,quad", [("S0", "Q0"), ("S2", "Q0"), ("S2", "Q1")])
def test_g1_force_is_gradient_of_data_energy(small, mode, quad):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, mode, "G1", quad)
    rng = np.random.default_rng(0)
    u = rng.uniform(-0.5, 0.5, size=(pb.n, 2))
    f, r, g = pb.sample(u)
    F = pb.force(u, f, r, g)
    h = 1e-6
    for i in rng.choice(pb.n, size=12, replace=False):
        for d in range(2):
            up = u.copy()
            um = u.copy()
            up[i, d] += h
            um[i, d] -= h
            fd = (pb.data_energy(up) - pb.data_energy(um)) / (2 * h)
            assert abs(fd - F[i, d]) <= 1e-6 * max(1.0, abs(F[i, d])), (i, d, fd, F[i, d])


@pytest.mark.parametrize("mode,grad,quad", MODES)
def test_linear_ramp_closed_form_trajectory(small, mode, grad, quad):
    """Te(x) = a.x + b0 and Re(x) = a.x + c: every node sees r = a.u + b0 - c
    and grad = a, so u stays uniform and r_k = (1 - tau |a|^2)^k r_0."""
    a = np.array([0.3, -0.2])
    b0, c, tau = 0.9, 0.4, 1.0

    def te(x, y):
        return a[0] * x + a[1] * y + b0, np.full_like(x, a[0]), np.full_like(x, a[1])

    def re(x, y):
        return a[0] * x + a[1] * y + c

    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, tau, mode, grad, quad,
                          te_sampler=te, re_sampler=re)
    n = 10
    u, _ = pb.run(n)
    r0 = b0 - c
    rn = (1 - tau * a @ a) ** n * r0
    expect = -(r0 - rn) * a / (a @ a)
    np.testing.assert_allclose(u, np.broadcast_to(expect, u.shape), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("quad", ["Q0", "Q1"])
def test_energy_decreases_for_fem_form(small, quad):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, "S2", "G1", quad)
    u = np.zeros((pb.n, 2))
    e_prev = pb.total_energy(u)
    for _ in range(25):
        u, _ = pb.step(u)
        e = pb.total_energy(u)
        assert e < e_prev
        e_prev = e


@pytest.mark.parametrize("mode,grad,quad", MODES)
def test_msd_decreases_on_phantom(case0, mode, grad, quad):
    pb = register.Problem(case0.V, case0.T, case0.Re, case0.Te, 0.1, 1.0, mode, grad, quad)
    u, _ = pb.run(20)
    assert pb.msd(u) < pb.msd(np.zeros_like(u))


@pytest.mark.parametrize("mode", ["S1", "S2"])
def test_solve_satisfies_the_linear_system(small, mode):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, mode, "G1", "Q0")
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, (pb.n, 2))
    F = rng.uniform(-1, 1, (pb.n, 2))
    u1 = pb.update(u, F)
    if mode == "S1":
        A = (1 + pb.lam) * np.diag(pb.m) - pb.lam * pb.Wadj.toarray()
        rhs = pb.m[:, None] * (u - pb.tau * F)
    else:
        M, K = mesh.p1_mass_stiffness(pb.V, pb.T)
        A = (M + pb.lam * K).toarray()
        rhs = M @ u - pb.tau * F
    np.testing.assert_allclose(A @ u1, rhs, atol=1e-11 * np.abs(rhs).max())


def test_warp_with_zero_displacement_is_the_template(small):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0)
    u = np.zeros((pb.n, 2))
    np.testing.assert_allclose(pb.warp(u), small.Te, atol=1e-11)
    np.testing.assert_allclose(pb.msd(u), np.mean((small.Te.astype(float) - small.Re) ** 2), rtol=1e-12)


def test_warp_by_integer_shift_reads_shifted_pixels(small):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0)
    u = np.tile([[2.0, 1.0]], (pb.n, 1))
    R = pb.warp(u)
    np.testing.assert_allclose(R[:-1, :-2], small.Te[1:, 2:], atol=1e-11)


def test_p1_interpolation_reproduces_affine_fields(small):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0)
    B = np.array([[0.01, -0.02], [0.03, 0.005]])
    t = np.array([0.4, -0.7])
    u = pb.V @ B.T + t
    ud = pb.dense_displacement(u)
    ys, xs = np.mgrid[0:pb.H, 0:pb.W].astype(float)
    X = np.stack([xs, ys], -1)
    np.testing.assert_allclose(ud, X @ B.T + t, atol=1e-12)
    ud = pb.dense_displacement(np.tile(t, (pb.n, 1)))
    np.testing.assert_allclose(ud, np.broadcast_to(t, ud.shape), atol=1e-14)


def test_point_location_against_exhaustive_search(small):
    P = small.V.astype(np.float64)
    T = small.T.astype(np.int64)
    H, W = small.Re.shape
    owner = register.locate_pixels(P, T, W, H, chunk=37)
    assert (owner >= 0).all()
    for y in range(0, H, 3):
        for x in range(W):
            px = np.full(len(T), float(x))
            py = np.full(len(T), float(y))
            a, b, c = T[:, 0], T[:, 1], T[:, 2]
            inside = ((register.edge_side(P, a, b, px, py) >= 0)
                      & (register.edge_side(P, b, c, px, py) >= 0)
                      & (register.edge_side(P, c, a, px, py) >= 0))
            assert owner[y, x] == np.flatnonzero(inside).min()
    # the owner really contains the pixel: barycentric coordinates are >= 0
    # and reproduce the pixel position
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    tri = T[owner.ravel()]
    lam_pos = register.interpolate_p1(P, T, owner, P, W, H)
    np.testing.assert_allclose(lam_pos[..., 0], xs, atol=1e-10)
    np.testing.assert_allclose(lam_pos[..., 1], ys, atol=1e-10)
    assert tri.shape[0] == H * W


def test_generated_meshes_cover_the_image(case0):
    owner = register.locate_pixels(case0.V, case0.T, 128, 128)
    assert (owner >= 0).all()
    A = mesh.signed_area(case0.V.astype(float), case0.T)
    assert A.min() > 0
    np.testing.assert_allclose(A.sum(), 127.0 * 127.0, rtol=1e-12)


@pytest.mark.parametrize("passes", [2, 5])
def test_repeated_smoothing_keeps_uniform_fields_and_the_valence_weighted_sum(small, passes):
    """Eq. 14 applied several times: A^Lap = D_m^-1 W with W symmetric, so each
    pass keeps sum_i m_i u_i (and any uniform field); with no force the
    update is exactly `passes` smoothing passes."""
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, "S0", "G1",
                          lam=0.8, smooth_passes=passes)
    rng = np.random.default_rng(1)
    u = rng.normal(size=(pb.n, 2))
    out = pb.update(u, np.zeros_like(u))
    np.testing.assert_allclose(pb.m @ out, pb.m @ u, rtol=1e-12)
    one = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, "S0", "G1", lam=0.8)
    ref = u
    for _ in range(passes):
        ref = one.update(ref, np.zeros_like(u))
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    uniform = np.broadcast_to([0.7, -0.3], u.shape)
    np.testing.assert_allclose(pb.update(uniform, np.zeros_like(u)), uniform, atol=1e-12)
    # smoothing is a contraction of the non-uniform part
    dev = lambda v: v - (pb.m @ v) / pb.m.sum()   # noqa: E731
    assert np.linalg.norm(dev(out)) < np.linalg.norm(dev(u))


def test_repeated_smoothing_is_explicit_only(small):
    with pytest.raises(ValueError):
        register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, "S1", "G0",
                         smooth_passes=2)


@pytest.mark.parametrize("passes", [1, 3])
def test_ramp_trajectory_with_repeated_smoothing(small, passes):
    """Uniform fields are fixed by every pass, so the closed-form ramp
    trajectory holds for any number of passes."""
    a = np.array([0.3, -0.2])
    b0, c, tau = 0.9, 0.4, 1.0

    def te(x, y):
        return a[0] * x + a[1] * y + b0, np.full_like(x, a[0]), np.full_like(x, a[1])

    def re(x, y):
        return a[0] * x + a[1] * y + c

    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, tau, "S0", "G0",
                          te_sampler=te, re_sampler=re, smooth_passes=passes)
    n = 10
    u, _ = pb.run(n)
    r0 = b0 - c
    rn = (1 - tau * a @ a) ** n * r0
    np.testing.assert_allclose(u, np.broadcast_to(-(r0 - rn) * a / (a @ a), u.shape), rtol=1e-9,
                               atol=1e-11)


@pytest.mark.parametrize("mode", ["S0", "S1", "S2"])
def test_smoothness_is_a_nonnegative_quadratic_vanishing_on_uniform_fields(small, mode):
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 1.0, mode, "G1")
    rng = np.random.default_rng(4)
    for _ in range(3):
        assert pb.smoothness(rng.normal(size=(pb.n, 2))) > 0.0
    assert abs(pb.smoothness(np.broadcast_to([1.3, -0.4], (pb.n, 2)))) < 1e-9
    # gradient by central differences equals L u (a symmetric quadratic form)
    u = rng.normal(size=(pb.n, 2))
    L = pb.K if mode == "S2" else (np.diag(pb.m) - pb.Wadj.toarray())
    g = (L @ u) if mode != "S2" else (pb.K @ u)
    h = 1e-6
    for a in rng.choice(pb.n, size=5, replace=False):
        up, um = u.copy(), u.copy()
        up[a, 0] += h
        um[a, 0] -= h
        fd = (pb.smoothness(up) - pb.smoothness(um)) / (2 * h)
        assert abs(fd - g[a, 0]) <= 1e-6 * max(1.0, abs(g[a, 0]))


def test_total_energy_decreases_for_the_umbrella_form(small):
    """S1 takes an explicit Euclidean step on D and an implicit step on
    alpha S in the D_m^-1 metric, so it is not an exact gradient flow of
    D + alpha S; for a small step (tau = 0.1) the total energy still
    decreases on this pair (with tau = 0.5 it does not)."""
    pb = register.Problem(small.V, small.T, small.Re, small.Te, 0.1, 0.1, "S1", "G1")
    u = np.zeros((pb.n, 2))
    e_prev = pb.total_energy(u)
    for _ in range(25):
        u, _ = pb.step(u)
        e = pb.total_energy(u)
        assert e < e_prev
        e_prev = e


def _exact_orient(ax, ay, bx, by, px, py):
    """Orientation of p against a -> b in exact rational arithmetic (every
    float is a dyadic rational, so Fraction holds it exactly)."""
    from fractions import Fraction as Fr
    ax, ay, bx, by, px, py = (Fr(float(v)) for v in (ax, ay, bx, by, px, py))
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax)


def test_point_location_exact_on_an_integer_mesh():
    """An independent pin of the owner rule (smallest index among the closed
    triangles that contain the pixel centre): a Delaunay mesh whose nodes all
    sit on pixel centres, so that many pixel centres lie exactly on edges and
    at vertices, located by exact integer orientation tests and compared with
    locate_pixels."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(5)
    W, H = 23, 17
    border = [(x, 0) for x in range(0, W, 4)] + [(x, H - 1) for x in range(0, W, 4)] \
        + [(0, y) for y in range(0, H, 4)] + [(W - 1, y) for y in range(0, H, 4)] \
        + [(W - 1, H - 1)]
    inner = {(int(x), int(y)) for x, y in zip(rng.integers(1, W - 1, 40), rng.integers(1, H - 1, 40))}
    P = np.array(sorted(set(border) | inner), dtype=np.int64)
    T = Delaunay(P.astype(float)).simplices.astype(np.int64)
    A2 = ((P[T[:, 1], 0] - P[T[:, 0], 0]) * (P[T[:, 2], 1] - P[T[:, 0], 1])
          - (P[T[:, 1], 1] - P[T[:, 0], 1]) * (P[T[:, 2], 0] - P[T[:, 0], 0]))
    T[A2 < 0] = T[A2 < 0][:, [0, 2, 1]]   # counter-clockwise
    T = T[A2 != 0]
    owner = register.locate_pixels(P.astype(np.float64), T, W, H)
    on_edge = 0
    for y in range(H):
        for x in range(W):
            best = -1
            for t, (a, b, c) in enumerate(T):
                o = [(P[j, 0] - P[i, 0]) * (y - P[i, 1]) - (P[j, 1] - P[i, 1]) * (x - P[i, 0])
                     for i, j in ((a, b), (b, c), (c, a))]   # exact in int64
                if min(o) >= 0:
                    on_edge += min(o) == 0
                    best = t
                    break
            assert owner[y, x] == best, (x, y)
    assert on_edge > 50   # the tie rule was really exercised


def test_point_location_owner_contains_the_pixel_exactly(small):
    """On a generated mesh (float coordinates), the owner of every pixel
    contains the pixel centre in exact rational arithmetic: its three exact
    orientations (the barycentric coordinates times twice its area) are >= 0
    and sum to twice its area."""
    P = small.V.astype(np.float64)
    T = small.T.astype(np.int64)
    H, W = small.Re.shape
    owner = register.locate_pixels(P, T, W, H)
    for y in range(0, H, 2):
        for x in range(0, W, 2):
            a, b, c = T[owner[y, x]]
            o = [_exact_orient(P[i, 0], P[i, 1], P[j, 0], P[j, 1], x, y)
                 for i, j in ((b, c), (c, a), (a, b))]
            area2 = _exact_orient(P[a, 0], P[a, 1], P[b, 0], P[b, 1], P[c, 0], P[c, 1])
            assert min(o) >= 0, (x, y)
            assert sum(o) == area2
