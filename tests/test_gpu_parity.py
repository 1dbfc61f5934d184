"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances
  * end to end (the accuracy target of the FP32 form): node displacements
    within 1e-4 px and MSD within 1e-5 relative of the oracle;
  * per step, from FP32 arithmetic: the prefilter is a stable recursion whose
    2-D gain is at most 9 (3 per pass), so coefficients agree to a few FP32
    ulps of the largest value (tolerance 5e-6 relative to max |c|); a spline
    sample sums 16 taps with weights summing to 1 (5e-6 of max |c|); the
    pixel -> triangle map is index work, compared bit for bit;
  * force: the mesh gradient divides value differences of neighbouring
    samples by edge lengths of a few px, so its absolute error is a few
    sample ulps per px (tolerance 2e-5 relative to max |F|).
"""
import numpy as np
import pytest

from oracle import bspline, register
from paper_1411_2141_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U_TOL = 1e-4       # px
MSD_RTOL = 1e-5
MODES = [("S0", "G0", "Q0"), ("S0", "G1", "Q0"), ("S1", "G0", "Q0"), ("S1", "G1", "Q0"),
         ("S2", "G0", "Q0"), ("S2", "G1", "Q0"), ("S2", "G1", "Q1")]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_2141_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def mreg():
    from paper_1411_2141_gb300 import mreg as m
    m.load()
    return m


@pytest.fixture(scope="module")
def c0():
    return inputs.make_case(inputs.config_spec(0))


@pytest.fixture(scope="module")
def c1():
    return inputs.make_case(inputs.config_spec(1))


def _reg(mreg, case, mode="S0", grad="G0", quad="Q0", **kw):
    return mreg.Registration(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                             mode=mode, grad=grad, quad=quad, **kw)


def _oracle(case, mode="S0", grad="G0", quad="Q0"):
    return register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                            mode, grad, quad)


def _ragged_case(H, W, seed):
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    Re = (np.sin(xs / 3.1 + 0.3) * np.cos(ys / 4.3) + 0.1 * rng.normal(size=(H, W))).astype(np.float32)
    Te = (np.sin((xs + 0.7) / 3.1 + 0.3) * np.cos((ys - 0.4) / 4.3)
          + 0.1 * rng.normal(size=(H, W))).astype(np.float32)
    n = max(4, min(300, (H * W) // 12))
    V, T = inputs.make_mesh(Te, n, seed)
    spec = inputs.CaseSpec(side=max(H, W), n_nodes=len(V), seed=seed)
    return inputs.Case(spec=spec, Re=Re, Te=Te, V=V, T=T, d=np.zeros((H, W, 2)))


RAGGED = [(2, 2), (3, 7), (37, 53), (5, 200), (200, 5), (64, 65), (24, 25), (130, 70), (300, 17)]


@pytest.mark.parametrize("hw", RAGGED)
def test_prefilter_and_node_samples(mreg, hw):
    case = _ragged_case(*hw, seed=hw[0] * 1000 + hw[1])
    with _reg(mreg, case) as r:
        for field, img in ((mreg.MREG_FIELD_COEF_RE, case.Re), (mreg.MREG_FIELD_COEF_TE, case.Te)):
            got = r.get_field(field)
            ref = bspline.prefilter_2d(img)
            tol = 5e-6 * np.abs(ref).max()
            err = np.abs(got - ref).max()
            assert err <= tol, (hw, field, err, tol)
        pb = _oracle(case)
        got = r.get_field(mreg.MREG_FIELD_RE_NODES)
        tol = 5e-6 * np.abs(pb.cRe).max()
        assert np.abs(got - pb.ReV).max() <= tol


def test_prefilter_config0(mreg, c0):
    with _reg(mreg, c0) as r:
        got = r.get_field(mreg.MREG_FIELD_COEF_TE)
    ref = bspline.prefilter_2d(c0.Te)
    assert np.abs(got - ref).max() <= 5e-6 * np.abs(ref).max()


def _grid_case(n=8, h=4, seed=3):
    """A mesh with every node on a pixel centre: the grid lines and the
    diagonals of its triangles pass through pixel centres, so many centres
    lie on edges and corners shared by several closed triangles."""
    side = n * h + 1
    g = np.arange(n + 1) * h
    V = np.array([(x, y) for y in g for x in g], np.float32)
    T = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            b, c = a + 1, a + n + 1
            d = c + 1
            T += [(a, b, d), (a, d, c)] if (i + j) % 2 == 0 else [(a, b, c), (b, d, c)]
    rng = np.random.default_rng(seed)
    Re = rng.normal(size=(side, side)).astype(np.float32)
    Te = rng.normal(size=(side, side)).astype(np.float32)
    spec = inputs.CaseSpec(side=side, n_nodes=len(V), seed=seed)
    return inputs.Case(spec=spec, Re=Re, Te=Te, V=V, T=np.array(T, np.int32),
                       d=np.zeros((side, side, 2)))


@pytest.mark.parametrize("which", ["c0", (37, 53), (130, 70), (2, 2), "grid"])
def test_pixel_map_bit_exact(mreg, c0, which):
    """The owner of every pixel centre, against the oracle's exhaustive
    search: the smallest-index closed triangle that contains it (the grid
    mesh puts centres on shared edges and corners)."""
    if which == "c0":
        case = c0
    elif which == "grid":
        case = _grid_case()
    else:
        case = _ragged_case(*which, seed=7)
    with _reg(mreg, case) as r:
        got = r.get_field(mreg.MREG_FIELD_PIXEL_TRI)
    H, W = case.Re.shape
    ref = register.locate_pixels(case.V, case.T, W, H)
    assert (ref >= 0).all()
    assert np.array_equal(got, ref.astype(np.int32))


@pytest.mark.parametrize("mode,grad,quad", MODES)
def test_first_iteration_fields(mreg, c0, mode, grad, quad):
    pb = _oracle(c0, mode, grad, quad)
    u0 = np.zeros((pb.n, 2))
    f, rr, g = pb.sample(u0)
    F = pb.force(u0, f, rr, g)
    u1 = pb.update(u0, F)
    f1, _, _ = pb.sample(u1)   # TE_NODES describes the current u after the step
    with _reg(mreg, c0, mode, grad, quad) as r:
        assert r.stats()["engine"] == mreg.MREG_ENGINE_GRID
        r.step(1)
        got_f = r.get_field(mreg.MREG_FIELD_TE_NODES)
        got_F = r.get_field(mreg.MREG_FIELD_FORCE)
        got_u = r.get_u()
        e = r.get_field(mreg.MREG_FIELD_ENERGY)
        r.stats()
    if quad != "Q1":
        assert np.abs(got_f - f1).max() <= 5e-6 * np.abs(pb.cTe).max()
    assert np.abs(got_F - F).max() <= 2e-5 * np.abs(F).max()
    assert np.abs(got_u - u1).max() <= 1e-6
    assert abs(e[0] - pb.data_energy(u0)) <= 1e-5 * pb.data_energy(u0)


@pytest.mark.parametrize("mode,grad,quad", MODES)
def test_registration_config0(mreg, c0, mode, grad, quad):
    n = c0.spec.n_iter
    pb = _oracle(c0, mode, grad, quad)
    u_ref, e_ref = pb.run(n)
    with _reg(mreg, c0, mode, grad, quad) as r:
        r.step(n)
        u = r.get_u()
        msd = r.msd()
        e = r.get_field(mreg.MREG_FIELD_ENERGY)
        st = r.stats()
        if mode != "S0":
            its = r.get_field(mreg.MREG_FIELD_PCG_ITERS)
            res = r.get_field(mreg.MREG_FIELD_PCG_RESID)
            assert (its > 0).all() and (res <= 1e-7).all()
    msd_ref = pb.msd(u_ref)
    du = np.abs(u - u_ref).max()
    dm = abs(msd - msd_ref) / msd_ref
    print(f"{mode}{grad}{quad}: du={du:.2e} dmsd={dm:.2e} its={st['max_pcg_iters']}")
    assert du <= U_TOL
    assert dm <= MSD_RTOL
    np.testing.assert_allclose(e, e_ref, rtol=1e-5)


@pytest.mark.parametrize("mode", ["S1", "S0"])
def test_registration_config1_full_size(mreg, c1, mode):
    """The 512^2 / 20k-node workload, full 200 iterations, in the launch
    configuration the bench times (automatic engine and shape)."""
    n = c1.spec.n_iter
    pb = _oracle(c1, mode)
    u_ref, _ = pb.run(n)
    with _reg(mreg, c1, mode) as r:
        assert r.stats()["engine"] == mreg.MREG_ENGINE_GRID
        r.step(n)
        u = r.get_u()
        msd = r.msd()
        r.stats()
    msd_ref = pb.msd(u_ref)
    du = np.abs(u - u_ref).max()
    dm = abs(msd - msd_ref) / msd_ref
    print(f"c1 {mode}: du={du:.2e} dmsd={dm:.2e}")
    assert du <= U_TOL
    assert dm <= MSD_RTOL


def test_warp_image(mreg, c0):
    pb = _oracle(c0, "S1")
    u_ref, _ = pb.run(20)
    R_ref = pb.warp(u_ref)
    with _reg(mreg, c0, "S1") as r:
        r.step(20)
        out = torch.empty(c0.Re.shape, dtype=torch.float32, device="cuda")
        msd_dev = torch.empty(1, dtype=torch.float64, device="cuda")
        r.warp(out, msd_dev)
        torch.cuda.synchronize()
        R = out.cpu().numpy()
        msd = float(msd_dev.cpu()[0])
    assert np.abs(R - R_ref).max() <= 1e-5
    assert abs(msd - pb.msd(u_ref)) <= MSD_RTOL * pb.msd(u_ref)


def test_msd_at_zero_displacement_is_pixel_mean(mreg, c0):
    with _reg(mreg, c0) as r:
        m = r.msd()
    ref = float(np.mean((c0.Te.astype(np.float64) - c0.Re) ** 2))
    assert abs(m - ref) <= 1e-6 * ref


def test_runs_are_bitwise_repeatable(mreg, c0):
    outs = []
    for _ in range(2):
        with _reg(mreg, c0, "S1") as r:
            r.step(30)
            outs.append((r.get_u(), r.msd()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


@pytest.mark.parametrize("mode", ["S0", "S1", "S2"])
def test_checkpoint_resume_is_bitwise(mreg, c0, mode):
    """A registration stopped after 10 iterations and resumed from a
    checkpoint of its state continues bit for bit as the uninterrupted one:
    the state is u and, for the Chebyshev solve of S1, the two iterates
    before it that its next starting guess is extrapolated from.  Ten plus
    ten iterations in two calls on one handle match too, and so do 1 + 1 +
    18 (the history grows from none to two across calls)."""
    with _reg(mreg, c0, mode) as r:
        r.step(20)
        u20 = r.get_u()
    for split in ((10, 10), (1, 1, 18)):
        with _reg(mreg, c0, mode) as r:
            for n in split:
                r.step(n)
            assert np.array_equal(r.get_u(), u20), split
    with _reg(mreg, c0, mode) as r:
        assert r.get_field(mreg.MREG_FIELD_U_PREV).size == 0
        r.step(10)
        u10, p10 = r.get_u(), r.get_field(mreg.MREG_FIELD_U_PREV)
    held = mode == "S1"
    assert p10.shape == ((2, c0.n_nodes, 2) if held else (0, c0.n_nodes, 2))
    with _reg(mreg, c0, mode) as r:
        r.set_u(u10)
        if held:
            r.set_u_prev(p10)
            assert np.array_equal(r.get_field(mreg.MREG_FIELD_U_PREV), p10)
        r.step(10)
        assert np.array_equal(r.get_u(), u20)


def test_previous_iterates_are_dropped_with_the_iterate(mreg, c0):
    """The history holds the iterates before u, newest first, growing to two;
    set_u and reset drop it (the next solve starts from u itself, then
    extrapolates linearly); set_u_prev checks its handle and values."""
    with _reg(mreg, c0, "S1") as r:
        r.step(1)
        u1 = r.get_u()
        assert r.get_field(mreg.MREG_FIELD_U_PREV).shape == (1, c0.n_nodes, 2)
        r.step(1)
        h = r.get_field(mreg.MREG_FIELD_U_PREV)
        assert h.shape == (2, c0.n_nodes, 2)
        assert np.array_equal(h[0], u1) and np.abs(h[1]).max() == 0.0   # u_1, then u_0 = 0
        u3 = r.get_u()
        r.set_u(u3)
        assert r.get_field(mreg.MREG_FIELD_U_PREV).size == 0
        r.step(2)
        r.reset()
        assert r.get_field(mreg.MREG_FIELD_U_PREV).size == 0
        r.step(3)
        r.set_u_prev(None)
        assert r.get_field(mreg.MREG_FIELD_U_PREV).size == 0
        bad = np.zeros((1, c0.n_nodes, 2), np.float32)
        bad[0, 5, 1] = np.inf
        with pytest.raises(mreg.MregError):
            r.set_u_prev(bad)
        # the first solve after set_u starts from u: a fresh handle given the
        # same u without history continues identically
        r.set_u(u3)
        r.step(4)
        a = r.get_u()
    with _reg(mreg, c0, "S1") as r:
        r.set_u(u3)
        r.step(4)
        assert np.array_equal(r.get_u(), a)
    with _reg(mreg, c0, "S0") as r:
        with pytest.raises(mreg.MregError):
            r.set_u_prev(np.zeros((1, c0.n_nodes, 2), np.float32))


def test_reset_restarts_the_registration(mreg, c0):
    with _reg(mreg, c0, "S0") as r:
        r.step(15)
        a = r.get_u()
        r.reset()
        assert np.abs(r.get_u()).max() == 0.0
        r.step(15)
        assert np.array_equal(r.get_u(), a)


def test_launch_shape_changes_only_rounding(mreg, c0):
    res = []
    for grid in (0, 3, 17):
        with _reg(mreg, c0, "S1", grid_blocks=grid, block_size=128, engine="grid") as r:
            r.step(30)
            res.append(r.get_u())
    for u in res[1:]:
        assert np.abs(u - res[0]).max() <= 1e-5


def test_device_images_with_row_stride(mreg, c0):
    H, W = c0.Re.shape
    big_re = torch.zeros((H, W + 13), dtype=torch.float32, device="cuda")
    big_te = torch.zeros((H, W + 13), dtype=torch.float32, device="cuda")
    big_re[:, :W] = torch.from_numpy(c0.Re)
    big_te[:, :W] = torch.from_numpy(c0.Te)
    with mreg.Registration(c0.V, c0.T, big_re[:, :W], big_te[:, :W], 0.1, 1.0, mode="S1") as r:
        r.step(10)
        ud = r.get_u()
    with _reg(mreg, c0, "S1") as r:
        r.step(10)
        uh = r.get_u()
    assert np.array_equal(ud, uh)


def test_nonfinite_device_image_is_rejected(mreg, c0):
    re = torch.from_numpy(c0.Re).cuda()
    te = torch.from_numpy(c0.Te).cuda()
    te[5, 7] = float("nan")
    with pytest.raises(mreg.MregError) as e:
        mreg.Registration(c0.V, c0.T, re, te, 0.1, 1.0)
    assert e.value.status == mreg.MREG_ERR_NONFINITE


def test_zero_iterations_and_tiny_image(mreg):
    case = _ragged_case(2, 2, seed=1)
    for mode in ("S0", "S1", "S2"):
        pb = _oracle(case, mode)
        u_ref, _ = pb.run(3)
        with _reg(mreg, case, mode) as r:
            r.step(0)
            assert np.abs(r.get_u()).max() == 0.0
            r.step(3)
            assert np.abs(r.get_u() - u_ref).max() <= 1e-6
            assert abs(r.msd() - pb.msd(u_ref)) <= 1e-5 * max(pb.msd(u_ref), 1e-12)


@pytest.mark.parametrize("mode,solver", [("S1", "chebyshev"), ("S1", "cg"), ("S2", "auto")])
def test_pcg_cap_is_reported(mreg, c0, mode, solver):
    with _reg(mreg, c0, mode, "G1" if mode == "S2" else "G0", pcg_maxit=1, pcg_rtol=1e-12,
              solver=solver) as r:
        r.step(3)
        st = r.stats(check=False)
        its = r.get_field(mreg.MREG_FIELD_PCG_ITERS)
    assert st["status"] == mreg.MREG_ERR_NOT_CONVERGED
    assert st["not_converged"] == 3 and st["max_pcg_iters"] == 1
    assert (its == 1).all()


# ---------------------------------------------------------------- extras
@pytest.mark.parametrize("grad,passes,engine", [("G0", 3, "grid"), ("G1", 4, "grid"),
                                                ("G0", 2, "batch")])
def test_repeated_smoothing_passes(mreg, c0, grad, passes, engine):
    """Eq. 14 applied several times per iteration (explicit mode)."""
    n = c0.spec.n_iter
    pb = register.Problem(c0.V, c0.T, c0.Re, c0.Te, c0.spec.alpha, c0.spec.tau, "S0", grad,
                          smooth_passes=passes)
    u_ref, e_ref = pb.run(n)
    msd_ref = pb.msd(u_ref)
    if engine == "batch":
        with mreg.Batch([(c0.V, c0.T, c0.Re, c0.Te)], c0.spec.alpha, c0.spec.tau, mode="S0",
                        grad=grad, smooth_passes=passes) as b:
            b.run(n)
            u, msd, e = b.get_u(0), b.msd()[0], b.get_field(0, mreg.MREG_FIELD_ENERGY)
    else:
        with _reg(mreg, c0, "S0", grad, smooth_passes=passes) as r:
            r.step(n)
            u, msd, e = r.get_u(), r.msd(), r.get_field(mreg.MREG_FIELD_ENERGY)
    assert np.abs(u - u_ref).max() <= U_TOL
    assert abs(msd - msd_ref) / msd_ref <= MSD_RTOL
    np.testing.assert_allclose(e, e_ref, rtol=1e-5)


def test_smoothing_passes_are_rejected_outside_the_explicit_mode(mreg, c0):
    with pytest.raises(mreg.MregError):
        _reg(mreg, c0, "S1", smooth_passes=2)


@pytest.mark.parametrize("grad,n", [("G0", 20), ("G1", 5)])
def test_paper_parameters_on_8bit_intensities(mreg, c0, grad, n):
    """The paper's own parameters, lambda = 0.8 and tau = 0.005, tuned for
    images in 0..255 (Eq. 5 and 14): the phantom scaled to that range.  On
    these data tau is an effective step 255^2 * 0.005 = 325 times that of the
    unit-range configs, and the explicit iteration amplifies rounding fast:
    perturbing the FP64 oracle by 1e-7 px per iteration moves u by 2e-6 px
    after 20 iterations and 8e-5 px after 50 with the mesh gradient, and by
    4e-6 px after 5 but 0.1 px after 20 with the spline gradient.  Parity is
    therefore checked over the horizon where the trajectory is stable.  With
    the spline gradient that step also overshoots: the MSD rises (75 -> 98
    in 5 iterations, in the oracle as on the GPU)."""
    Re, Te = (c0.Re * 255.0).astype(np.float32), (c0.Te * 255.0).astype(np.float32)
    pb = register.Problem(c0.V, c0.T, Re, Te, c0.spec.alpha, 0.005, "S0", grad, lam=0.8)
    u_ref, _ = pb.run(n)
    msd_ref = pb.msd(u_ref)
    with mreg.Registration(c0.V, c0.T, Re, Te, c0.spec.alpha, 0.005, mode="S0", grad=grad,
                           lam=0.8) as r:
        r.step(n)
        u, msd = r.get_u(), r.msd()
    assert np.abs(u).max() > 0.1                      # the registration moves
    assert np.abs(u - u_ref).max() <= U_TOL
    assert abs(msd - msd_ref) / msd_ref <= MSD_RTOL
    if grad == "G0":
        assert msd < pb.msd(np.zeros_like(u_ref))


@pytest.mark.parametrize("mode,grad,quad", [("S0", "G0", "Q0"), ("S1", "G0", "Q0"),
                                            ("S2", "G0", "Q0"), ("S2", "G1", "Q1")])
def test_device_and_host_mesh_precomputation_agree_bitwise(mreg, c0, mode, grad, quad):
    """Algorithm 1's pre-computation built on the device and on the host give
    the same arrays (incidence order, 1-rings, edge ids, FP64-summed weights
    and operators), hence bitwise the same registration."""
    out = []
    for host in (False, True):
        with _reg(mreg, c0, mode, grad, quad, host_topology=host) as r:
            r.step(20)
            out.append((r.get_u(), r.msd(), r.get_field(mreg.MREG_FIELD_ENERGY),
                        r.get_field(mreg.MREG_FIELD_FORCE)))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_device_precomputation_rejects_a_node_outside_every_triangle(mreg, c0):
    V = np.concatenate([c0.V, [[5.5, 7.25]]]).astype(np.float32)   # unused extra node
    with pytest.raises(mreg.MregError, match="no triangle"):
        mreg.Registration(V, c0.T, c0.Re, c0.Te, 0.1, 1.0)


@pytest.mark.parametrize("mode", ["S0", "S1"])
def test_run_longer_than_one_launch(mreg, mode):
    """1100 iterations: the iteration kernel is launched in chunks of 1024,
    so the state, the force buffers and the histories cross a launch."""
    case = _ragged_case(24, 25, seed=3)
    n = 1100
    pb = _oracle(case, mode)
    u_ref, e_ref = pb.run(n)
    with _reg(mreg, case, mode) as r:
        r.step(n)
        u = r.get_u()
        e = r.get_field(mreg.MREG_FIELD_ENERGY)
        F = r.get_field(mreg.MREG_FIELD_FORCE)
        r.stats()
    assert len(e) == n
    assert np.abs(u - u_ref).max() <= U_TOL
    np.testing.assert_allclose(e, e_ref, rtol=1e-5, atol=1e-12)
    # the force the last iteration applied: F at u_{n-1}
    u_prev, _ = pb.run(n - 1)
    f, rr, g = pb.sample(u_prev)
    F_ref = pb.force(u_prev, f, rr, g)
    assert np.abs(F - F_ref).max() <= 1e-4 * max(np.abs(F_ref).max(), 1e-6)


def test_caller_allocator(mreg, c0):
    """Every device buffer of a handle or batch can come from the caller's
    allocator (here PyTorch's caching allocator) and goes back to it."""
    alloc = mreg.TorchAllocator()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with _reg(mreg, c0, "S1", allocator=alloc) as r:
        assert torch.cuda.memory_allocated() > base   # the arena is torch's memory
        r.step(20)
        u_a, m_a = r.get_u(), r.msd()
        g_a = torch.empty(c0.n_nodes, 2, device="cuda")
        r.warp_energy_grad(torch.from_numpy(u_a).cuda(), None, g_a)   # adjoint scratch too
        torch.cuda.synchronize()
        del g_a
    with _reg(mreg, c0, "S1") as r:
        r.step(20)
        assert np.array_equal(u_a, r.get_u()) and m_a == r.msd()
    with mreg.Batch([(c0.V, c0.T, c0.Re, c0.Te)] * 2, 0.1, 1.0, mode="S1", allocator=alloc) as b:
        b.run(5)
        assert np.isfinite(b.msd()).all()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base   # everything was given back

    class Failing:
        alloc_fn = mreg.ALLOC_FN(lambda n, s, c: None)
        free_fn = mreg.FREE_FN(lambda p, s, c: None)
    with pytest.raises(mreg.MregError) as e:
        _reg(mreg, c0, "S1", allocator=Failing())
    assert e.value.status == mreg.MREG_ERR_OOM


@pytest.mark.parametrize("mode,grad,quad", [("S0", "G0", "Q0"), ("S1", "G0", "Q0"),
                                            ("S2", "G1", "Q0"), ("S2", "G1", "Q1")])
def test_energy_terms_of_eq1(mreg, c0, mode, grad, quad):
    """mreg_energy = D + alpha S at the current u, against the oracle's data
    term and regulariser at the GPU's own u (so only the evaluation is
    compared: D from FP32 spline samples, S in FP64)."""
    pb = _oracle(c0, mode, grad, quad)
    with _reg(mreg, c0, mode, grad, quad) as r:
        r.step(10)
        u = r.get_u().astype(np.float64)
        d, sm = r.energy_terms()
        e = r.energy()
    d_ref, s_ref = pb.data_energy(u), pb.smoothness(u)
    assert abs(d - d_ref) <= 1e-5 * d_ref
    assert abs(sm - s_ref) <= 1e-6 * s_ref + 1e-12
    assert e == pytest.approx(d + c0.spec.alpha * sm, rel=1e-15)


@pytest.mark.parametrize("mode,grad,quad", [m for m in MODES if m[0] != "S0"])
def test_two_lanes_per_node(mreg, c0, mode, grad, quad):
    """The implicit forms with each node's neighbour and incidence lists split
    between two lanes (the automatic choice when one node per lane pair fits
    the grid) and with one lane per node: both within the FP32 tolerances of
    the oracle, and equal to each other up to summation order."""
    n = 30
    pb = _oracle(c0, mode, grad, quad)
    u_ref, _ = pb.run(n)
    msd_ref = pb.msd(u_ref)
    out = {}
    for lanes in (1, 2):
        with _reg(mreg, c0, mode, grad, quad, engine="grid", node_lanes=lanes) as r:
            r.step(n)
            out[lanes] = (r.get_u(), r.msd(), r.stats())
    assert out[1][2]["node_lanes"] == 1 and out[2][2]["node_lanes"] == 2
    assert out[2][2]["block_size"] == 512
    for lanes in (1, 2):
        u, msd, _ = out[lanes]
        assert np.abs(u - u_ref).max() <= U_TOL
        assert abs(msd - msd_ref) / msd_ref <= MSD_RTOL
    assert np.abs(out[1][0] - out[2][0]).max() <= 1e-5
    with _reg(mreg, c0, mode, grad, quad) as r:
        assert r.stats()["node_lanes"] == 2


def test_automatic_lanes_follow_the_mesh_size(mreg):
    """More than 256 nodes per SM: one lane per node, blocks of 512; the
    explicit mode always runs one lane per node."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    side = int(np.ceil(np.sqrt(sms * 256 + 1))) + 1   # side^2 nodes > 256 per SM
    ys, xs = np.mgrid[0:side, 0:side]
    V = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float32)
    idx = (ys * side + xs)[:-1, :-1].ravel()
    T = np.concatenate([np.stack([idx, idx + 1, idx + side + 1], 1),
                        np.stack([idx, idx + side + 1, idx + side], 1)]).astype(np.int32)
    img = np.zeros((side, side), np.float32)
    with mreg.Registration(V, T, img, img, 0.1, 1.0, mode="S1") as r:
        st = r.stats()
        assert st["node_lanes"] == 1 and st["block_size"] == 512
    with mreg.Registration(V, T, img, img, 0.1, 1.0, mode="S0") as r:
        assert r.stats()["node_lanes"] == 1


@pytest.mark.parametrize("hw", RAGGED)
@pytest.mark.parametrize("amp", [0.7, 6.0])
def test_warp_on_ragged_images(mreg, hw, amp):
    """The warp + MSD against the oracle on images whose sides are not
    multiples of the 32 x 16 tile, down to 2 x 2 (no 4 x 4 window inside the
    image), with displacements that keep the taps inside (0.7 px) or push
    many of them through the mirror extension (6 px)."""
    H, W = hw
    case = _ragged_case(H, W, seed=11)
    x = case.V[:, 0].astype(np.float64)
    y = case.V[:, 1].astype(np.float64)
    u = (amp * np.stack([np.sin(x / 5.0 + 0.3), np.cos(y / 4.0 - 0.2)], 1)).astype(np.float32)
    pb = _oracle(case)
    R_ref = pb.warp(u.astype(np.float64))
    msd_ref = pb.msd(u.astype(np.float64))
    with _reg(mreg, case) as r:
        r.set_u(u)
        out = torch.empty((H, W), dtype=torch.float32, device="cuda")
        msd_dev = torch.empty(1, dtype=torch.float64, device="cuda")
        r.warp(out, msd_dev)
        torch.cuda.synchronize()
        R = out.cpu().numpy()
        msd = float(msd_dev.cpu()[0])
        assert abs(r.msd() - msd) <= 1e-12 * msd + 1e-18   # the MSD-only instance
    scale = max(1.0, float(np.abs(case.Te).max()))
    assert np.abs(R - R_ref).max() <= 1e-5 * scale
    assert abs(msd - msd_ref) <= 1e-5 * msd_ref + 1e-12


# ------------------------------------------------ the solve's stated residual
@pytest.mark.parametrize("mode,grad,quad,solver", [
    ("S1", "G0", "Q0", "auto"), ("S1", "G1", "Q0", "auto"), ("S1", "G0", "Q0", "cg"),
    ("S2", "G0", "Q0", "auto"), ("S2", "G1", "Q1", "auto")])
def test_solve_residual_recomputed_in_fp64(mreg, c0, c1, mode, grad, quad, solver):
    """The stopping rule of the semi-implicit solve, ||b - A u'||_2 <=
    rtol ||b||_2 per component, recomputed on the host in FP64 from what the
    library hands out: u before and after one step and the force that step
    applied (MREG_FIELD_FORCE).  S1: b = D_m (u - tau F), A = (1+l) D_m - l W
    with l in full precision (the kernel carries l and tau as float-float
    pairs).  S2: b = M u - tau F_w, A = M + l K, with the FP32 matrix entries
    the kernel is given (the FP64 assembly rounded to FP32, as here).  The
    step is taken from a state 20 iterations in, on both the 128^2 and the
    512^2 pair.  S1 runs both solvers (Chebyshev semi-iteration by default,
    CG on request)."""
    import scipy.sparse as sp
    rtol = 1e-7
    for case in (c0, c1):
        pb = _oracle(case, mode, grad, quad)
        with _reg(mreg, case, mode, grad, quad, solver=solver) as r:
            r.step(20)
            u = r.get_u().astype(np.float64)
            r.step(1)
            u1 = r.get_u().astype(np.float64)
            F = r.get_field(mreg.MREG_FIELD_FORCE).reshape(-1, 2).astype(np.float64)
            reported = r.get_field(mreg.MREG_FIELD_PCG_RESID)
        tau, lam = case.spec.tau, pb.lam
        if mode == "S1":
            A = ((1.0 + lam) * sp.diags(pb.m) - lam * pb.Wadj).tocsr()
            b = pb.m[:, None] * (u - tau * F)
        else:
            M, K = pb.M.tocsr(), pb.K.tocsr()
            M32 = M.astype(np.float32).astype(np.float64)
            A = (M + lam * K).tocsr().astype(np.float32).astype(np.float64)
            b = M32 @ u - tau * F
        res = b - A @ u1
        rel = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
        print(f"{mode}{grad}{quad} {solver} {case.spec.side}^2: FP64 residual {rel.max():.2e}, "
              f"reported {reported[-1]:.2e}")
        assert (rel <= rtol).all()
        assert reported[-1] <= rtol


@pytest.mark.parametrize("grad", ["G0", "G1"])
def test_umbrella_solvers_agree(mreg, c0, c1, grad):
    """S1 solved by Chebyshev semi-iteration (the default) and by CG: every
    solve of both meets the verified residual bound, both registrations meet
    the parity bar against the oracle's direct solve (and so agree with each
    other to within it).  The Chebyshev step counts stay small (the
    spectrum of the Jacobi-scaled matrix lies in [1/(1+l), (1+2l)/(1+l)])."""
    for case in (c0, c1):
        n = case.spec.n_iter
        pb = _oracle(case, "S1", grad)
        u_ref, _ = pb.run(n)
        out = {}
        for solver in ("cg", "chebyshev"):
            with _reg(mreg, case, "S1", grad, solver=solver) as r:
                r.step(n)
                st = r.stats()
                out[solver] = (r.get_u(), r.get_field(mreg.MREG_FIELD_PCG_ITERS),
                               r.get_field(mreg.MREG_FIELD_PCG_RESID), st)
        for solver, (u, its, res, st) in out.items():
            du = np.abs(u - u_ref).max()
            print(f"S1{grad} {solver} {case.spec.side}^2: du={du:.2e} steps mean "
                  f"{its.mean():.2f} max {its.max()} resid max {res.max():.2e}")
            assert du <= U_TOL
            assert len(res) == n and (res <= 1e-7).all()
            assert st["not_converged"] == 0
        assert np.abs(out["cg"][0] - out["chebyshev"][0]).max() <= U_TOL
        assert out["chebyshev"][1].mean() <= 8


@pytest.mark.parametrize("grad", ["G0", "G1"])
def test_neighbour_sync_changes_no_bit(mreg, c0, c1, grad):
    """The Chebyshev steps synchronise each block only with the blocks that
    own its nodes' neighbours; that changes when a block may proceed, never
    what it computes, so the registration is bitwise the same as with the
    grid barrier after every step (and so, through the parity tests, the
    oracle's)."""
    for case in (c0, c1):
        out = []
        for ns in (True, False):
            with _reg(mreg, case, "S1", grad, neighbour_sync=ns) as r:
                assert r.stats()["neighbour_sync"] == (1 if ns else 0)
                r.step(case.spec.n_iter)
                out.append((r.get_u(), r.msd(), r.get_field(mreg.MREG_FIELD_PCG_ITERS)))
        assert np.array_equal(out[0][0], out[1][0])
        assert out[0][1] == out[1][1]
        assert np.array_equal(out[0][2], out[1][2])
