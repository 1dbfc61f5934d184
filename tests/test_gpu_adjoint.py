"""The differentiation form: the adjoint kernel of the warp-plus-SSD energy
against the FP64 oracle (its analytic gradient and central differences of
its energy), and the torch.autograd.Function around it.

Tolerances: the energy is an FP32 sum of squares accumulated in float-float,
held to 1e-5 relative.  A node's gradient sums ~10-100 pixel terms r grad Te,
each carrying the FP32 error of a spline sample (5e-6 of max |c|) times
|grad Te|, so the gradient is held to 1e-4 of max |dE/du| (and so is the
comparison with central differences of the FP64 energy, whose own error at
h = 1e-6 is ~1e-9 relative).
"""
import numpy as np
import pytest

from oracle import adjoint, register
from paper_1411_2141_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

G_RTOL = 1e-4
E_RTOL = 1e-5


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


def _smooth_u(c, amp, seed):
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 1.5, size=4)
    x, y = c.V[:, 0].astype(np.float64), c.V[:, 1].astype(np.float64)
    s = c.spec.side
    return (amp * np.stack([np.sin(2 * np.pi * k[0] * x / s + k[1]),
                            np.cos(2 * np.pi * k[2] * y / s + k[3])], axis=1)).astype(np.float32)


def _check(mreg, case, u, n_fd=8):
    pb = register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                          "S0", "G1")
    E_ref, g_ref = adjoint.warp_energy_grad(pb, u.astype(np.float64))
    with mreg.Registration(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                           mode="S0", grad="G1") as r:
        ud = torch.from_numpy(u).cuda()
        E = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty_like(ud)
        r.warp_energy_grad(ud, E, g)
        g2 = torch.empty_like(ud)
        r.warp_energy_grad(ud, None, g2)
        torch.cuda.synchronize()
        E, g, g2 = float(E.item()), g.cpu().numpy(), g2.cpu().numpy()
    scale = np.abs(g_ref).max()
    dg = np.abs(g - g_ref).max() / scale
    print(f"n={case.n_nodes}: dE={abs(E - E_ref) / E_ref:.2e} dg={dg:.2e} (max|g|={scale:.3g})")
    assert abs(E - E_ref) <= E_RTOL * E_ref
    assert dg <= G_RTOL
    assert np.array_equal(g, g2)            # bitwise repeatable, energy or not
    rng = np.random.default_rng(1)
    h = 1e-6
    for a in rng.choice(pb.n, size=n_fd, replace=False):
        for c in range(2):
            up = u.astype(np.float64)
            um = up.copy()
            up[a, c] += h
            um[a, c] -= h
            fd = (adjoint.warp_energy(pb, up) - adjoint.warp_energy(pb, um)) / (2 * h)
            assert abs(g[a, c] - fd) <= G_RTOL * scale


@pytest.mark.parametrize("amp", [0.0, 1.5])
def test_adjoint_config0(mreg, case0, amp):
    _check(mreg, case0, _smooth_u(case0, amp, 7))


def test_adjoint_batch_of_256px_pairs(mreg):
    """The differentiation workload: 256x256 pairs with ~5k-node meshes (a
    sample of 4 of its 64 pairs, at a smooth displacement of ~2 px)."""
    specs = inputs.batched_specs(4)
    for spec in specs[:: len(specs) // 4][:4]:
        case = inputs.make_case(spec)
        _check(mreg, case, _smooth_u(case, 2.0, spec.seed), n_fd=4)


def test_autograd_function(mreg, case0):
    from paper_1411_2141_gb300.autograd import warp_energy
    u0 = _smooth_u(case0, 1.0, 3)
    with mreg.Registration(case0.V, case0.T, case0.Re, case0.Te, 0.1, 1.0) as r:
        u = torch.from_numpy(u0).cuda().requires_grad_(True)
        E = warp_energy(u, r)
        assert E.dtype == torch.float64 and E.dim() == 0
        (3.0 * E + (u * u).sum()).backward()
        g_direct = torch.empty_like(u)
        r.warp_energy_grad(u.detach(), None, g_direct)
        torch.testing.assert_close(u.grad, 3.0 * g_direct + 2.0 * u.detach(), rtol=1e-6, atol=1e-6)
        # no gradient requested: forward only
        with torch.no_grad():
            E2 = warp_energy(u.detach(), r)
        assert float(E2) == float(E)


def _unroll_check(mreg, case, u0, K, n_fd):
    """The library's unrolled gradient against the oracle's adjoint recursion
    and central differences of the oracle's composed FP64 energy.  Twenty
    FP32 forward steps and twenty FP32 adjoint steps each add the rounding
    of the single-step gradient (~1e-6 of its max), so the bar is 1e-4 of
    max |dE/du0|."""
    pb = register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                          "S0", "G1")
    E_ref, g_ref = adjoint.unrolled_grad(pb, u0.astype(np.float64), K)
    with mreg.Registration(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                           mode="S0", grad="G1") as r:
        ud = torch.from_numpy(u0).cuda()
        E = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty_like(ud)
        r.unroll_grad(ud, K, E, g)
        torch.cuda.synchronize()
        E, g = float(E.item()), g.cpu().numpy()
        uK = r.get_u()
    u_ref, _ = pb.run(K, u0.astype(np.float64))
    scale = np.abs(g_ref).max()
    dg = np.abs(g - g_ref).max() / scale
    print(f"unroll K={K} n={case.n_nodes}: du_K={np.abs(uK - u_ref).max():.2e} "
          f"dE={abs(E - E_ref) / E_ref:.2e} dg={dg:.2e}")
    assert np.abs(uK - u_ref).max() <= 1e-4
    assert abs(E - E_ref) <= 1e-5 * E_ref
    assert dg <= 1e-4
    rng = np.random.default_rng(4)
    h = 1e-6
    for a in rng.choice(pb.n, size=n_fd, replace=False):
        c = int(rng.integers(2))
        up = u0.astype(np.float64)
        um = up.copy()
        up[a, c] += h
        um[a, c] -= h
        fd = (adjoint.unrolled_energy(pb, up, K) - adjoint.unrolled_energy(pb, um, K)) / (2 * h)
        assert abs(g[a, c] - fd) <= 1e-4 * scale


def test_unrolled_gradient_config0(mreg, case0):
    _unroll_check(mreg, case0, _smooth_u(case0, 0.5, 11), 20, n_fd=6)


def test_unrolled_gradient_256px_pairs(mreg):
    """The 20-iteration unroll on two of the 64 differentiation pairs
    (256x256, ~5k nodes)."""
    specs = inputs.batched_specs(4)
    for spec in (specs[0], specs[33]):
        case = inputs.make_case(spec)
        _unroll_check(mreg, case, _smooth_u(case, 1.0, spec.seed), spec.n_iter, n_fd=2)


def test_unrolled_autograd_and_mode_check(mreg, case0):
    from paper_1411_2141_gb300.autograd import unrolled_warp_energy
    u0 = _smooth_u(case0, 0.5, 12)
    with mreg.Registration(case0.V, case0.T, case0.Re, case0.Te, 0.1, 1.0, mode="S0",
                           grad="G1") as r:
        u = torch.from_numpy(u0).cuda().requires_grad_(True)
        E = unrolled_warp_energy(u, r, 5)
        E.backward()
        g = torch.empty_like(u)
        r.unroll_grad(u.detach(), 5, None, g)
        assert torch.equal(u.grad, g)
    with mreg.Registration(case0.V, case0.T, case0.Re, case0.Te, 0.1, 1.0, mode="S1") as r:
        with pytest.raises(mreg.MregError):
            r.unroll_grad(torch.zeros(case0.n_nodes, 2, device="cuda"), 3)


def test_unrolled_gradient_with_repeated_smoothing(mreg, case0):
    pb = register.Problem(case0.V, case0.T, case0.Re, case0.Te, case0.spec.alpha,
                          case0.spec.tau, "S0", "G1", smooth_passes=3)
    u0 = _smooth_u(case0, 0.5, 13)
    _, g_ref = adjoint.unrolled_grad(pb, u0.astype(np.float64), 10)
    with mreg.Registration(case0.V, case0.T, case0.Re, case0.Te, case0.spec.alpha,
                           case0.spec.tau, mode="S0", grad="G1", smooth_passes=3) as r:
        g = torch.empty(case0.n_nodes, 2, device="cuda")
        r.unroll_grad(torch.from_numpy(u0).cuda(), 10, None, g)
        g = g.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_unroll_of_zero_iterations_is_the_warp_gradient(mreg, case0):
    u0 = torch.from_numpy(_smooth_u(case0, 0.5, 14)).cuda()
    with mreg.Registration(case0.V, case0.T, case0.Re, case0.Te, 0.1, 1.0, mode="S0",
                           grad="G1") as r:
        g0 = torch.empty_like(u0)
        g1 = torch.empty_like(u0)
        E0 = torch.empty(1, dtype=torch.float64, device="cuda")
        E1 = torch.empty_like(E0)
        r.unroll_grad(u0, 0, E0, g0)
        r.warp_energy_grad(u0, E1, g1)
        torch.cuda.synchronize()
        assert torch.equal(g0, g1) and torch.equal(E0, E1)
        assert np.abs(r.get_u() - u0.cpu().numpy()).max() == 0.0   # the iterate is u0


@pytest.mark.parametrize("passes", [1, 3])
def test_checkpointed_unroll_is_bitwise_the_dense_one(mreg, passes):
    """Keeping only every c-th state and recomputing the segments in the
    backward pass gives the gradient, the energy and the final iterate of
    the run that keeps every state, bit for bit (the segments are recomputed
    by the same kernel in the same launch shape), for segment lengths that
    divide K, that do not, of one iteration, and K itself."""
    from paper_1411_2141_gb300.autograd import unrolled_warp_energy
    case = inputs.make_case(inputs.batched_specs(4)[5])
    K = case.spec.n_iter
    u0 = torch.from_numpy(_smooth_u(case, 1.0, 21)).cuda()
    with mreg.Registration(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                           mode="S0", grad="G1", smooth_passes=passes) as r:
        def run(c):
            E = torch.empty(1, dtype=torch.float64, device="cuda")
            g = torch.empty_like(u0)
            r.unroll_grad(u0, K, E, g, checkpoint_every=c)
            torch.cuda.synchronize()
            return E.cpu(), g.cpu(), r.get_u()
        E0, g0, u0K = run(0)
        for c in (1, 3, 5, 7, K):
            E, g, uK = run(c)
            assert torch.equal(E, E0) and torch.equal(g, g0), c
            assert np.array_equal(uK, u0K), c
        u = u0.clone().requires_grad_(True)
        Ea = unrolled_warp_energy(u, r, K, 4)
        Ea.backward()
        assert torch.equal(u.grad.cpu(), g0) and float(Ea) == float(E0)
        with pytest.raises(mreg.MregError):
            r.unroll_grad(u0, K, None, torch.empty_like(u0), checkpoint_every=-1)
