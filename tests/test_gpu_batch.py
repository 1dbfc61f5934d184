"""The batched engine (many pairs of uneven size in one persistent launch,
replayed from a CUDA graph) against the FP64 oracle, pair by pair.

Tolerances are those of the one-pair FP32 form: node displacements within
1e-4 px and MSD within 1e-5 relative of the oracle.  The per-iteration data
energy follows the trajectory, which on these small pairs amplifies rounding
about 100x over 30 iterations (perturbing the FP64 oracle by 1e-7 px per
iteration moves u by up to 1.2e-5 px with the spline gradient), so it is
held to 5e-5 relative.  A pair's result may depend on the team shape
(the order of its reductions) but not on the other pairs: that is checked
bit for bit.
"""
import numpy as np
import pytest

from oracle import register
from paper_1411_2141_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U_TOL = 1e-4
MSD_RTOL = 1e-5


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


def _small_specs():
    """Six uneven pairs in the size range of the batched workload (sides
    96-200, node counts by its rule 500 (side/96)^2.107), small enough for
    the oracle.  (Coarser meshes on smaller images amplify FP32 rounding
    along the trajectory ~100x over 30 iterations, which would test the
    problem's conditioning rather than the kernels.)"""
    out = []
    for k, side in enumerate([96, 200, 110, 150, 128, 175]):
        out.append(inputs.CaseSpec(side=side, n_nodes=int(round(500 * (side / 96.0) ** 2.107)),
                                   seed=5000 + k, n_blobs=20, n_ellipses=10, supersample=4,
                                   dmax=min(8.0, 3.0 * side / 128.0), n_iter=30))
    return out


@pytest.fixture(scope="module")
def small():
    return [inputs.make_case(s) for s in _small_specs()]


def _batch(mreg, cases, **kw):
    return mreg.Batch([(c.V, c.T, c.Re, c.Te) for c in cases], cases[0].spec.alpha,
                      cases[0].spec.tau, **kw)


def _oracle(case, mode, grad, quad, n):
    pb = register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                          mode, grad, quad)
    u, e = pb.run(n)
    return u, e, pb.msd(u)


@pytest.fixture(scope="module")
def oracle_small(small):
    cache = {}

    def get(k, mode, grad, quad, n):
        key = (k, mode, grad, quad, n)
        if key not in cache:
            cache[key] = _oracle(small[k], mode, grad, quad, n)
        return cache[key]
    return get


@pytest.mark.parametrize("mode,grad,quad,ctas,block", [
    ("S1", "G0", "Q0", 2, 256), ("S1", "G0", "Q0", 1, 128), ("S1", "G0", "Q0", 4, 512),
    ("S0", "G0", "Q0", 2, 256), ("S0", "G1", "Q0", 1, 256), ("S1", "G1", "Q0", 8, 128),
    ("S2", "G0", "Q0", 2, 256), ("S2", "G1", "Q0", 2, 256), ("S2", "G1", "Q1", 2, 256)])
def test_batch_matches_oracle(mreg, small, oracle_small, mode, grad, quad, ctas, block):
    n = 30
    with _batch(mreg, small, mode=mode, grad=grad, quad=quad, team_ctas=ctas,
                block_size=block) as b:
        assert b.shape()[:2] == (ctas, block)
        b.run(n)
        msd = b.msd()
        for k, case in enumerate(small):
            u_ref, e_ref, msd_ref = oracle_small(k, mode, grad, quad, n)
            u = b.get_u(k)
            e = b.get_field(k, mreg.MREG_FIELD_ENERGY)
            st = b.stats(k)
            du = np.abs(u - u_ref).max()
            dm = abs(msd[k] - msd_ref) / msd_ref
            print(f"{mode}{grad}{quad} {ctas}x{block} pair {k} (n={case.n_nodes}): "
                  f"du={du:.2e} dmsd={dm:.2e} cg={st['max_pcg_iters']}")
            assert du <= U_TOL
            assert dm <= MSD_RTOL
            np.testing.assert_allclose(e, e_ref, rtol=5e-5)
            if mode != "S0":
                res = b.get_field(k, mreg.MREG_FIELD_PCG_RESID)
                assert len(res) == n and (res <= 1e-7).all()


def test_pair_result_does_not_depend_on_the_batch(mreg, small):
    """Same team shape: a pair registered inside the batch and alone give
    the same bits; two runs of the batch give the same bits."""
    n = 20
    with _batch(mreg, small, mode="S1", team_ctas=2, block_size=256) as b:
        b.run(n)
        u_all = [b.get_u(k) for k in range(len(small))]
        m_all = b.msd()
        b.run(n)
        for k in range(len(small)):
            assert np.array_equal(b.get_u(k), u_all[k])
        assert np.array_equal(b.msd(), m_all)
    for k in (1, 4):
        with _batch(mreg, [small[k]], mode="S1", team_ctas=2, block_size=256) as b1:
            b1.run(n)
            assert np.array_equal(b1.get_u(0), u_all[k])
            assert b1.msd()[0] == m_all[k]


def test_autotuner_picks_a_timed_shape(mreg, small, oracle_small):
    n = 30
    with _batch(mreg, small, mode="S1") as b:
        best, times = b.tune(n)
        timed = {k: v for k, v in times.items() if v is not None}
        assert best in timed and timed[best] == min(timed.values())
        assert b.shape()[:3] == best
        b.run(n)
        for k in (0, 1):
            u_ref, _, msd_ref = oracle_small(k, "S1", "G0", "Q0", n)
            assert np.abs(b.get_u(k) - u_ref).max() <= U_TOL
            assert abs(b.msd()[k] - msd_ref) / msd_ref <= MSD_RTOL


@pytest.mark.parametrize("mode,grad", [("S1", "G0"), ("S2", "G1")])
def test_two_ctas_per_sm_register_budget(mreg, small, oracle_small, mode, grad):
    """The 64-register variant of the iteration kernel (spills to local
    memory) gives the oracle's results too."""
    n = 30
    with _batch(mreg, small, mode=mode, grad=grad, team_ctas=2, block_size=256,
                team_blocks_per_sm=2) as b:
        assert b.shape()[:3] == (2, 256, 2)
        b.run(n)
        msd = b.msd()
        for k in range(len(small)):
            u_ref, _, msd_ref = oracle_small(k, mode, grad, "Q0", n)
            assert np.abs(b.get_u(k) - u_ref).max() <= U_TOL
            assert abs(msd[k] - msd_ref) / msd_ref <= MSD_RTOL


def test_fields_of_a_pair(mreg, small):
    from oracle import bspline, register
    with _batch(mreg, small[:3], mode="S1", coeff_bf16=True) as b:
        b.run(3)
        for k, case in enumerate(small[:3]):
            pix = b.get_field(k, mreg.MREG_FIELD_PIXEL_TRI)
            H, W = case.Re.shape
            assert np.array_equal(pix, register.locate_pixels(case.V, case.T, W, H).astype(np.int32))
            c = bspline.prefilter_2d(case.Te.astype(np.float64))
            cg = b.get_field(k, mreg.MREG_FIELD_COEF_TE)
            assert np.abs(cg - c).max() <= 5e-6 * np.abs(c).max()
            c16 = b.get_field(k, mreg.MREG_FIELD_COEF_TE_16)
            assert c16.shape == case.Re.shape
            assert len(b.get_field(k, mreg.MREG_FIELD_PCG_ITERS)) == 3


def test_batched_workload_full_size(mreg):
    """The 256-pair workload (sides 96-768, 500-40k nodes, 100 iterations) in
    the launch configuration the bench times; EVERY pair is checked against
    its own FP64 oracle registration (run on the host cores in parallel,
    largest pairs first, while the GPU works), and for a lower MSD than
    before registration.

    A few pairs of this workload fold their mesh so badly that their FP64
    trajectory is itself ill-conditioned at FP32 level: the oracle's result
    moves by more than a tenth of the node tolerance when its own iterate is
    rounded to FP32 after every iteration (see oracle_jobs; decided from the
    oracle alone).  Their trajectories are chaotic -- the triangle gradient
    of Eq. 9 changes sign with the deformed area, so the force jumps where a
    triangle inverts -- and node-wise parity is not defined for them; they
    are checked for an MSD within 2e-3 relative of the oracle's (measured:
    at most 6e-4), finite displacements and a lower MSD than before
    registration.  Every other pair meets the full bar, and the
    ill-conditioned ones are at most a few percent of the batch."""
    from tests import oracle_jobs
    specs = inputs.batched_specs(3)
    n = specs[0].n_iter
    big_first = sorted(range(len(specs)), key=lambda k: -specs[k].side)
    with oracle_jobs.pool() as ex:
        futs = {k: ex.submit(oracle_jobs.registration_and_sensitivity,
                             (specs[k], "S1", "G0", "Q0", n))
                for k in big_first}
        cases = inputs.make_cases(specs)
        with _batch(mreg, cases, mode="S1") as b:
            b.run(n)
            msd = b.msd()
            us = [b.get_u(k) for k in range(len(cases))]
            for k in range(len(cases)):
                b.stats(k)
        refs = {k: f.result() for k, f in futs.items()}
    du = np.array([np.abs(us[k] - refs[k][0]).max() for k in range(len(cases))])
    dm = np.array([abs(msd[k] - refs[k][2]) / refs[k][2] for k in range(len(cases))])
    spread = np.array([refs[k][3] for k in range(len(cases))])
    ill = spread > 0.1 * U_TOL
    ok = ~ill
    w = int(np.argmax(np.where(ok, du, 0.0)))
    print(f"256 pairs: {ok.sum()} well-conditioned, max du={du[ok].max():.2e} px (pair {w}, "
          f"side {cases[w].spec.side}, n={cases[w].n_nodes}), max dmsd={dm[ok].max():.2e}")
    for k in np.flatnonzero(ill):
        print(f"  ill-conditioned pair {k} (side {cases[k].spec.side}): oracle spread "
              f"{spread[k]:.2e} px, du={du[k]:.2e} px, dmsd={dm[k]:.2e}")
    assert ill.sum() <= 16
    assert (du[ok] <= U_TOL).all()
    assert (dm[ok] <= MSD_RTOL).all()
    assert (dm[ill] <= 2e-3).all()
    assert all(np.isfinite(us[k]).all() for k in range(len(cases)))
    before = np.array([np.mean((c.Re.astype(np.float64) - c.Te) ** 2) for c in cases])
    assert np.isfinite(msd).all() and (msd < before).all()


def _ragged_case(H, W, seed):
    """A small H x W pair (any aspect ratio) with a regular mesh of its
    corners and a few interior nodes."""
    from tests.test_gpu_parity import _ragged_case as make
    return make(H, W, seed)


def test_batch_with_degenerate_and_ragged_pairs(mreg, small):
    """A 2x2 pair (two triangles), a ragged non-square pair and normal pairs in
    one batch, every form; and a batch of a single pair."""
    tiny = _ragged_case(2, 2, seed=1)
    ragged = _ragged_case(37, 70, seed=2)
    cases = [small[0], tiny, ragged, small[2]]
    n = 6
    for mode, grad in (("S0", "G0"), ("S1", "G0"), ("S2", "G1")):
        with mreg.Batch([(c.V, c.T, c.Re, c.Te) for c in cases], 0.1, 1.0, mode=mode,
                        grad=grad) as b:
            b.run(n)
            msd = b.msd()
            for k, c in enumerate(cases):
                pb = register.Problem(c.V, c.T, c.Re, c.Te, 0.1, 1.0, mode, grad)
                u_ref, _ = pb.run(n)
                m_ref = pb.msd(u_ref)
                assert np.abs(b.get_u(k) - u_ref).max() <= U_TOL
                assert abs(msd[k] - m_ref) <= MSD_RTOL * max(m_ref, 1e-12)
    with mreg.Batch([(tiny.V, tiny.T, tiny.Re, tiny.Te)], 0.1, 1.0, mode="S1") as b:
        b.run(3)
        assert b.shape()[3] == 1 and np.isfinite(b.msd()).all()
