"""Failure detection of the persistent iteration kernel, without a GPU fault.

Every grid-barrier wait of the iteration kernel is bounded.  The test hook
mreg_test_barrier_timeout makes one block leave out one barrier arrival and
shortens the bound to 1 ms, so the other blocks' waits (and its own) run out
on schedule: nothing traps, nothing hangs, and the GPU context stays usable.
The tests check that the failure is reported (MREG_ERR_DEVICE_CHECK), that
the handle refuses further steps until it is reset, that the autograd
wrapper refuses to hand back a gradient of the unfinished run, and that a
reset handle registers exactly as a fresh one.
"""
import numpy as np
import pytest

from paper_1411_2141_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TIMEOUT_NS = 1_000_000   # 1 ms
STATUS_TIMEOUT, STATUS_ABORT = 2, 4


@pytest.fixture(scope="module")
def mreg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_2141_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    from paper_1411_2141_gb300 import mreg as m
    m.load()
    return m


@pytest.fixture(scope="module")
def c0():
    return inputs.make_case(inputs.config_spec(0))


def _reg(mreg, case, mode, grad="G0", **kw):
    return mreg.Registration(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                             mode=mode, grad=grad, **kw)


# Synchronisation numbers of an S1 launch (Chebyshev solve): 1 after the
# iterate is copied in, 2 after the first sample, 3 after the force phase of
# iteration 0 (grid barriers), then the solve's steps (the neighbour
# synchronisation when nsync, else grid barriers): 5 and 7 fall on steps, in
# the first and the second solve.
@pytest.mark.parametrize("mode,barrier,nsync", [("S0", 3, True), ("S1", 1, True),
                                                ("S1", 5, True), ("S1", 7, True),
                                                ("S1", 5, False)])
def test_barrier_timeout_is_reported_and_reset_recovers(mreg, c0, mode, barrier, nsync):
    with _reg(mreg, c0, mode) as ref:
        ref.step(10)
        u_ref = ref.get_u()
    with _reg(mreg, c0, mode, neighbour_sync=nsync) as r:
        grid = r.stats()["grid_blocks"]
        r.test_barrier_timeout(grid - 1, barrier, TIMEOUT_NS)
        r.step(10)
        r.step(3)   # a later launch on the failed handle leaves at once
        with pytest.raises(mreg.MregError) as e:
            r.stats()
        assert e.value.status == mreg.MREG_ERR_DEVICE_CHECK
        st = r.stats(check=False)
        assert st["status"] == mreg.MREG_ERR_DEVICE_CHECK
        assert st["device_status"] & STATUS_TIMEOUT and st["device_status"] & STATUS_ABORT
        with pytest.raises(mreg.MregError) as e:   # refused on the host until reset
            r.step(1)
        assert e.value.status == mreg.MREG_ERR_DEVICE_CHECK
        r.reset()
        r.step(10)
        assert np.array_equal(r.get_u(), u_ref)
        assert r.stats()["device_status"] == 0


def test_unreached_barrier_leaves_the_launch_alone(mreg, c0):
    with _reg(mreg, c0, "S0") as ref:
        ref.step(2)
        u_ref = ref.get_u()
    with _reg(mreg, c0, "S0") as r:
        r.test_barrier_timeout(0, 1000, TIMEOUT_NS)   # 2 iterations pass ~4 barriers
        r.step(2)
        assert r.stats()["device_status"] == 0
        assert np.array_equal(r.get_u(), u_ref)


def test_unrolled_gradient_refuses_a_timed_out_run(mreg, c0):
    from paper_1411_2141_gb300 import autograd
    with _reg(mreg, c0, "S0", "G1") as r:
        u0 = torch.zeros((r.n_nodes, 2), dtype=torch.float32, device="cuda", requires_grad=True)
        r.test_barrier_timeout(0, 2, TIMEOUT_NS)
        E = autograd.unrolled_warp_energy(u0, r, 5)
        with pytest.raises(mreg.MregError) as e:
            E.backward()
        assert e.value.status == mreg.MREG_ERR_DEVICE_CHECK
        r.reset()
        u1 = torch.zeros_like(u0, requires_grad=True)
        E = autograd.unrolled_warp_energy(u1, r, 5)
        E.backward()
        assert torch.isfinite(u1.grad).all()


def test_timeout_hook_validates_its_arguments(mreg, c0):
    with _reg(mreg, c0, "S1") as r:
        grid = r.stats()["grid_blocks"]
        for args in [(-1, 1, TIMEOUT_NS), (grid, 1, TIMEOUT_NS), (0, 0, TIMEOUT_NS),
                     (0, 1, 10), (0, 1, 3_000_000_000)]:
            with pytest.raises(mreg.MregError) as e:
                r.test_barrier_timeout(*args)
            assert e.value.status == mreg.MREG_ERR_INVALID_ARG
