"""The standalone system-matrix product (mreg_apply_operator and its batched
form) against the oracle's matrices in FP64.

S1: A = (1+l) D_m - l W; S2: A = M + l K (Eq. 1, 7, 11-13).  The product is
FP32 with fused multiply-adds over rows of ~7 entries, so each y_i is within
a few FP32 ulps of sum_j |A_ij| |x_j| (tolerance 1e-6 of that, per entry).
"""
import numpy as np
import pytest

from oracle import register
from paper_1411_2141_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def _matrix(case, mode, grad):
    pb = register.Problem(case.V, case.T, case.Re, case.Te, case.spec.alpha, case.spec.tau,
                          mode, grad)
    if mode == "S2":   # the FP32 entries the library holds, as FP64
        return (pb.M + pb.lam * pb.K).tocsr().astype(np.float32).astype(np.float64)
    return pb.Asys.tocsr()


def _check(A, x, y):
    ref = A @ x
    scale = abs(A) @ np.abs(x)
    assert (np.abs(y - ref) <= 1e-6 * scale + 1e-30).all()


@pytest.mark.parametrize("mode,grad", [("S1", "G0"), ("S2", "G1")])
def test_operator_matches_the_oracle_matrix(mreg, c0, mode, grad):
    A = _matrix(c0, mode, grad)
    rng = np.random.default_rng(3)
    x = rng.normal(scale=3.0, size=(c0.n_nodes, 2)).astype(np.float32)
    with mreg.Registration(c0.V, c0.T, c0.Re, c0.Te, c0.spec.alpha, c0.spec.tau, mode=mode,
                           grad=grad) as r:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        r.apply_operator(xd, yd)
        y1 = yd.cpu().numpy().astype(np.float64)
        r.apply_operator(xd, yd)   # bitwise repeatable
        assert np.array_equal(yd.cpu().numpy().astype(np.float64), y1)
        with pytest.raises(mreg.MregError):
            r.apply_operator(xd, xd)
    _check(A, x.astype(np.float64), y1)


def test_operator_rejects_the_explicit_mode(mreg, c0):
    with mreg.Registration(c0.V, c0.T, c0.Re, c0.Te, 0.1, 1.0, mode="S0") as r:
        x = torch.zeros((c0.n_nodes, 2), dtype=torch.float32, device="cuda")
        with pytest.raises(mreg.MregError) as e:
            r.apply_operator(x, torch.empty_like(x))
        assert e.value.status == mreg.MREG_ERR_INVALID_ARG


@pytest.mark.parametrize("mode,grad", [("S1", "G0"), ("S2", "G1")])
def test_batched_operator_matches_every_pair(mreg, mode, grad):
    """The batched product (sliced-ELLPACK rows) against the oracle's matrix
    of every pair, and bitwise against the one-pair product (CSR rows): both
    sum a row's entries in the same order with the same fused operations.
    The pairs' node counts leave ragged last slices of 32 rows."""
    cases = inputs.make_cases(inputs.batched_specs(3, 6))
    assert any(c.n_nodes % 32 for c in cases)
    rng = np.random.default_rng(4)
    xs = [rng.normal(scale=3.0, size=(c.n_nodes, 2)).astype(np.float32) for c in cases]
    with mreg.Batch([(c.V, c.T, c.Re, c.Te) for c in cases], cases[0].spec.alpha,
                    cases[0].spec.tau, mode=mode, grad=grad) as b:
        xd = torch.from_numpy(np.concatenate(xs)).cuda()
        yd = torch.full_like(xd, float("nan"))
        b.apply_operator(xd, yd)
        y = yd.cpu().numpy()
        yd2 = torch.full_like(xd, float("nan"))
        b.apply_operator(xd, yd2)   # the layout is built once; bitwise repeatable
        assert np.array_equal(yd2.cpu().numpy(), y)
    off = 0
    for c, x in zip(cases, xs):
        yc = y[off:off + c.n_nodes]
        _check(_matrix(c, mode, grad), x.astype(np.float64), yc.astype(np.float64))
        with mreg.Registration(c.V, c.T, c.Re, c.Te, c.spec.alpha, c.spec.tau, mode=mode,
                               grad=grad) as r:
            x1 = torch.from_numpy(x).cuda()
            y1 = torch.empty_like(x1)
            r.apply_operator(x1, y1)
            assert np.array_equal(y1.cpu().numpy(), yc)
        off += c.n_nodes
    assert off == len(y)
