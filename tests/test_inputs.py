"""The seeded input generator: reproducible, and its meshes are valid inputs."""
import numpy as np

from paper_1411_2141_gb300 import inputs


def test_generator_is_deterministic():
    s = inputs.CaseSpec(side=40, n_nodes=150, seed=3)
    a = inputs.make_case(s)
    b = inputs.make_case(s)
    for x, y in ((a.Re, b.Re), (a.Te, b.Te), (a.V, b.V), (a.T, b.T)):
        assert np.array_equal(x, y)


def test_mesh_is_valid_and_ccw():
    for spec in (inputs.CaseSpec(side=40, n_nodes=150, seed=3),
                 inputs.CaseSpec(side=64, n_nodes=300, seed=4, n_ellipses=3, supersample=2)):
        c = inputs.make_case(spec)
        V = c.V.astype(np.float64)
        s = spec.side
        assert V.min() >= 0 and V.max() <= s - 1
        a = V[c.T]
        area2 = ((a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1])
                 - (a[:, 1, 1] - a[:, 0, 1]) * (a[:, 2, 0] - a[:, 0, 0]))
        assert area2.min() > 0
        np.testing.assert_allclose(area2.sum() / 2, (s - 1) ** 2, rtol=1e-9)
        assert len(np.unique(c.T)) == len(V)
        assert abs(len(V) - spec.n_nodes) <= 0.02 * spec.n_nodes + 4
        d = np.sqrt(np.sum((V[:, None, :] - V[None, :, :]) ** 2, -1)) + np.eye(len(V)) * 9
        assert d.min() >= 0.75


def test_config_shapes():
    assert inputs.config_spec(1).side == 512 and inputs.config_spec(1).n_nodes == 20000
    specs = inputs.batched_specs(3, count=8)
    assert all(96 <= s.side <= 768 for s in specs)
