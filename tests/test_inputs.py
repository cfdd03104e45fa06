"""The seeded input module that both the CUDA path and the oracle read: it is
deterministic, its vectors are in the documented orders and its workload
recipes have the stated shapes and value distributions."""
import numpy as np
import pytest

from oracle import geometry
from paper_1608_02461_gb300 import inputs


@pytest.mark.parametrize("name", sorted(inputs.WORKLOADS))
def test_workload_rhs_is_deterministic_and_shaped(name):
    w = inputs.WORKLOADS[name]
    a = inputs.workload_rhs(name)
    b = inputs.workload_rhs(name)
    assert a.dtype == np.complex128 and a.shape == (w["n"] ** 3,)
    assert np.array_equal(a, b)
    assert np.all(np.isfinite(a))


def test_node_coords_follow_the_interior_order():
    for n in (3, 7):
        assert np.array_equal(inputs.node_coords(n), geometry.interior_nodes(n))


def test_gaussian_recipe():
    """Eight Gaussians of width 0.05 and unit amplitude, centres in
    [0.2, 0.8]^3, over a uniform[-1, 1] background."""
    n, seed = 24, 2
    f = inputs.rhs("gaussians", n, seed).real
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, (8, 3))
    bg = rng.uniform(-1.0, 1.0, n ** 3)
    assert np.all((centres >= 0.2) & (centres <= 0.8))
    bumps = f - bg
    assert bumps.min() >= 0 and bumps.max() <= 8.0 + 1e-12
    # far from every centre the bumps vanish
    x = inputs.node_coords(n)
    dmin = np.min(np.linalg.norm(x[:, None, :] - centres[None, :, :], axis=-1), axis=1)
    assert np.all(bumps[dmin > 0.5] < 1e-10)


def test_uniform_and_complex_normal_statistics():
    u = inputs.rhs("uniform_real", 32, 1)
    assert np.all(u.imag == 0) and u.real.min() >= -1 and u.real.max() <= 1
    assert abs(u.real.mean()) < 0.01
    z = inputs.complex_normal(200000, 5)
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01


def test_batched_problem_set():
    probs = inputs.batched_problems()
    assert len(probs) == 48
    assert probs == inputs.batched_problems()
    for q in probs:
        assert q["n"] in (24, 32, 48, 64, 96) and q["p"] in (4, 6)
        assert 4.0 <= q["k"] <= min(32.0, 2 * np.pi * (q["n"] + 1) / 8.0)
