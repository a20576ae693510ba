"""The seeded input generators shared by both sides of the parity tests.

The CUDA path receives FP32 points and parameters and the oracle FP64, so the
generated values must survive the FP32 round trip exactly: then both sides
compute on identical inputs.
"""
import numpy as np

from oracle import pyoracle as O
from tests import inputs


def _on_lattice_inside(p):
    k = (p + 1.0) / inputs.Q
    return np.all(k == np.round(k)) and k.min() >= 1 and k.max() <= 2**23 - 1


def test_points_are_lattice_points_inside_the_cube_and_exact_in_fp32():
    p = inputs.mixed_points(500, 300, seed=4)
    assert p.shape == (500 + 300 + len(inputs.boundary_points()), 3)
    assert _on_lattice_inside(p)
    assert np.all(np.abs(p) < 1.0)
    assert np.array_equal(p.astype(np.float32).astype(np.float64), p)
    # the hand-placed points reach the last lattice point before the faces
    assert np.max(np.abs(inputs.boundary_points())) == 1.0 - inputs.Q


def test_shell_points_straddle_the_benchmark_interfaces():
    p = inputs.shell_points(2000, seed=5)
    r = np.linalg.norm(p, axis=1)
    assert r.min() >= 0.35 - 1e-6 and r.max() <= 0.65 + 1e-6
    assert np.mean(r < 0.5) > 0.3 and np.mean(r > 0.5) > 0.3


def test_generators_are_deterministic_per_seed():
    assert np.array_equal(inputs.mixed_points(50, 20, 7), inputs.mixed_points(50, 20, 7))
    assert not np.array_equal(inputs.uniform_points(50, 7), inputs.uniform_points(50, 8))
    assert np.array_equal(inputs.glorot_params(16, 2, 3), inputs.glorot_params(16, 2, 3))


def test_glorot_parameters_follow_the_layout_and_bounds():
    width, n_hidden = 16, 3
    th = inputs.glorot_params(width, n_hidden, seed=1)
    pr = O.make_problem(n_hidden=n_hidden, width=width)
    assert th.dtype == np.float32 and len(th) == 2 * O.params_per_net(pr)
    dims = [(3, width)] + [(width, width)] * (n_hidden - 1) + [(width, 1)]
    off = 0
    for _ in range(2):
        for fi, fo in dims:
            a = np.sqrt(6.0 / (fi + fo))
            w = th[off:off + fi * fo]
            assert np.all(np.abs(w) <= a) and np.abs(w).max() > 0.5 * a
            off += fi * fo
            assert np.all(th[off:off + fo] == 0.0)  # zero biases by default
            off += fo
    assert off == len(th)
