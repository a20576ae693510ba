"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the tests.

Holds none of the method's arithmetic: collocation points on the 2^-22 lattice
(uniform in the cube, or uniform in a spherical shell that straddles the
interfaces of the benchmark geometries), a few hand-placed points next to the
cube boundary, and Glorot-uniform network parameters.
"""
import numpy as np

Q = 2.0 ** -22


def lattice(x):
    k = np.clip(np.round((np.asarray(x, np.float64) + 1.0) / Q), 1, 2**23 - 1)
    return -1.0 + k * Q


def uniform_points(n, seed):
    rng = np.random.default_rng(seed)
    return -1.0 + rng.integers(1, 2**23, size=(n, 3)).astype(np.float64) * Q


def shell_points(n, seed, r_lo=0.35, r_hi=0.65):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = rng.uniform(r_lo, r_hi, size=n)
    return lattice(d * r[:, None])


def boundary_points():
    a = 1.0 - Q
    return lattice(np.array([[a, 0.1, -0.2], [-a, -a, 0.3], [0.2, a, -a], [0.97, -0.99, 0.5],
                             [-0.999, 0.0, 0.0], [0.0, 0.0, 1.0 - 2 * Q]]))


def mixed_points(n_uniform, n_shell, seed):
    return np.concatenate([uniform_points(n_uniform, seed), shell_points(n_shell, seed + 1),
                           boundary_points()])


def glorot_params(width, n_hidden, seed, bias_scale=0.0):
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(2):
        dims = [(3, width)] + [(width, width)] * (n_hidden - 1) + [(width, 1)]
        for fi, fo in dims:
            a = np.sqrt(6.0 / (fi + fo))
            parts.append(rng.uniform(-a, a, size=fi * fo))
            parts.append(rng.uniform(-bias_scale, bias_scale, size=fo))
    return np.concatenate(parts).astype(np.float32)
