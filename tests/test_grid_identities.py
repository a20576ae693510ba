"""Identities the GPU grid solver relies on, checked on the oracle's dense
assembly of the grid system (CPU only)."""
import numpy as np

from oracle import pyoracle as O


def test_scaled_cg_iterates_equal_jacobi_pcg_on_the_oracle_system():
    """The identity the GPU grid solver relies on: CG on the Jacobi-scaled system
    D^-1/2 A D^-1/2 x^ = D^-1/2 b gives the iterates x = D^-1/2 x^ of Jacobi PCG
    on A, and ||b - A x|| = (sum d r^2)^1/2 with r^ the scaled residual."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    n = 8
    m = (n - 1) ** 3
    A, b = O.grid_assemble_dense(pr, n)
    d = np.diag(A).copy()
    s = 1.0 / np.sqrt(d)
    As, bs = A * s[:, None] * s[None, :], b * s
    # Jacobi PCG on A
    x = np.zeros(m); r = b.copy(); z = r / d; p = z.copy(); rz = r @ z
    # CG on the scaled system
    xs = np.zeros(m); rs = bs.copy(); ps = rs.copy(); rr = rs @ rs
    for _ in range(25):
        Ap = A @ p; a = rz / (p @ Ap); x += a * p; r -= a * Ap
        z = r / d; rz_new = r @ z; p = z + (rz_new / rz) * p; rz = rz_new
        Aps = As @ ps; a_s = rr / (ps @ Aps); xs += a_s * ps; rs -= a_s * Aps
        rr_new = rs @ rs; ps = rs + (rr_new / rr) * ps; rr = rr_new
        assert np.max(np.abs(x - s * xs)) <= 1e-10 * np.max(np.abs(x))
        assert abs(np.linalg.norm(b - A @ x) - np.sqrt(d @ rs ** 2)) <= 1e-9 * np.linalg.norm(b)
