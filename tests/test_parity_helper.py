"""The per-point parity helper (tests/parity.py) on the oracle alone: its
interface-point scale is nonzero exactly for the cut cells that carry a
value-jump row (checked against every point's cell geometry, without the
radius prefilter), and the bound accepts the oracle's own residuals and
rejects one planted 1 % error."""
import numpy as np

from oracle import pyoracle as O
from tests import inputs, parity


def test_jump_scale_marks_exactly_the_cut_cells_with_an_interface():
    for geom, h in ((O.GEOM_SPHERE, 2 / 32), (O.GEOM_FLOWER, 2 / 64)):
        o = O.make_problem(geometry=geom, n_hidden=2, width=16, h=h, mu_minus=1.0,
                           mu_plus=100.0)
        th = inputs.glorot_params(16, 2, seed=1, bias_scale=0.1).astype(np.float64)
        pts = inputs.mixed_points(300, 300, seed=5)
        s = parity.jump_scale(o, th, pts)
        want = np.array([O.cell_geometry(o, p)["cut"] and O.cell_geometry(o, p)["S"] > 0
                         for p in pts])
        assert want.sum() > 10
        assert np.array_equal(s > 0, want)


def test_bound_accepts_the_oracle_and_rejects_a_planted_point_error():
    o = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=2, width=16, h=2 / 32, mu_minus=1.0,
                       mu_plus=10.0)
    th = inputs.glorot_params(16, 2, seed=2, bias_scale=0.1).astype(np.float64)
    pts = inputs.mixed_points(400, 100, seed=6)
    _, r2 = O.loss(o, th, pts, want_r2=True)
    s = parity.jump_scale(o, th, pts)
    tol, tol_j = parity.bf16_tols(2)
    assert parity.worst_ratio(r2, r2, s, tol, tol_j) == 0.0
    bad = r2.copy()
    i = int(np.argmax(r2 * (s == 0)))  # an uncut point with a large residual
    bad[i] *= 1.01 ** 2  # its r 1 % off
    assert parity.worst_ratio(bad, r2, s, tol, tol_j) > 1.0
