"""Pins of the FP64 CPU oracle against facts fixed by the paper or by mathematics.

None of these checks re-types an oracle formula: each compares the oracle with
a closed form, a brute-force count, a textbook special case, a published
known-answer vector or a convergence order.  Citations are to arXiv 2210.14907
(Sec. 2: the interface problem; Sec. 3 / Fig. 2: the NBM cell, residual,
preconditioner, aggregation and Adam).
"""
import math
import os

import numpy as np
import pytest

from oracle import pyoracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al. 2011)."""
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert O.philox(r[0:4], r[4:6]) == r[6:10]


# ------------------------------------------------------ linear-cell fractions
def _mc_simplex_fraction(vals, n, rng):
    """Brute force: uniform points of the simplex, sign of the linear interpolant."""
    d = len(vals)
    lam = rng.dirichlet(np.ones(d), size=n)
    return float(np.mean(lam @ np.asarray(vals) <= 0.0))


@pytest.mark.parametrize("seed", range(6))
def test_fractions_match_monte_carlo(seed):
    rng = np.random.default_rng(100 + seed)
    n = 400_000
    tol = 5.0 / math.sqrt(n)
    # force every sign pattern: 1, 2 negatives for triangles; 1, 2, 3 for tets
    for k in (1, 2):
        v = np.abs(rng.normal(size=3)) + 0.05
        v[:k] *= -1
        rng.shuffle(v)
        assert abs(O.tri_fraction(*v) - _mc_simplex_fraction(v, n, rng)) < tol
    for k in (1, 2, 3):
        v = np.abs(rng.normal(size=4)) + 0.05
        v[:k] *= -1
        rng.shuffle(v)
        assert abs(O.tet_fraction(*v) - _mc_simplex_fraction(v, n, rng)) < tol


def test_fraction_symmetries():
    rng = np.random.default_rng(7)
    for _ in range(200):
        v = rng.normal(size=4)
        t = v[:3]
        # complement: the <=0 part of v and of -v tile the simplex (no zero values here)
        assert abs(O.tet_fraction(*v) + O.tet_fraction(*(-v)) - 1.0) < 1e-12
        assert abs(O.tri_fraction(*t) + O.tri_fraction(*(-t)) - 1.0) < 1e-12
        # positive homogeneity
        c = float(np.exp(rng.normal()))
        assert abs(O.tet_fraction(*(c * v)) - O.tet_fraction(*v)) < 1e-12
    # symmetric two-two split halves the tetrahedron
    assert abs(O.tet_fraction(-1, -1, 1, 1) - 0.5) < 1e-15
    assert O.tet_fraction(0, 0, 1, 1) == 0.0  # zero values count as minus side


# --------------------------------------------------------- cell geometry ----
def _band_points(pr, n, half_width, rng):
    """points at radial offset t, |t| < half_width, from the interface along rays"""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    t = rng.uniform(-half_width, half_width, size=n)
    out = []
    for di, ti in zip(d, t):
        lo, hi = 0.2, 0.8
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if O.phi(pr, mid * di) <= 0:
                lo = mid
            else:
                hi = mid
        out.append((lo + ti) * di)
    return np.array(out)


def test_sphere_volume_and_area_converge():
    """Sum of cell volume fractions -> (4/3) pi r^3; interface area -> 4 pi r^2 (r = 1/2)."""
    errs_v, errs_a = [], []
    for n in (32, 64):
        h = 2.0 / n
        pr = O.make_problem(geometry=O.GEOM_SPHERE, h=h)
        c = -1.0 + h * (np.arange(n) + 0.5)
        X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
        R = np.sqrt(X**2 + Y**2 + Z**2)
        band = np.abs(R - 0.5) < h  # all cells that can be cut (half-diagonal < h)
        vol = float(np.sum(R[~band] < 0.5)) * h**3
        area = 0.0
        for p in np.stack([X[band], Y[band], Z[band]], axis=1):
            g = O.cell_geometry(pr, p, h)
            vol += g["V"][0] * h**3
            area += g["S"] * h**2
        errs_v.append(abs(vol - 4.0 / 3.0 * math.pi / 8.0))
        errs_a.append(abs(area - math.pi))
    assert errs_v[1] < 2e-3 and errs_a[1] < 5e-3
    assert errs_v[0] / errs_v[1] > 3.8 and errs_a[0] / errs_a[1] > 3.8  # second order


def _grid_nodes(n):
    g = -1.0 + np.arange(n + 1) * 2.0 / n
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)  # x fastest


def test_mesh_level_set_reproduces_trilinear_functions():
    """Sec. 3 level set on a coarse mesh: trilinear interpolation of the node
    values is exact for every trilinear function, and so is its gradient."""
    rng = np.random.default_rng(31)
    a = rng.normal(size=8)

    def f(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return (a[0] + a[1] * X + a[2] * Y + a[3] * Z + a[4] * X * Y + a[5] * X * Z
                + a[6] * Y * Z + a[7] * X * Y * Z)

    def grad(x):
        X, Y, Z = x
        return np.array([a[1] + a[4] * Y + a[5] * Z + a[7] * Y * Z,
                         a[2] + a[4] * X + a[6] * Z + a[7] * X * Z,
                         a[3] + a[5] * X + a[6] * Y + a[7] * X * Y])

    pr = O.make_problem(geometry=O.GEOM_GRID, phi_grid=f(_grid_nodes(6)))
    for x in np.concatenate([rng.uniform(-1, 1, size=(200, 3)), [[1.0, 1.0, 1.0], [-1, 0.2, 1]]]):
        assert abs(O.phi(pr, x) - f(x)) < 1e-13
        assert np.allclose(O.grad_phi(pr, x), grad(x), atol=1e-12)


def test_mesh_level_set_of_the_sphere_converges():
    """The sphere's level set stored at the nodes of 8^3, 16^3 and 32^3 meshes: the
    enclosed volume and the interface area (cells of spacing 1/32) approach the
    sphere's at second order in the mesh spacing."""
    h = 2.0 / 64
    c = -1.0 + h * (np.arange(64) + 0.5)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    R = np.sqrt(X**2 + Y**2 + Z**2)
    band = np.abs(R - 0.5) < 0.2
    pts = np.stack([X[band], Y[band], Z[band]], axis=1)
    errs_v, errs_a = [], []
    for n in (8, 16, 32):
        x = _grid_nodes(n)
        pr = O.make_problem(geometry=O.GEOM_GRID, h=h,
                            phi_grid=np.sqrt((x ** 2).sum(1)) - 0.5)
        vol = float(np.sum(R[~band] < 0.5)) * h**3
        area = 0.0
        for p in pts:
            g = O.cell_geometry(pr, p, h)
            vol += g["V"][0] * h**3
            area += g["S"] * h**2
        errs_v.append(abs(vol - 4.0 / 3.0 * math.pi / 8.0))
        errs_a.append(abs(area - math.pi))
    assert errs_v[0] / errs_v[1] > 3.0 and errs_v[1] / errs_v[2] > 3.0
    assert errs_a[2] < 0.02 and errs_a[0] / errs_a[2] > 6.0


def test_cut_cell_consistency_on_a_mesh_level_set():
    """A plane stored on a coarse mesh (represented exactly): with the exact u^+-,
    cut-cell rows are O(h^2) and the value jump is met exactly."""
    x = _grid_nodes(4)
    plane = 0.3 * x[:, 0] - 0.2 * x[:, 1] + 0.9 * x[:, 2] - 0.1
    rng = np.random.default_rng(32)
    mx = []
    for h in (1 / 32, 1 / 64, 1 / 128):
        pr = O.make_problem(geometry=O.GEOM_GRID, h=h, mu_minus=1.0, mu_plus=10.0,
                            phi_grid=plane)
        res = []
        while len(res) < 100:
            p = rng.uniform(-0.8, 0.8, size=3)
            q = p - (O.phi(pr, p) + rng.uniform(-0.3, 0.3) * h) * np.array([0.3, -0.2, 0.9]) / 0.94
            t = O.point_terms(pr, None, q, mode=1)
            if t["cut"]:
                res.append(t)
        mx.append(max(abs(r["B"]) for r in res))
        assert max(abs(r["J"]) for r in res) < 1e-13
    assert mx[0] / mx[1] > 3.4 and mx[1] / mx[2] > 3.4


def test_uncut_cells_are_exactly_zero_one():
    pr = O.make_problem(geometry=O.GEOM_SPHERE, h=1.0 / 16)
    for p, s in (([0.0, 0.0, 0.0], 0), ([0.9, 0.9, 0.9], 1), ([0.2, -0.1, 0.05], 0)):
        g = O.cell_geometry(pr, p)
        assert g["cut"] == 0 and g["phase"] == s
        assert g["V"][s] == 1.0 and g["V"][1 - s] == 0.0
        assert np.all(g["A"][s] == 1.0) and np.all(g["A"][1 - s] == 0.0) and g["S"] == 0.0


def test_shared_face_fractions_agree_between_neighbour_cells():
    """A face seen from both cells of a grid is split the same way (consistent Kuhn split)."""
    rng = np.random.default_rng(11)
    h = 1.0 / 16
    pr = O.make_problem(geometry=O.GEOM_FLOWER, h=h)
    hits = 0
    for p in _band_points(pr, 60, 0.5 * h, rng):
        p = np.round(p / h) * h  # put the cell centres on a grid of spacing h
        for ax in range(3):
            q = p.copy()
            q[ax] += h
            a = O.cell_geometry(pr, p, h)["A"][0][2 * ax + 1]
            b = O.cell_geometry(pr, q, h)["A"][0][2 * ax]
            assert a == b
            hits += 0.0 < a < 1.0
    assert hits > 10


def test_projection_lands_on_interface():
    rng = np.random.default_rng(5)
    for geom in (O.GEOM_SPHERE, O.GEOM_FLOWER):
        pr = O.make_problem(geometry=geom, h=1.0 / 64)
        for p in _band_points(pr, 100, 0.4 / 64, rng):
            g = O.cell_geometry(pr, p)
            if g["cut"] and g["S"] > 0:
                assert abs(O.phi(pr, g["xg"])) < 1e-9
                assert np.linalg.norm(g["xg"] - p) < 1.0 / 64


# ---------------------------------------------- manufactured problem (Sec. 2)
def _fd_grad(f, x, e=1e-5):
    g = np.zeros(3)
    for i in range(3):
        d = np.zeros(3)
        d[i] = e
        g[i] = (f(x + d) - f(x - d)) / (2 * e)
    return g


def test_level_set_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    for geom in (O.GEOM_SPHERE, O.GEOM_FLOWER):
        pr = O.make_problem(geometry=geom)
        for _ in range(50):
            x = rng.uniform(-0.9, 0.9, size=3)
            if np.hypot(x[0], x[1]) < 0.05:
                continue
            fd = _fd_grad(lambda y: O.phi(pr, y), x)
            assert np.allclose(O.grad_phi(pr, x), fd, atol=1e-7)


def test_rhs_and_jumps_match_finite_differences():
    """f = k u - mu Lap(u); alpha = [u]; beta = [mu d_n u] (Sec. 2), by FD of u."""
    rng = np.random.default_rng(3)
    pr = O.make_problem(geometry=O.GEOM_FLOWER, mu_minus=1.0, mu_plus=100.0, k_minus=0.3,
                        k_plus=2.0)
    e = 1e-3
    for _ in range(30):
        x = rng.uniform(-0.8, 0.8, size=3)
        for s, mu, k in ((0, 1.0, 0.3), (1, 100.0, 2.0)):
            lap = sum((O.exact_u(pr, s, x + e * ei) - 2 * O.exact_u(pr, s, x)
                       + O.exact_u(pr, s, x - e * ei)) / e**2 for ei in np.eye(3))
            assert abs(O.rhs_f(pr, s, x) - (k * O.exact_u(pr, s, x) - mu * lap)) < 1e-4
            assert np.allclose(O.exact_grad_u(pr, s, x),
                               _fd_grad(lambda y: O.exact_u(pr, s, y), x), atol=1e-8)
    for p in _band_points(pr, 30, 0.0, rng):
        if np.hypot(p[0], p[1]) < 0.05:
            continue
        n = O.grad_phi(pr, p)
        n /= np.linalg.norm(n)
        dn = [(O.exact_u(pr, s, p + 1e-5 * n) - O.exact_u(pr, s, p - 1e-5 * n)) / 2e-5
              for s in (0, 1)]
        assert abs(O.beta(pr, p) - (100.0 * dn[1] - 1.0 * dn[0])) < 1e-6
        assert abs(O.alpha(pr, p) - (O.exact_u(pr, 1, p) - O.exact_u(pr, 0, p))) < 1e-15


def test_sec41_pair_matches_finite_differences():
    """Sec. 4.1 pair (variable mu): f = k u - div(mu grad u) against a central
    difference of the flux mu grad u; beta = [mu d_n u] with mu at the point."""
    rng = np.random.default_rng(23)
    pr = O.make_problem(geometry=O.GEOM_SPHERE, k_minus=0.4, k_plus=1.1, solution=O.SOL_SEC41)
    e = 1e-3
    for _ in range(30):
        x = rng.uniform(-0.8, 0.8, size=3)
        for s, k in ((0, 0.4), (1, 1.1)):
            div = 0.0
            for ei in np.eye(3):
                fp = O.mu(pr, s, x + 0.5 * e * ei) * (O.exact_u(pr, s, x + e * ei) - O.exact_u(pr, s, x))
                fm = O.mu(pr, s, x - 0.5 * e * ei) * (O.exact_u(pr, s, x) - O.exact_u(pr, s, x - e * ei))
                div += (fp - fm) / e**2
            assert abs(O.rhs_f(pr, s, x) - (k * O.exact_u(pr, s, x) - div)) < 1e-5
            assert np.allclose(O.exact_grad_u(pr, s, x),
                               _fd_grad(lambda y: O.exact_u(pr, s, y), x), atol=1e-8)
    for p in _band_points(pr, 30, 0.0, rng):
        n = O.grad_phi(pr, p)
        n /= np.linalg.norm(n)
        dn = [(O.exact_u(pr, s, p + 1e-5 * n) - O.exact_u(pr, s, p - 1e-5 * n)) / 2e-5
              for s in (0, 1)]
        assert abs(O.beta(pr, p) - (O.mu(pr, 1, p) * dn[1] - O.mu(pr, 0, p) * dn[0])) < 1e-6


# ------------------------------------------------ residual rows (Sec. 3) ----
def test_balance_row_vanishes_for_quadratic_solution():
    """No interface, constant mu: the 7-point FV row is exact for quadratics."""
    rng = np.random.default_rng(4)
    pr = O.make_problem(geometry=O.GEOM_ALL_PLUS, mu_plus=10.0, k_plus=1.5, h=1.0 / 16)
    pts = np.concatenate([rng.uniform(-1, 1, size=(200, 3)),
                          rng.uniform(0.96, 0.999, size=(20, 3))])  # boundary neighbours too
    for p in pts:
        t = O.point_terms(pr, None, p, mode=1)
        assert abs(t["B"]) < 1e-12 * 10.0
        assert t["has_jump"] == 0


def test_preconditioner_is_jacobi_diagonal_of_7_point_operator():
    for mu, k, h in ((10.0, 0.0, 1 / 16), (1.0, 3.0, 1 / 64)):
        pr = O.make_problem(geometry=O.GEOM_ALL_PLUS, mu_plus=mu, k_plus=k, h=h)
        t = O.point_terms(pr, None, [0.1, 0.2, 0.3], mode=1)
        assert abs(t["D"] - (6 * mu + h * h * k)) < 1e-14


@pytest.mark.parametrize("geom,sol", [(O.GEOM_ALL_MINUS, O.SOL_BENCH),
                                      (O.GEOM_ALL_MINUS, O.SOL_SEC41),
                                      (O.GEOM_ALL_PLUS, O.SOL_SEC41)])
def test_uncut_truncation_is_fourth_order_in_B(geom, sol):
    """B = h^2 x (PDE residual) so its truncation error is O(h^4) away from Gamma."""
    rng = np.random.default_rng(6)
    pts = rng.uniform(-0.8, 0.8, size=(40, 3))
    mx = []
    for h in (1 / 8, 1 / 16, 1 / 32):
        pr = O.make_problem(geometry=geom, mu_minus=2.0, h=h, solution=sol)
        mx.append(max(abs(O.point_terms(pr, None, p, mode=1)["B"]) for p in pts))
    assert mx[0] / mx[1] > 15.0 and mx[1] / mx[2] > 15.5


@pytest.mark.parametrize("sol", [O.SOL_BENCH, O.SOL_SEC41])
def test_cut_cell_consistency_is_second_order(sol):
    """Exact u^+- in cut cells: B = O(h^2); this fails if the interface flux term,
    its sign, a face fraction or a volume fraction is wrong (and, for the Sec. 4.1
    pair, if mu is not taken at the face centres and at x_G)."""
    rng = np.random.default_rng(8)
    mx = []
    for h in (1 / 32, 1 / 64, 1 / 128):
        pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0, h=h,
                            solution=sol)
        res = [O.point_terms(pr, None, p, mode=1) for p in _band_points(pr, 150, 0.5 * h, rng)]
        assert all(r["cut"] for r in res)
        mx.append(max(abs(r["B"]) for r in res))
        assert max(abs(r["J"]) for r in res) < 1e-13  # value jump met exactly
    assert mx[0] / mx[1] > 3.4 and mx[1] / mx[2] > 3.4



@pytest.mark.parametrize("sol", [O.SOL_BENCH, O.SOL_SEC41])
def test_jump_row_vanishes_for_the_exact_pair_on_the_flower(sol):
    """The value-jump row J = U+(x_G) - U-(x_G) - alpha(x_G) is zero to rounding
    when U is the manufactured pair, on the flower interface too (x_G from the
    Newton projection of a non-distance level set)."""
    rng = np.random.default_rng(9)
    h = 1 / 64
    pr = O.make_problem(geometry=O.GEOM_FLOWER, mu_minus=1.0, mu_plus=100.0, h=h, solution=sol)
    res = [O.point_terms(pr, None, p, mode=1) for p in _band_points(pr, 120, 0.5 * h, rng)]
    cut = [r for r in res if r["cut"] and r["has_jump"]]
    assert len(cut) > 100
    assert max(abs(r["J"]) for r in cut) < 1e-13


# --------------------------------------------------------------- network ----
def test_mlp_textbook_cases():
    pr = O.make_problem(n_hidden=2, width=4)
    P = O.params_per_net(pr)
    assert P == 4 * 4 + (4 * 4 + 4) + 4 + 1
    # 5 hidden layers of 10 units, two nets: 982 parameters (Sec. 4.1)
    assert 2 * O.params_per_net(O.make_problem(n_hidden=5, width=10)) == 982
    th = np.zeros(P)
    x = np.array([0.3, -0.2, 0.7])
    th[-1] = 0.25  # output bias only
    assert O.mlp_eval(pr, th, x) == 0.25
    # one active path: unit 0 of layer 1 reads x_1, feeds unit 0 of layer 2, output weight 2
    th[:] = 0.0
    th[0 * 3 + 1] = 0.8      # W1[0][1]
    th[12 + 0] = 0.1         # b1[0]
    off2 = 16
    th[off2 + 0] = 1.3       # W2[0][0]
    th[off2 + 16 + 0] = -0.2  # b2[0]
    th[off2 + 20 + 0] = 2.0  # w[0]
    th[-1] = -0.5
    ref = 2.0 * math.tanh(1.3 * math.tanh(0.8 * x[1] + 0.1) - 0.2) - 0.5
    assert abs(O.mlp_eval(pr, th, x) - ref) < 1e-15
    # the same path with sine activations (Sec. 4.1 networks)
    prs = O.make_problem(n_hidden=2, width=4, activation=O.ACT_SIN)
    ref = 2.0 * math.sin(1.3 * math.sin(0.8 * x[1] + 0.1) - 0.2) - 0.5
    assert abs(O.mlp_eval(prs, th, x) - ref) < 1e-15
    # tiny weights: the network is linear to first order
    rng = np.random.default_rng(0)
    th = rng.normal(size=P) * 1e-4
    lin = O.mlp_eval(pr, th, x)
    assert abs(lin - th[-1]) < 1e-6


# -------------------------------------------------------------- gradient ----
def _small_problem(geom=O.GEOM_SPHERE, solution=O.SOL_BENCH, activation=O.ACT_TANH):
    return O.make_problem(geometry=geom, n_hidden=3, width=8, h=2.0 / 16, mu_minus=1.0,
                          mu_plus=10.0, k_minus=0.5, k_plus=0.2, solution=solution,
                          activation=activation)


@pytest.mark.parametrize("geom,sol,act", [(O.GEOM_SPHERE, O.SOL_BENCH, O.ACT_TANH),
                                          (O.GEOM_FLOWER, O.SOL_BENCH, O.ACT_TANH),
                                          (O.GEOM_SPHERE, O.SOL_SEC41, O.ACT_SIN)])
def test_hand_gradient_matches_central_differences(geom, sol, act):
    """d(loss)/d(theta) by the hand-derived reverse mode vs central FD, step 1e-6."""
    pr = _small_problem(geom, sol, act)
    rng = np.random.default_rng(9)
    P = 2 * O.params_per_net(pr)
    th = rng.normal(size=P) * 0.5
    pts = O.sample_points(pr, 1, 1, 200, 56)
    pts = np.concatenate([pts, [[0.97, 0.1, -0.2], [-0.1, -0.95, 0.99]]])  # boundary rows
    L, g = O.loss_grad(pr, th, pts)
    assert abs(L - O.loss(pr, th, pts)) < 1e-14 * max(1.0, L)
    Pn = P // 2
    idx = list(rng.choice(P, size=64, replace=False)) + [Pn - 1, P - 1]
    for j in idx:
        e = np.zeros(P)
        e[j] = 1e-6
        fd = (O.loss(pr, th + e, pts) - O.loss(pr, th - e, pts)) / 2e-6
        assert abs(fd - g[j]) <= 1e-6 * np.max(np.abs(g)) + 1e-6 * abs(g[j])


def test_loss_is_mean_of_point_residuals_and_splits_over_ranks():
    """L = (1/N) sum r_p^2 (aggregation, Sec. 3); count-weighted sub-batch gradients
    sum to the full-batch gradient (the data-parallel exchange, Sec. 3)."""
    pr = _small_problem()
    rng = np.random.default_rng(10)
    th = rng.normal(size=2 * O.params_per_net(pr)) * 0.5
    pts = O.sample_points(pr, 3, 2, 120, 40)
    L, r2 = O.loss(pr, th, pts, want_r2=True)
    assert abs(L - r2.mean()) < 1e-14
    Lf, gf = O.loss_grad(pr, th, pts)
    parts = [pts[:50], pts[50:]]
    gs = sum(len(p) * O.loss_grad(pr, th, p)[1] for p in parts) / len(pts)
    assert np.allclose(gs, gf, rtol=1e-12, atol=1e-15)


def test_refinement_levels_stack_the_rows_of_every_spacing():
    """Implicit refinement (Sec. 3, Fig. 2; reading: the rows of the cells of
    spacing h, h/2, h/4 around the same point are stacked into r_p): the
    multi-level r_p^2 equals the per-point terms of each spacing summed, a point
    can be cut at one level and uncut at another, and the multi-level gradient
    matches central differences of the multi-level loss."""
    pr = _small_problem(O.GEOM_FLOWER)
    rng = np.random.default_rng(14)
    P = 2 * O.params_per_net(pr)
    th = rng.normal(size=P) * 0.5
    pts = O.sample_points(pr, 5, 3, 90, 60)
    q = O.level_problem(pr, 2)
    assert q.h == pr.h / 4 and q.mu_plus == pr.mu_plus and q.geometry == pr.geometry
    L, r2 = O.loss_levels(pr, 2, th, pts, want_r2=True)
    assert abs(L - r2.mean()) < 1e-13 * max(1.0, L)
    n_changed = 0
    for i, p in enumerate(pts):
        terms = [O.point_terms(O.level_problem(pr, lv), th, p) for lv in range(3)]
        ref = sum(t["r2"] for t in terms)
        assert abs(r2[i] - ref) <= 1e-12 * max(1.0, ref)
        n_changed += len({t["cut"] for t in terms}) > 1
    assert n_changed > 0
    Lg, g = O.loss_grad_levels(pr, 2, th, pts)
    assert abs(Lg - L) < 1e-13 * max(1.0, L)
    for j in rng.choice(P, size=24, replace=False):
        e = np.zeros(P)
        e[j] = 1e-6
        fd = (O.loss_levels(pr, 2, th + e, pts) - O.loss_levels(pr, 2, th - e, pts)) / 2e-6
        assert abs(fd - g[j]) <= 1e-6 * np.max(np.abs(g)) + 1e-6 * abs(g[j])


# ------------------------------------------------------------------ Adam ----
def test_adam_closed_form_first_two_steps():
    """Kingma & Ba: with zero state, step 1 moves each weight by lr*g/(|g|+eps)."""
    g1 = np.array([0.3, -2.0, 1e-3, 0.0])
    g2 = np.array([-0.1, -1.0, 2e-3, 0.5])
    th = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    O.adam_step(th, m, v, g1, 1, lr, b1, b2, eps)
    ref1 = np.array([1.0, 2.0, 3.0, 4.0]) - lr * g1 / (np.abs(g1) + eps)
    assert np.allclose(th, ref1, rtol=0, atol=1e-15)
    O.adam_step(th, m, v, g2, 2, lr, b1, b2, eps)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1**2)
    vh = (b2 * (1 - b2) * g1**2 + (1 - b2) * g2**2) / (1 - b2**2)
    assert np.allclose(th, ref1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-15)


# -------------------------------------------------------------- sampling ----
def test_sampler_lattice_band_and_determinism():
    h = 2.0 / 256
    pr = O.make_problem(geometry=O.GEOM_FLOWER, h=h)
    n, nb = 4000, 1200
    pts = O.sample_points(pr, 1, 5, n, nb)
    k = (pts + 1.0) * 2.0**22
    assert np.all(k == np.round(k)) and k.min() >= 1 and k.max() <= 2**23 - 1
    ph = np.array([O.phi(pr, p) for p in pts[n - nb:]])
    assert np.all(np.abs(ph) < 4 * h + 2.0**-21)
    assert np.std(ph) > h  # spread over the band, not collapsed on Gamma
    assert np.array_equal(pts, O.sample_points(pr, 1, 5, n, nb))
    assert not np.array_equal(pts, O.sample_points(pr, 1, 6, n, nb))
    # uniform part: mean ~ 0, variance ~ 1/3 per axis
    u = pts[: n - nb]
    assert np.all(np.abs(u.mean(0)) < 0.05) and np.all(np.abs(u.var(0) - 1 / 3) < 0.03)


# ------------------------------------------------------------ grid scheme ----
def test_grid_matrix_symmetric_positive_definite_and_cg_matches_direct():
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    n = 8
    A, b = O.grid_assemble_dense(pr, n)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    x = np.linalg.solve(A, b)
    st, u, it, rr = O.grid_cg_solve(pr, n, rtol=1e-13, max_iter=1000)
    assert st == 0 and rr <= 1e-13
    ui = u.reshape(n + 1, n + 1, n + 1)[1:-1, 1:-1, 1:-1]  # [k][j][i]
    assert np.allclose(ui.reshape(-1), x, rtol=0, atol=1e-10)


def test_grid_matrix_with_face_centred_variable_mu_is_symmetric():
    """Sec. 4.1 coefficients: the face coefficient mu at the face centre is the same
    seen from both cells of the face, so the grid operator stays symmetric (a
    cell-centred mu would break the symmetry by O(h |grad mu|))."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, solution=O.SOL_SEC41)
    A, b = O.grid_assemble_dense(pr, 8)
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    off = A - np.diag(np.diag(A))
    assert np.ptp(off[off != 0]) > 0.1  # the face weights do vary


def test_grid_second_order_without_interface():
    errs = []
    for n in (8, 16, 32):
        pr = O.make_problem(geometry=O.GEOM_ALL_MINUS, mu_minus=2.0, k_minus=1.0)
        st, u, it, rr = O.grid_cg_solve(pr, n, rtol=1e-12, max_iter=5000)
        assert st == 0
        errs.append(O.grid_error(pr, n, u)[0])
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


@pytest.mark.parametrize("mu_plus", [10.0, 1000.0])
def test_grid_with_interface_is_second_order_on_the_sphere(mu_plus):
    """With the exact node jump, the grid solve of the sphere problem converges
    at second order in L-inf and RMS (error ratios > 3.5 per halving of h).
    A dropped or wrongly signed jump term in the cut rows leaves an O(1) or
    O(h) error and fails this."""
    errs = []
    for n in (16, 32, 64):
        pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=mu_plus)
        st, u, it, rr = O.grid_cg_solve(pr, n, rtol=1e-12, max_iter=40000)
        assert st == 0
        errs.append(O.grid_error(pr, n, u))
    for i in range(2):
        assert errs[i][0] / errs[i + 1][0] > 3.5 and errs[i][1] / errs[i + 1][1] > 3.5


# ------------------------------- extrapolated node jump of the grid scheme ----
# The benchmark pair written out here (not through the oracle): u- = e^x cos y
# sin z, u+ = x^2 + y^2 + z^2, on the sphere |x| = 1/2 (normal x / |x|).
def _um(x):
    return math.exp(x[0]) * math.cos(x[1]) * math.sin(x[2])


def _up(x):
    return float(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)


def _sphere_nodes_near_interface(n, width):
    h = 2.0 / n
    g = -1.0 + np.arange(1, n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    r = np.linalg.norm(x, axis=1)
    return x[np.abs(r - 0.5) <= width * h]


def test_jump_projection_and_distance_on_the_sphere():
    """x_G = x / (2|x|), d = |x| - 1/2 and n = x / |x| in closed form."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    n = 32
    for x in _sphere_nodes_near_interface(n, 2.5)[::7]:
        ok, J0, xg, nrm, ss = O.jump_extrap(pr, x, 2.0 / n)
        r = np.linalg.norm(x)
        assert ok and ss == 0
        assert np.allclose(xg, x / (2 * r), atol=1e-14)
        assert np.allclose(nrm, x / r, atol=1e-14)
    far = np.array([0.0, 0.1, 0.05])  # 0.39 from Gamma: outside the 3h band
    assert not O.jump_extrap(pr, far, 2.0 / n)[0]


@pytest.mark.parametrize("mu_m,mu_p", [(1.0, 10.0), (7.0, 2.0)])
def test_jump_slope_is_the_normal_derivative_jump(mu_m, mu_p):
    """With the small side's exact normal derivative, (J - [u](x_G)) / d is
    d_n u+ - d_n u- at x_G for either ordering of mu (the flux-jump algebra)."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=mu_m, mu_plus=mu_p)
    h = 2.0 / 32
    for x in _sphere_nodes_near_interface(32, 2.0)[::11]:
        ok, _, xg, nrm, ss = O.jump_extrap(pr, x, h)
        d = np.linalg.norm(x) - 0.5
        if abs(d) < 0.2 * h:
            continue
        dn = {0: _fd_grad(_um, xg) @ nrm, 1: _fd_grad(_up, xg) @ nrm}
        assert ss == (0 if mu_m <= mu_p else 1)
        _, J, *_ = O.jump_extrap(pr, x, h, dn[ss])
        G = (J - (_up(xg) - _um(xg))) / d
        assert abs(G - (dn[1] - dn[0])) <= 1e-7 * max(1.0, abs(dn[1] - dn[0]))


def test_jump_extrapolation_orders():
    """At nodes within h of Gamma: the lagged J is off u+ - u- by O(h^2), the
    first-order J (lag dropped) by O(h)."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    e1, e2 = [], []
    for n in (16, 32, 64):
        h = 2.0 / n
        a1 = a2 = 0.0
        for x in _sphere_nodes_near_interface(n, 1.0):
            ok, J0, xg, nrm, ss = O.jump_extrap(pr, x, h)
            assert ok
            Jt = _up(x) - _um(x)
            _, J, *_ = O.jump_extrap(pr, x, h, _fd_grad(_um, xg) @ nrm)
            a1, a2 = max(a1, abs(J0 - Jt)), max(a2, abs(J - Jt))
        e1.append(a1)
        e2.append(a2)
    assert all(1.6 < e1[i] / e1[i + 1] < 2.6 for i in range(2))
    assert all(e2[i] / e2[i + 1] > 3.5 for i in range(2))


def test_fit_recovers_linear_data_exactly():
    """The least-squares fit reproduces the normal derivative of any linear
    node data, on either side and for interface points all around the sphere."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    n = 24
    h = 2.0 / n
    g = -1.0 + np.arange(n + 1) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    rng = np.random.default_rng(12)
    c = rng.normal(size=3)
    u = 0.3 + nodes @ c
    for _ in range(40):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        xg = 0.5 * v
        for s in (0, 1):
            dn = O.fit_dn(pr, n, u, s, xg, v)
            assert dn is not None and abs(dn - c @ v) <= 1e-11


def test_grid_jump_modes():
    """Node jump modes of the grid solve: exact (equal to the plain solve),
    extrapolated with the lagged derivative (second order in L-inf and RMS,
    a contracting fixed point) and first order (the lag dropped)."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    st, u0, *_ = O.grid_cg_solve(pr, 16, rtol=1e-12, max_iter=5000)
    st0, ue, *_ = O.grid_solve_jump(pr, 16, O.JUMP_EXACT, rtol=1e-12, max_iter=5000)
    assert st == st0 == 0 and np.max(np.abs(u0 - ue)) <= 1e-12 * np.max(np.abs(u0))
    lag, first = [], []
    for n in (16, 32, 64):
        st1, u1, it, rr, passes, dj = O.grid_solve_jump(pr, n, O.JUMP_EXTRAP, rtol=1e-12,
                                                        max_iter=20000)
        assert st1 == 0 and 2 <= passes <= 10 and rr <= 1e-12
        st2, u2, *_ = O.grid_solve_jump(pr, n, O.JUMP_FIRST_ORDER, rtol=1e-12, max_iter=20000)
        assert st2 == 0
        lag.append(O.grid_error(pr, n, u1))
        first.append(O.grid_error(pr, n, u2))
    for i in range(2):
        assert lag[i][0] / lag[i + 1][0] > 3.0 and lag[i][1] / lag[i + 1][1] > 3.5
        assert 1.5 < first[i][0] / first[i + 1][0] < 3.0
    # the fixed point contracts: max |J_new - J| falls by > 5x per pass
    djs = [O.grid_solve_jump(pr, 32, O.JUMP_EXTRAP, rtol=1e-12, max_iter=20000, max_passes=k,
                             jtol=0.0)[5] for k in (2, 3, 4, 5)]
    assert all(djs[i] / djs[i + 1] > 5.0 for i in range(3))


def test_grid_jump_equal_mu_and_fallback():
    """Equal mu: G = beta / mu needs no lag, so the second pass changes
    nothing.  A fixed point stopped early falls back to the first-order jump."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=3.0, mu_plus=3.0)
    st, u1, it, rr, passes, dj = O.grid_solve_jump(pr, 16, O.JUMP_EXTRAP, rtol=1e-12,
                                                   max_iter=5000)
    _, u2, *_ = O.grid_solve_jump(pr, 16, O.JUMP_FIRST_ORDER, rtol=1e-12, max_iter=5000)
    assert st == 0 and passes == 2 and dj == 0.0
    assert np.max(np.abs(u1 - u2)) <= 1e-10 * np.max(np.abs(u2))
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    st, u1, it, rr, passes, dj = O.grid_solve_jump(pr, 16, O.JUMP_EXTRAP, rtol=1e-12,
                                                   max_iter=5000, max_passes=2, jtol=1e-12)
    _, u2, *_ = O.grid_solve_jump(pr, 16, O.JUMP_FIRST_ORDER, rtol=1e-12, max_iter=5000)
    assert st == 2 and passes == 2 and dj > 1e-12
    assert np.max(np.abs(u1 - u2)) <= 1e-9 * np.max(np.abs(u2))

