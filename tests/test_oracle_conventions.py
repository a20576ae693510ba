"""Pins of the oracle's stated readings and conventions (CPU only).

The paper fixes none of these choices, but the GPU path must reproduce each
one, so each is checked here against something outside the oracle's own
arithmetic:

- the sampler's counter layout and lattice map, as stated in include/nbm.h;
- the band's width and isotropy (statistics of the drawn points);
- the tie rules at phi = 0 and on the faces of the cube;
- the weight lambda of the jump rows;
- the step numbering of the training loop;
- the choice of network and the node order in grid evaluation;
- the agreement of the point rows with the grid rows;
- the grid CG against a library Jacobi-PCG;
- the warm start of the lagged passes;
- the grid error metrics and the boundary values of the grid solution.
"""
import math

import numpy as np
import pytest

from oracle import pyoracle as O

LATTICE = 2.0**-22


# ------------------------------------------------------------- sampling ----
def test_uniform_points_follow_the_documented_counter_layout():
    """A uniform point i of step t is the Philox4x32-10 block at counter
    (i, t mod 2^32, t div 2^32, 0x4E424D31) under the key (seed mod 2^32,
    seed div 2^32).  Word j gives the lattice index k = 1 + floor(w_j (2^23 - 1)
    / 2^32) and the coordinate -1 + k 2^-22.  Philox itself is pinned by the
    published known answers."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, h=2.0 / 128)
    seed, step, n = 0x0123_4567_89AB_CDEF, (5 << 32) + 17, 48
    pts = O.sample_points(pr, seed, step, n, 0)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(n):
        w = O.philox((i, step & 0xFFFFFFFF, step >> 32, 0x4E424D31), key)
        k = [1 + ((w[j] * (2**23 - 1)) >> 32) for j in range(3)]
        assert pts[i].tolist() == [-1.0 + kj * LATTICE for kj in k]


@pytest.mark.parametrize("geom", [O.GEOM_SPHERE, O.GEOM_FLOWER])
def test_band_points_fill_the_shell_uniformly(geom):
    """Band points sit at a signed offset t, uniform on (-4h, 4h), from the
    interface along an isotropic direction.  For both level sets phi equals t
    up to the lattice rounding.  So phi has mean 0, variance (4h)^2 / 3 and
    reaches the band edge, and the directions have mean 0 and E[z^2] = 1/3."""
    h = 2.0 / 64
    pr = O.make_problem(geometry=geom, h=h)
    n = 20000
    pts = O.sample_points(pr, 77, 3, n, n)
    ph = np.array([O.phi(pr, p) for p in pts])
    w = 4.0 * h
    assert np.max(np.abs(ph)) < w + 2.0 * LATTICE and np.max(np.abs(ph)) > 0.99 * w
    assert abs(ph.mean()) < 0.03 * w
    assert abs(ph.var() / (w * w / 3.0) - 1.0) < 0.05
    d = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    assert np.all(np.abs(d.mean(0)) < 0.03)
    assert np.all(np.abs((d * d).mean(0) - 1.0 / 3.0) < 0.02)


# ----------------------------------------------------------- tie rules ----
def test_points_on_the_interface_belong_to_the_minus_side():
    """Reading: the zero level set belongs to Omega-.  Nodes on the sphere
    |x| = 1/2 are exact in binary, so phi is exactly 0 there."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, r0=0.5)
    for x in ([0.5, 0.0, 0.0], [0.0, -0.5, 0.0], [0.0, 0.0, 0.5], [0.3, 0.4, 0.0]):
        assert O.phi(pr, x) == 0.0 and O.phase(pr, x) == 0
    assert O.phase(pr, [0.5 + LATTICE, 0.0, 0.0]) == 1
    assert O.phase(pr, [0.5 - LATTICE, 0.0, 0.0]) == 0


def test_a_neighbour_on_the_cube_face_takes_the_dirichlet_value():
    """A stencil point on the face |x_i| = 1 is boundary data g, not the
    network (Sec. 2: Dirichlet data on the cube).  With both networks
    identically zero and no interface, the row of the point p = (1 - h, y, z)
    is B = -h^2 f(p) - mu g(p + h e_x).  A point a lattice step further in
    has all six neighbours inside, and its row is B = -h^2 f.  The outer
    solution is u+ = |x|^2 (written out here)."""
    h, mu, k = 1.0 / 16, 3.0, 0.5
    pr = O.make_problem(geometry=O.GEOM_ALL_PLUS, n_hidden=2, width=4, h=h, mu_plus=mu,
                        k_plus=k)
    th = np.zeros(2 * O.params_per_net(pr))
    y, z = 0.25, -0.375
    p = np.array([1.0 - h, y, z])
    q = p + np.array([h, 0.0, 0.0])
    assert q[0] == 1.0
    t = O.point_terms(pr, th, p)
    g = q @ q
    assert abs(t["B"] + h * h * O.rhs_f(pr, 1, p) + mu * g) < 1e-14
    p2 = p - np.array([LATTICE, 0.0, 0.0])
    t2 = O.point_terms(pr, th, p2)
    assert abs(t2["B"] + h * h * O.rhs_f(pr, 1, p2)) < 1e-14
    # the same on the lower face, through the -y neighbour
    p3 = np.array([0.125, -1.0 + h, 0.5])
    t3 = O.point_terms(pr, th, p3)
    q3 = p3 - np.array([0.0, h, 0.0])
    assert abs(t3["B"] + h * h * O.rhs_f(pr, 1, p3) + mu * (q3 @ q3)) < 1e-14


# -------------------------------------------------------- loss weights ----
def test_lambda_weights_the_jump_rows_linearly():
    """r_p^2 = (B/D)^2 + lambda J^2: the loss and its gradient are affine in
    lambda, and the jump rows contribute (cut cells are present)."""
    rng = np.random.default_rng(31)

    def prob(lam):
        return O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=2, width=8, h=2.0 / 16,
                              mu_minus=1.0, mu_plus=10.0, lambda_jump=lam)

    P = 2 * O.params_per_net(prob(1.0))
    th = rng.normal(size=P) * 0.5
    pts = O.sample_points(prob(1.0), 4, 1, 150, 100)
    (L0, g0), (L1, g1), (L25, g25) = (O.loss_grad(prob(lam), th, pts) for lam in (0.0, 1.0, 2.5))
    assert L1 - L0 > 1e-3 * L1
    assert abs((L25 - L0) - 2.5 * (L1 - L0)) <= 1e-12 * L25
    assert np.allclose(g25 - g0, 2.5 * (g1 - g0), rtol=0, atol=1e-12 * np.max(np.abs(g25)))
    assert np.max(np.abs(g1 - g0)) > 1e-3 * np.max(np.abs(g1))


# ------------------------------------------------------------ training ----
def test_training_step_t_samples_at_counter_t_and_uses_adam_step_t():
    """Step t = step0 + 1, step0 + 2, ... draws its points at Philox counter t,
    takes the loss gradient there and applies Adam with bias correction for t
    (the numbering stated for nbm_train_steps)."""
    pr = O.make_problem(geometry=O.GEOM_FLOWER, n_hidden=2, width=8, h=2.0 / 16)
    rng = np.random.default_rng(5)
    P = 2 * O.params_per_net(pr)
    th0 = rng.normal(size=P) * 0.3
    m0 = rng.normal(size=P) * 1e-3
    v0 = np.abs(rng.normal(size=P)) * 1e-5
    step0, n_steps, batch, band, seed = 4, 3, 40, 12, 11
    th, m, v = th0.copy(), m0.copy(), v0.copy()
    hist = O.train(pr, th, m, v, step0, n_steps, batch, band, lr=2e-3, seed=seed, n_threads=1)
    th2, m2, v2 = th0.copy(), m0.copy(), v0.copy()
    for j in range(n_steps):
        t = step0 + 1 + j
        pts = O.sample_points(pr, seed, t, batch, band)
        L, g = O.loss_grad(pr, th2, pts, n_threads=1)
        assert hist[j] == L
        O.adam_step(th2, m2, v2, g, t, lr=2e-3)
    assert np.array_equal(th, th2) and np.array_equal(m, m2) and np.array_equal(v, v2)


# ---------------------------------------------------- grid evaluation ----
@pytest.mark.parametrize("n", [4, 8])
def test_grid_evaluation_takes_the_network_of_the_node_phase(n):
    """With the minus network identically 0 and the plus network identically
    1, the evaluated grid is the indicator of |x| > 1/2.  Nodes on the sphere
    (exact in binary for these n) take the minus network."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, r0=0.5, n_hidden=2, width=4)
    Pn = O.params_per_net(pr)
    th = np.zeros(2 * Pn)
    th[2 * Pn - 1] = 1.0  # output bias of the plus network
    u = O.eval_grid(pr, th, n).reshape(n + 1, n + 1, n + 1)
    g = -1.0 + np.arange(n + 1) * (2.0 / n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    ref = (X * X + Y * Y + Z * Z > 0.25).astype(float)
    assert np.array_equal(u, ref)
    assert np.any(X * X + Y * Y + Z * Z == 0.25)


def test_grid_evaluation_orders_nodes_x_fastest():
    """Node (i, j, k) of the evaluated grid is at (-1 + i h, -1 + j h, -1 + k h)
    and sits at index i + (n+1)(j + (n+1) k).  Seen through a mesh level set
    that is linear in x, y and z with different slopes: its indicator is not
    symmetric under any swap of the axes.  phi is at least 1/40 away from 0 at
    every node."""
    m, n = 4, 8

    def lin(x, y, z):
        return x + 0.5 * y - 0.25 * z - 0.1

    gm = -1.0 + np.arange(m + 1) * (2.0 / m)
    Zm, Ym, Xm = np.meshgrid(gm, gm, gm, indexing="ij")
    pr = O.make_problem(geometry=O.GEOM_GRID, n_hidden=2, width=4, phi_grid=lin(Xm, Ym, Zm))
    Pn = O.params_per_net(pr)
    th = np.zeros(2 * Pn)
    th[2 * Pn - 1] = 1.0
    u = O.eval_grid(pr, th, n)
    g = -1.0 + np.arange(n + 1) * (2.0 / n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    ph = lin(X, Y, Z)
    assert np.min(np.abs(ph)) >= 0.025 - 1e-15
    assert np.array_equal(u, (ph > 0).astype(float).reshape(-1))


# ------------------------------------------------ point rows vs grid rows ----
def _interior_nodes(n):
    g = -1.0 + np.arange(1, n) * (2.0 / n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


@pytest.mark.parametrize("geom", [O.GEOM_ALL_MINUS, O.GEOM_ALL_PLUS])
def test_point_row_is_the_grid_row_for_any_node_values(geom):
    """Without an interface, the point residual of Sec. 3 at a node, with the
    network's values at the stencil points, is the grid row of that node
    applied to the network's node values: B_p = (A x - b)_p and D_p = A_pp.
    The grid matrix with face-centred mu is pinned symmetric, so this pins
    the point row's face coefficients too.  The Sec. 4.1 mu varies along x
    and y on the minus side and along z on the plus side."""
    n = 8
    pr = O.make_problem(geometry=geom, n_hidden=2, width=8, h=2.0 / n, k_minus=0.7,
                        k_plus=1.3, solution=O.SOL_SEC41)
    rng = np.random.default_rng(8)
    Pn = O.params_per_net(pr)
    th = rng.normal(size=2 * Pn) * 0.7
    s = 0 if geom == O.GEOM_ALL_MINUS else 1
    nodes = _interior_nodes(n)
    x = np.array([O.mlp_eval(pr, th[s * Pn:(s + 1) * Pn], q) for q in nodes])
    A, b = O.grid_assemble_dense(pr, n)
    R = A @ x - b
    sc = np.max(np.abs(b)) + np.max(np.abs(A @ x))
    for r, q in enumerate(nodes):
        t = O.point_terms(pr, th, q)
        assert abs(t["B"] - R[r]) <= 1e-14 * sc
        assert abs(t["D"] - A[r, r]) <= 1e-14 * A[r, r]


@pytest.mark.parametrize("geom,sol", [(O.GEOM_SPHERE, O.SOL_BENCH), (O.GEOM_FLOWER, O.SOL_SEC41)])
def test_point_row_is_the_grid_row_at_the_exact_solution(geom, sol):
    """With an interface: the grid row with the exact node jump, applied to
    the exact node values, is the point residual of the exact pair at that
    node (mode 1), cut rows included."""
    n = 16
    pr = O.make_problem(geometry=geom, h=2.0 / n, mu_minus=1.0, mu_plus=10.0, k_minus=0.3,
                        k_plus=0.6, solution=sol)
    nodes = _interior_nodes(n)
    x = np.array([O.exact_u(pr, O.phase(pr, q), q) for q in nodes])
    A, b = O.grid_assemble_dense(pr, n)
    R = A @ x - b
    sc = np.max(np.abs(b)) + np.max(np.abs(A @ x))
    n_cut = 0
    for r, q in enumerate(nodes):
        t = O.point_terms(pr, None, q, mode=1)
        assert abs(t["B"] - R[r]) <= 1e-13 * sc
        assert abs(t["D"] - A[r, r]) <= 1e-14 * A[r, r]
        n_cut += t["cut"]
    assert n_cut > 20


# ------------------------------------------------ grid CG and node jumps ----
@pytest.mark.parametrize("mu_plus", [10.0, 1000.0])
def test_grid_cg_is_jacobi_pcg(mu_plus):
    """The oracle's grid CG is Jacobi-preconditioned CG from x = 0 stopped at
    ||b - A x|| <= rtol ||b||.  scipy's cg with M = diag(A)^-1 takes the same
    number of iterations (to one, for rounding at the threshold) to the same
    solution."""
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    n = 12
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=mu_plus)
    A, b = O.grid_assemble_dense(pr, n)
    st, u, it, rr = O.grid_cg_solve(pr, n, rtol=1e-10, max_iter=5000)
    count = [0]

    def cb(_):
        count[0] += 1

    x, info = spla.cg(sp.csr_matrix(A), b, rtol=1e-10, M=sp.diags(1.0 / np.diag(A)),
                      callback=cb, maxiter=5000)
    assert st == 0 and info == 0
    assert abs(it - count[0]) <= 1
    ui = u.reshape(n + 1, n + 1, n + 1)[1:n, 1:n, 1:n].reshape(-1)
    assert np.max(np.abs(ui - x)) <= 1e-12 * np.max(np.abs(x))
    assert rr <= 1e-10 and abs(rr - np.linalg.norm(b - A @ ui) / np.linalg.norm(b)) <= 1e-13


def test_lagged_passes_restart_from_the_previous_solution():
    """Each later pass of the lagged jump re-solves from the previous pass's
    solution, so it takes well under the iterations of a solve from zero."""
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    n = 32
    it1 = O.grid_solve_jump(pr, n, O.JUMP_FIRST_ORDER, rtol=1e-12, max_iter=20000)[2]
    st, u, it, rr, passes, dj = O.grid_solve_jump(pr, n, O.JUMP_EXTRAP, rtol=1e-12,
                                                  max_iter=20000)
    assert st == 0 and passes >= 3
    assert it - it1 < 0.75 * (passes - 1) * it1


@pytest.mark.parametrize("geom,s", [(O.GEOM_ALL_MINUS, 0), (O.GEOM_ALL_PLUS, 1)])
def test_normal_derivative_fit_is_centred_one_spacing_into_its_side(geom, s):
    """The least-squares fit of the lagged jump uses the 3x3x3 block of nodes
    around the node nearest x_G - h n (minus side) or x_G + h n (plus side).
    For a quadratic u, the linear fit over a block symmetric about its centre c
    has slope grad u(c) exactly (the even quadratic part is orthogonal to the
    odd linear basis).  So the fitted d_n u is grad u(c) . n, and c is visible."""
    n = 16
    h = 2.0 / n
    pr = O.make_problem(geometry=geom)
    Hm = np.array([[2.0, 0.5, -0.3], [0.5, -1.0, 0.2], [-0.3, 0.2, 1.5]])
    bv = np.array([0.3, -0.7, 0.4])
    g = -1.0 + np.arange(n + 1) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    Q = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    u = 0.5 * np.einsum("pi,ij,pj->p", Q, Hm, Q) + Q @ bv
    rng = np.random.default_rng(12)
    for _ in range(20):
        xg = rng.uniform(-0.5, 0.5, size=3)
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        target = xg + (h if s == 1 else -h) * nrm
        c_idx = np.rint((target + 1.0) / h)
        if np.any(np.abs((target + 1.0) / h - c_idx) > 0.49):
            continue  # too close to a tie between two nodes
        c = -1.0 + c_idx * h
        dn = O.fit_dn(pr, n, u, s, xg, nrm)
        assert dn is not None
        assert abs(dn - (Hm @ c + bv) @ nrm) <= 1e-11


# -------------------------------------------------------- grid metrics ----
def test_grid_error_is_taken_over_the_interior_nodes():
    """L-inf and RMS of u minus the exact solution of each node's phase, over
    the (n-1)^3 interior nodes: a constant offset c on the interior gives
    L-inf = RMS = |c|; a single wrong node gives RMS = |e| / (n-1)^1.5; the
    boundary nodes do not count."""
    n = 8
    pr = O.make_problem(geometry=O.GEOM_SPHERE)
    g = -1.0 + np.arange(n + 1) * (2.0 / n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    ex = np.array([O.exact_u(pr, O.phase(pr, q), q) for q in pts])
    inner = ((np.abs(pts) < 1.0).all(1))
    u = ex + 0.125 * inner + 7.0 * ~inner
    linf, rms = O.grid_error(pr, n, u)
    assert abs(linf - 0.125) < 1e-14 and abs(rms - 0.125) < 1e-14
    u = ex.copy()
    u[np.flatnonzero(inner)[37]] += 0.5
    linf, rms = O.grid_error(pr, n, u)
    assert abs(linf - 0.5) < 1e-14 and abs(rms - 0.5 / (n - 1) ** 1.5) < 1e-15


@pytest.mark.parametrize("mode", [O.JUMP_EXACT, O.JUMP_EXTRAP, O.JUMP_FIRST_ORDER])
def test_grid_solution_carries_the_dirichlet_data_on_the_boundary(mode):
    """The solved node array holds g = u+ = |x|^2 (written out here) on every
    boundary node."""
    n = 12
    pr = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    st, u, *_ = O.grid_solve_jump(pr, n, mode, rtol=1e-10, max_iter=5000)
    assert st == 0
    g = -1.0 + np.arange(n + 1) * (2.0 / n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    bnd = (np.abs(X) == 1.0) | (np.abs(Y) == 1.0) | (np.abs(Z) == 1.0)
    ref = (X * X + Y * Y + Z * Z)[bnd]
    assert np.max(np.abs(u.reshape(n + 1, n + 1, n + 1)[bnd] - ref)) <= 1e-15


# ------------------------------------------------------ degenerate cases ----
def test_flower_gradient_on_the_polar_axis_is_radial():
    """On the z axis the flower's angular term has no derivative (a conical
    point: sin(5 theta) cos(3 psi) behaves like rho cos(3 psi) / z there).
    The reading takes the radial gradient x / |x|, the average of the
    directional derivatives around the axis."""
    pr = O.make_problem(geometry=O.GEOM_FLOWER)
    for z in (0.5, -0.25, 0.625):
        g = O.grad_phi(pr, np.array([0.0, 0.0, z]))
        assert np.array_equal(g, np.array([0.0, 0.0, math.copysign(1.0, z)]))


def test_empty_batch_has_zero_loss_and_gradient():
    pr = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=2, width=4, h=2.0 / 16)
    th = np.random.default_rng(2).normal(size=2 * O.params_per_net(pr))
    pts = np.zeros((0, 3))
    assert O.loss(pr, th, pts) == 0.0
    L, g = O.loss_grad(pr, th, pts)
    assert L == 0.0 and np.all(g == 0.0) and len(g) == len(th)
    assert O.sample_points(pr, 1, 1, 0, 0).shape == (0, 3)


def test_normal_derivative_fit_refuses_degenerate_node_sets():
    """The fit needs four side-s nodes that span an affine basis.  Coplanar
    side-s nodes in the block, or fewer than four of them, give no value, and
    the node keeps its first-order jump."""
    m, n = 8, 16
    h = 2.0 / n
    gm = -1.0 + np.arange(m + 1) * (2.0 / m)
    Zm, Ym, Xm = np.meshgrid(gm, gm, gm, indexing="ij")
    u = np.zeros((n + 1) ** 3)
    node = -1.0 + 9 * h
    # phi = x - c with c a quarter spacing above the node plane x = node - h.
    # The block centred at (node, -h, 0) (normal along y) spans the planes
    # node - h, node, node + h, and only the first is on the minus side.
    c = node - 0.75 * h
    pr = O.make_problem(geometry=O.GEOM_GRID, phi_grid=Xm - c)
    xg = np.array([node, 0.0, 0.0])
    assert O.fit_dn(pr, n, u, 0, xg, np.array([0.0, 1.0, 0.0])) is None
    # off the node, rounding leaves the degenerate pivot at about +2e-15
    # instead of 0: the relative guard still refuses the set
    xg_off = np.array([0.12632993277877888, 0.0, 0.0])
    assert O.fit_dn(pr, n, u, 0, xg_off, np.array([0.0, 1.0, 0.0])) is None
    # the plus side of the same block holds two planes: a valid fit (u = 0)
    assert O.fit_dn(pr, n, u, 1, xg, np.array([0.0, -1.0, 0.0])) == 0.0
    # a corner: x + y + z <= c3 keeps only the block's corner node
    c3 = 3.0 * node - 2.5 * h
    pr3 = O.make_problem(geometry=O.GEOM_GRID, phi_grid=Xm + Ym + Zm - c3)
    d = np.full(3, 1.0 / math.sqrt(3.0))
    assert O.fit_dn(pr3, n, u, 0, np.full(3, node) + h * d, d) is None
    # a quarter spacing further out it keeps four nodes, a tetrahedron: a fit
    pr4 = O.make_problem(geometry=O.GEOM_GRID, phi_grid=Xm + Ym + Zm - (c3 + 1.25 * h))
    assert O.fit_dn(pr4, n, u, 0, np.full(3, node) + h * d, d) == 0.0
