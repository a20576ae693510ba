"""Grid evaluation of the surrogate and the grid CG solve, against the FP64 oracle.

Evaluation tolerances (norm-wise relative over the nodes): FP32 1e-5; FP16
hidden GEMMs 2e-3 (11-bit operands and SFU tanh, the mixed-path residual
bar); BF16 1e-2 (8-bit operands).  CG: both sides solve to a relative residual
of 1e-12, the solutions agree to 1e-8 of max|u|.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


def _nbm():
    import paper_2210_14907_gb300 as nbm
    return nbm


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _clear_of_interface(o, n):
    """Grids with a node on phi = 0 leave the side of that node to the last ulp of
    the platform's FP64 cos/atan2 (the oracle's and CUDA's differ there); the
    parity grids below keep every node at least 1e-9 away from the interface."""
    x = -1.0 + np.arange(n + 1) * 2.0 / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ph = [abs(O.phi(o, p)) for p in np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)]
    return min(ph) > 1e-9


@pytest.mark.parametrize("geom,H,L,n", [(O.GEOM_SPHERE, 64, 2, 16), (O.GEOM_FLOWER, 128, 4, 18),
                                        (O.GEOM_SPHERE, 128, 3, 1), (O.GEOM_FLOWER, 128, 3, 5)])
def test_eval_grid_fp32_matches_oracle(geom, H, L, n):
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=H)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, n_hidden=L, width=H)
    if geom == O.GEOM_FLOWER:
        assert _clear_of_interface(o, n)
    th = inputs.glorot_params(H, L, seed=21, bias_scale=0.2)
    ref = O.eval_grid(o, th.astype(np.float64), n)
    got = prob.eval_grid(torch.from_numpy(th).cuda(), n, precision=nbm.PREC_FP32).cpu().numpy()
    assert got.shape == ref.shape
    assert _rel(got, ref) <= 1e-5


@pytest.mark.parametrize("prec,tol", [(2, 2e-3), (1, 1e-2)], ids=["fp16", "bf16"])
@pytest.mark.parametrize("L,n", [(3, 22), (4, 17), (4, 1)])
def test_eval_grid_tensor_cores_match_oracle(prec, tol, L, n):
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, n_hidden=L, width=128, precision=nbm.PREC_BF16)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_FLOWER, n_hidden=L, width=128)
    assert _clear_of_interface(o, n)
    th = inputs.glorot_params(128, L, seed=22, bias_scale=0.2)
    ref = O.eval_grid(o, th.astype(np.float64), n)
    got = prob.eval_grid(torch.from_numpy(th).cuda(), n, precision=prec).cpu().numpy()
    err = _rel(got, ref)
    print(f"eval prec {prec} L {L} n {n}: rel {err:.2e}")
    assert err <= tol


@pytest.mark.parametrize("prec,tol", [(2, 2e-3), (1, 1e-2)], ids=["fp16", "bf16"])
@pytest.mark.parametrize("L", [3, 4])
def test_eval_grid_tensor_cores_at_size(prec, tol, L):
    """Grids of many tiles per CTA (161^3 nodes, about 27 tile pairs per SM), so
    both tiles of a pair are in flight, across mixed flower tiles: the 16-bit
    tensor-core evaluation against the FP32 path (itself equal to the oracle)."""
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, n_hidden=L, width=128)
    prob = nbm.Problem(d)
    th = torch.from_numpy(inputs.glorot_params(128, L, seed=23, bias_scale=0.2)).cuda()
    n = 160
    ref = prob.eval_grid(th, n, precision=nbm.PREC_FP32).double()
    got = prob.eval_grid(th, n, precision=prec).double()
    err = (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item()
    mx = (torch.max(torch.abs(got - ref)) / torch.max(torch.abs(ref))).item()
    print(f"eval at size prec {prec} L {L}: rel {err:.2e}, max {mx:.2e}")
    assert err <= tol and mx <= 4 * tol
    gen = torch.Generator(device="cuda").manual_seed(29)
    pts = (torch.rand(100_003, 3, device="cuda", generator=gen) * 1.9 - 0.95).contiguous()
    a = prob.eval_points(th, pts, precision=nbm.PREC_FP32).double()
    b = prob.eval_points(th, pts, precision=prec).double()
    assert (torch.linalg.norm(b - a) / torch.linalg.norm(a)).item() <= tol


@pytest.mark.parametrize("geom,mu_p,n", [(O.GEOM_SPHERE, 10.0, 16), (O.GEOM_FLOWER, 100.0, 14),
                                         (O.GEOM_ALL_MINUS, 10.0, 9)])
def test_grid_cg_matches_oracle(geom, mu_p, n):
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=geom, mu_minus=1.0, mu_plus=mu_p, k_minus=0.5)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, mu_minus=1.0, mu_plus=mu_p, k_minus=0.5)
    if geom == O.GEOM_FLOWER:
        assert _clear_of_interface(o, n)
    st, ref, it_ref, rr_ref = O.grid_cg_solve(o, n, rtol=1e-12, max_iter=20000)
    assert st == 0
    u, it, rr, ok = prob.grid_cg_solve(n, rtol=1e-12, max_iter=20000)
    assert ok and rr <= 1e-12
    u = u.cpu().numpy()
    assert np.max(np.abs(u - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert abs(it - it_ref) <= 12  # the device checks convergence every 10 iterations


def test_grid_cg_second_order_without_interface():
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=nbm.GEOM_ALL_MINUS, mu_minus=2.0, k_minus=1.0)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_ALL_MINUS, mu_minus=2.0, k_minus=1.0)
    errs = []
    for n in (16, 32, 64):
        u, it, rr, ok = prob.grid_cg_solve(n, rtol=1e-12, max_iter=50000)
        assert ok
        errs.append(O.grid_error(o, n, u.cpu().numpy())[0])
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_grid_cg_reports_non_convergence():
    nbm = _nbm()
    prob = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE))
    u, it, rr, ok = prob.grid_cg_solve(32, rtol=1e-12, max_iter=3)
    assert not ok and it == 3 and rr > 1e-12
    assert torch.isfinite(u).all()
    with pytest.raises(nbm.NBMError) as e:
        prob.grid_cg_solve(1, rtol=1e-10)
    assert e.value.code == 1


@pytest.mark.parametrize("geom,mu_p,n", [(O.GEOM_SPHERE, 10.0, 16), (O.GEOM_FLOWER, 100.0, 14),
                                         (O.GEOM_FLOWER, 1000.0, 22), (O.GEOM_ALL_MINUS, 10.0, 9)])
def test_refined_solve_matches_oracle(geom, mu_p, n):
    """FP32 inner corrections of FP64 residuals reach the oracle's FP64 CG
    solution of the same rows (the stopping test is the true FP64 residual)."""
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=geom, mu_minus=1.0, mu_plus=mu_p, k_minus=0.5)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, mu_minus=1.0, mu_plus=mu_p, k_minus=0.5)
    if geom == O.GEOM_FLOWER:
        assert _clear_of_interface(o, n)
    st, ref, it_ref, rr_ref = O.grid_cg_solve(o, n, rtol=1e-13, max_iter=50000)
    assert st == 0
    u, it, rr, ok = prob.grid_solve_refined(n, rtol=1e-12, max_iter=50000)
    assert ok and rr <= 1e-12
    u = u.cpu().numpy()
    err = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    print(f"refined geom {geom} mu+ {mu_p} n {n}: {it} inner iterations (FP64 CG {it_ref}), "
          f"max err {err:.2e}")
    assert err <= 1e-8


@pytest.mark.parametrize("n", [42, 97])
def test_refined_solve_agrees_with_fp64_cg(n):
    """Beyond the oracle's sizes: the refined and the FP64 CG solutions of the
    same system agree to the accuracy their residual tests allow, and the
    refined solve needs at most twice the FP64 iterations."""
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, mu_minus=1.0, mu_plus=10.0)
    prob = nbm.Problem(d)
    a, it_a, rr_a, ok_a = prob.grid_cg_solve(n, rtol=1e-12, max_iter=100000)
    b, it_b, rr_b, ok_b = prob.grid_solve_refined(n, rtol=1e-12, max_iter=100000)
    assert ok_a and ok_b and rr_b <= 1e-12
    err = (torch.max(torch.abs(a - b)) / torch.max(torch.abs(a))).item()
    print(f"n {n}: FP64 CG {it_a} it, refined {it_b} inner it, max diff {err:.2e}")
    assert err <= 1e-9
    assert it_b <= 2 * it_a
    if n == 42:  # small enough for the oracle's CG
        o = O.make_problem(geometry=O.GEOM_FLOWER, mu_minus=1.0, mu_plus=10.0)
        st, ref, _, _ = O.grid_cg_solve(o, n, rtol=1e-13, max_iter=50000)
        assert st == 0
        assert np.max(np.abs(b.cpu().numpy() - ref)) <= 1e-8 * np.max(np.abs(ref))


def test_refined_solve_reports_non_convergence_and_bad_arguments():
    nbm = _nbm()
    prob = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE))
    u, it, rr, ok = prob.grid_solve_refined(32, rtol=1e-12, max_iter=3)
    assert not ok and it == 3 and 0 < rr < 1.0
    assert torch.isfinite(u).all()
    with pytest.raises(nbm.NBMError) as e:
        prob.grid_solve_refined(1, rtol=1e-10)
    assert e.value.code == 1
    with pytest.raises(nbm.NBMError) as e:
        prob.grid_solve_refined(8, rtol=0.0)
    assert e.value.code == 1


@pytest.mark.parametrize("geom,mu_p,n", [(O.GEOM_SPHERE, 10.0, 16), (O.GEOM_FLOWER, 100.0, 14),
                                         (O.GEOM_SPHERE, 1000.0, 22)])
@pytest.mark.parametrize("mode", [1, 2], ids=["extrap", "first_order"])
@pytest.mark.parametrize("solver", ["cg", "refined"])
def test_grid_jump_modes_match_oracle(geom, mu_p, n, mode, solver):
    """Extrapolated node jump (lagged small-mu derivative, or first order): the
    GPU solve equals the oracle's, pass for pass."""
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=geom, mu_minus=1.0, mu_plus=mu_p, grid_jump=mode)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, mu_minus=1.0, mu_plus=mu_p)
    if geom == O.GEOM_FLOWER:
        assert _clear_of_interface(o, n)
    st, ref, it_ref, rr_ref, passes_ref, dj_ref = O.grid_solve_jump(o, n, mode, rtol=1e-12,
                                                                    max_iter=50000)
    assert st == 0
    f = prob.grid_cg_solve if solver == "cg" else prob.grid_solve_refined
    u, it, rr, ok = f(n, rtol=1e-12, max_iter=50000)
    passes, dj, fell_back = prob.grid_jump_info()
    assert ok and rr <= 1e-12 and not fell_back
    assert passes == passes_ref
    err = np.max(np.abs(u.cpu().numpy() - ref)) / np.max(np.abs(ref))
    print(f"jump mode {mode} {solver} geom {geom} mu+ {mu_p} n {n}: {passes} passes, "
          f"max err {err:.2e}")
    assert err <= 1e-8


@pytest.mark.parametrize("solver", ["cg", "refined"])
def test_grid_lagged_jump_second_order(solver):
    """At GPU sizes the lagged jump keeps the grid scheme second order (RMS and
    L-inf, n = 32, 64, 128); the first-order jump is first order."""
    nbm = _nbm()
    o = O.make_problem(geometry=O.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0)
    errs = {1: [], 2: []}
    for mode in (1, 2):
        prob = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0,
                                           grid_jump=mode))
        f = prob.grid_cg_solve if solver == "cg" else prob.grid_solve_refined
        for n in (32, 64, 128):
            u, it, rr, ok = f(n, rtol=1e-11, max_iter=100000)
            passes, dj, fell_back = prob.grid_jump_info()
            assert ok and not fell_back and (passes == 1) == (mode == 2)
            errs[mode].append(O.grid_error(o, n, u.cpu().numpy()))
    print(solver, errs)
    for i in range(2):
        assert errs[1][i][0] / errs[1][i + 1][0] > 3.0 and errs[1][i][1] / errs[1][i + 1][1] > 3.5
        assert 1.5 < errs[2][i][0] / errs[2][i + 1][0] < 3.0


def test_large_grid_solves_with_separate_reductions():
    """n = 202 (8.1 M unknowns): past the size where the reductions are folded
    into the producing kernels, so every sum goes through the separate
    reduction launch.  Both solvers reach the same solution, second-order
    close to the exact one (2.2e-5 at n = 256, so about 3.6e-5 here)."""
    nbm = _nbm()
    prob = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0))
    n = 202
    assert (n - 1) ** 3 > 8_000_000
    a, it_a, rr_a, ok_a = prob.grid_cg_solve(n, rtol=1e-10, max_iter=100000)
    b, it_b, rr_b, ok_b = prob.grid_solve_refined(n, rtol=1e-10, max_iter=100000)
    assert ok_a and ok_b and rr_a <= 1e-10 and rr_b <= 1e-10
    diff = (torch.max(torch.abs(a - b)) / torch.max(torch.abs(a))).item()
    g = -1.0 + torch.arange(n + 1, device="cuda", dtype=torch.float64) * (2.0 / n)
    Z, Y, X = torch.meshgrid(g, g, g, indexing="ij")
    r = torch.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    exact = torch.where(r <= 0.5, torch.exp(X) * torch.cos(Y) * torch.sin(Z), r ** 2).reshape(-1)
    interior = torch.zeros((n + 1,) * 3, dtype=torch.bool, device="cuda")
    interior[1:-1, 1:-1, 1:-1] = True
    linf = torch.max(torch.abs(a - exact)[interior.reshape(-1)]).item()
    print(f"n {n}: FP64 CG {it_a} it, refined {it_b} inner it, diff {diff:.2e}, L-inf {linf:.2e}")
    assert diff <= 1e-8 and linf <= 5e-5


@pytest.mark.parametrize("geom, mu_p", [(O.GEOM_SPHERE, 10.0), (O.GEOM_FLOWER, 100.0)],
                         ids=["sphere", "flower"])
def test_grid_node_jump_matches_oracle_in_every_mode(geom, mu_p):
    """nbm_grid_node_jump on all (n+1)^3 nodes against the oracle: the exact jump
    u+ - u- of the manufactured pair, the first-order jump alpha + d beta/mu_big
    within 3h of Gamma, and the lagged jump with the small side's d_n u fitted
    from given node values (here the grid solution)."""
    import paper_2210_14907_gb300 as nbm
    n = 22
    prob = nbm.Problem(nbm.ProblemDesc(geometry=geom, mu_minus=1.0, mu_plus=mu_p,
                                       grid_jump=nbm.JUMP_EXTRAP))
    u, _, _, ok = prob.grid_cg_solve(n, rtol=1e-10)
    assert ok
    uh = u.cpu().numpy()
    o = O.make_problem(geometry=geom, mu_minus=1.0, mu_plus=mu_p)
    h = 2.0 / n
    g = -1.0 + np.arange(n + 1) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    assert min(abs(O.phi(o, x)) for x in nodes) > 1e-9  # no node decided by rounding
    J = prob.grid_node_jump(n, nbm.JUMP_EXACT).cpu().numpy()
    ref = np.array([O.exact_u(o, 1, x) - O.exact_u(o, 0, x) for x in nodes])
    assert np.max(np.abs(J - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())
    J1 = prob.grid_node_jump(n, nbm.JUMP_FIRST_ORDER).cpu().numpy()
    Jl = prob.grid_node_jump(n, nbm.JUMP_EXTRAP, u).cpu().numpy()
    r1 = np.zeros(len(nodes))
    rl = np.zeros(len(nodes))
    band = 0
    for e, x in enumerate(nodes):
        inb, j1, xg, nrm, ss = O.jump_extrap(o, x, h)
        if not inb:
            continue
        band += 1
        r1[e] = j1
        dn = O.fit_dn(o, n, uh, ss, xg, nrm)
        rl[e] = O.jump_extrap(o, x, h, dn)[1] if dn is not None else j1
    assert band > 100
    assert np.max(np.abs(J1 - r1)) <= 1e-10
    assert np.max(np.abs(Jl - rl)) <= 1e-10
    assert np.max(np.abs(Jl - J1)) > 1e-6  # the lag term is there
    with pytest.raises(nbm.NBMError):
        prob.grid_node_jump(n, nbm.JUMP_EXTRAP)  # the lagged mode needs node values
