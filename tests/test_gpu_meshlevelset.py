"""Level set stored on a coarse mesh (Sec. 3: the level set lives on a
separate coarse mesh), trilinearly interpolated, on the GPU
against the FP64 oracle: residual rows, gradients, grid evaluation and the
grid CG solve of problems whose interface is given only by mesh values.
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _nodes(n):
    g = -1.0 + np.arange(n + 1) * 2.0 / n
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


def _flower_phi(x):
    """The flower level set of the benchmark, sampled at mesh nodes (polar angle
    from +z, azimuth in the xy plane)."""
    r = np.sqrt((x ** 2).sum(1))
    th = np.arctan2(np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2), x[:, 2])
    ps = np.arctan2(x[:, 1], x[:, 0])
    return r - 0.5 - 0.1 * np.sin(5 * th) * np.cos(3 * ps)


def _pair(prec, H, L, h, phi, n_phi, **kw):
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=nbm.GEOM_GRID, n_hidden=L, width=H, precision=prec, h=h,
                        mu_minus=1.0, mu_plus=10.0, **kw)
    prob = nbm.Problem(d)
    prob.set_level_set(torch.from_numpy(phi).cuda(), n_phi)
    o = O.make_problem(geometry=O.GEOM_GRID, n_hidden=L, width=H, h=h, mu_minus=1.0,
                       mu_plus=10.0, phi_grid=phi, **kw)
    return prob, o


def _shell_points(phi_fn, n, seed):
    """uniform points plus points near the interface of the mesh level set"""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    s = d * rng.uniform(0.35, 0.65, size=n)[:, None]
    return np.concatenate([u, s]).astype(np.float32)


@pytest.mark.parametrize("prec,H,L,h,shape,n_phi,res_tol,grad_tol", [
    (0, 64, 2, 2 / 32, "sphere", 20, 1e-5, 1e-4),
    (0, 128, 3, 2 / 64, "flower", 24, 1e-5, 1e-4),
    (1, 128, 3, 2 / 128, "flower", 32, 2e-3, 5e-3),
], ids=["fp32-sphere20", "fp32-flower24", "bf16-flower32"])
def test_mesh_level_set_rows_and_gradient_match_oracle(prec, H, L, h, shape, n_phi, res_tol,
                                                       grad_tol):
    x = _nodes(n_phi)
    phi = np.sqrt((x ** 2).sum(1)) - 0.5 if shape == "sphere" else _flower_phi(x)
    prob, o = _pair(prec, H, L, h, phi, n_phi)
    pts = _shell_points(None, 600, seed=n_phi)
    th = inputs.glorot_params(H, L, seed=37, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    n_cut = sum(O.point_terms(o, th.astype(np.float64), p)["cut"] for p in pts[600:])
    assert n_cut > 20
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    er = _rel(np.sqrt(r2.cpu().numpy()), np.sqrt(r2_ref))
    eg = _rel(g.cpu().numpy(), g_ref)
    print(f"mesh level set {shape} {n_phi}^3 prec {prec}: residual {er:.2e} "
          f"loss {abs(loss - L_ref) / L_ref:.2e} grad {eg:.2e} ({n_cut} cut)")
    assert er <= res_tol
    assert abs(loss - L_ref) <= res_tol * L_ref and abs(loss2 - L_ref) <= res_tol * L_ref
    assert eg <= grad_tol


def test_mesh_level_set_grid_evaluation_and_cg_match_oracle():
    """The level-set mesh (13^3) shares no interior plane with the CG grid (14^3):
    the interpolant's gradient jumps across mesh faces, and an interface point on
    such a face would take its normal from whichever side rounding picks."""
    import paper_2210_14907_gb300 as nbm
    n_phi = 13
    x = _nodes(n_phi)
    phi = _flower_phi(x) + 0.013  # keep the nodes of the test grids off the interface
    prob, o = _pair(0, 64, 2, 2 / 32, phi, n_phi)
    th = inputs.glorot_params(64, 2, seed=41, bias_scale=0.2)
    n = 18
    xs = _nodes(n)
    assert min(abs(O.phi(o, p)) for p in xs) > 1e-9
    ref = O.eval_grid(o, th.astype(np.float64), n)
    got = prob.eval_grid(torch.from_numpy(th).cuda(), n, precision=nbm.PREC_FP32).cpu().numpy()
    assert _rel(got, ref) <= 1e-5
    st, uref, it_ref, rr_ref = O.grid_cg_solve(o, 14, rtol=1e-12, max_iter=20000)
    assert st == 0
    u, it, rr, ok = prob.grid_cg_solve(14, rtol=1e-12, max_iter=20000)
    assert ok and np.max(np.abs(u.cpu().numpy() - uref)) <= 1e-8 * np.max(np.abs(uref))


def test_mesh_level_set_errors():
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=nbm.GEOM_GRID, n_hidden=2, width=64)
    prob = nbm.Problem(d)
    params = nbm.xavier_init(d, seed=0, device="cuda")
    with pytest.raises(nbm.NBMError) as e:  # no level set yet
        prob.residual(params, n=1024)
    assert e.value.code == 1
    with pytest.raises(nbm.NBMError) as e:
        nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_GRID, band_fraction=0.2))
    assert e.value.code == 1
    other = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE))
    with pytest.raises(nbm.NBMError) as e:
        other.set_level_set(torch.zeros(27, dtype=torch.float64, device="cuda"), 2)
    assert e.value.code == 1
    # a level set that is negative everywhere: every point in Omega-, as for ALL_MINUS
    prob.set_level_set(-torch.ones(9 ** 3, dtype=torch.float64, device="cuda"), 8)
    ref = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_ALL_MINUS, n_hidden=2, width=64))
    pts = torch.rand(2048, 3, device="cuda") * 1.8 - 0.9
    a, _ = prob.residual(params, pts)
    b, _ = ref.residual(params, pts)
    assert a == b


def test_mesh_level_set_lagged_jump_cg_matches_oracle():
    """The extrapolated node jump on a mesh level set (projection, normal and
    fit all through the trilinear interpolant)."""
    import paper_2210_14907_gb300 as nbm
    n_phi = 13
    x = _nodes(n_phi)
    phi = _flower_phi(x) + 0.013
    _, o = _pair(0, 64, 2, 2 / 32, phi, n_phi)
    prob = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_GRID, mu_minus=1.0, mu_plus=10.0,
                                       grid_jump=nbm.JUMP_EXTRAP))
    prob.set_level_set(torch.from_numpy(phi).cuda(), n_phi)
    st, uref, it_ref, rr_ref, passes_ref, _ = O.grid_solve_jump(o, 14, O.JUMP_EXTRAP, rtol=1e-12,
                                                                max_iter=20000)
    assert st == 0
    u, it, rr, ok = prob.grid_cg_solve(14, rtol=1e-12, max_iter=20000)
    passes, dj, fell_back = prob.grid_jump_info()
    assert ok and passes == passes_ref and not fell_back
    assert np.max(np.abs(u.cpu().numpy() - uref)) <= 1e-8 * np.max(np.abs(uref))
