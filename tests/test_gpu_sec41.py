"""The convergence study of Sec. 4.1 on the GPU: the manufactured pair with
variable diffusion coefficients (mu at the face centres of the implicit cell)
on every path, against the FP64 oracle.

Tolerances are those of each path (FP32: residual 1e-5, gradient 1e-4; mixed:
2e-3, 5e-3; grid CG: 1e-8 of max|u|).
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec,geom,H,L,h,fp64,res_tol,grad_tol", [
    (0, O.GEOM_SPHERE, 64, 2, 2 / 32, -1, 1e-5, 1e-4),
    (0, O.GEOM_FLOWER, 128, 3, 2 / 64, -1, 1e-5, 1e-4),
    (1, O.GEOM_SPHERE, 128, 3, 2 / 128, -1, 2e-3, 5e-3),
    (1, O.GEOM_SPHERE, 128, 4, 2 / 512, 1, 2e-3, 5e-3),   # FP64 rows
], ids=["fp32-sphere", "fp32-flower", "bf16", "bf16-fp64rows"])
def test_variable_mu_loss_residual_gradient_match_oracle(prec, geom, H, L, h, fp64, res_tol,
                                                         grad_tol):
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=H, precision=prec, h=h,
                        k_minus=0.3, k_plus=0.7, solution=nbm.SOL_SEC41, fp64_stencil=fp64)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, n_hidden=L, width=H, h=h, k_minus=0.3, k_plus=0.7,
                       solution=O.SOL_SEC41)
    pts = inputs.mixed_points(700, 300, seed=L + 60)
    th = inputs.glorot_params(H, L, seed=17, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    er = _rel(np.sqrt(r2.cpu().numpy()), np.sqrt(r2_ref))
    eg = _rel(g.cpu().numpy(), g_ref)
    print(f"Sec. 4.1 prec {prec} H {H} L {L} h {h}: residual {er:.2e} "
          f"loss {abs(loss - L_ref) / L_ref:.2e} grad {eg:.2e}")
    assert er <= res_tol
    assert abs(loss - L_ref) <= res_tol * L_ref and abs(loss2 - L_ref) <= res_tol * L_ref
    assert eg <= grad_tol


@pytest.mark.parametrize("geom,n", [(O.GEOM_SPHERE, 16), (O.GEOM_ALL_PLUS, 12)])
def test_variable_mu_grid_cg_matches_oracle(geom, n):
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=geom, solution=nbm.SOL_SEC41, k_minus=0.5)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, solution=O.SOL_SEC41, k_minus=0.5)
    st, ref, it_ref, rr_ref = O.grid_cg_solve(o, n, rtol=1e-12, max_iter=20000)
    assert st == 0
    u, it, rr, ok = prob.grid_cg_solve(n, rtol=1e-12, max_iter=20000)
    assert ok and rr <= 1e-12
    assert np.max(np.abs(u.cpu().numpy() - ref)) <= 1e-8 * np.max(np.abs(ref))


def test_variable_mu_training_decreases_the_loss():
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE, n_hidden=3, width=128,
                        precision=nbm.PREC_BF16, h=2 / 64, solution=nbm.SOL_SEC41)
    prob = nbm.Problem(d)
    params = nbm.xavier_init(d, seed=5, device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    hist = torch.zeros(200, device="cuda")
    prob.train_steps(params, m, v, 0, 200, 32768, lr=1e-3, seed=3, loss_hist=hist)
    h = hist.cpu().numpy()
    assert np.all(np.isfinite(h)) and h[-20:].mean() < 0.2 * h[:5].mean()


@pytest.mark.parametrize("sol,act,H,L,h,geom", [
    (1, 1, 10, 5, 2 / 32, O.GEOM_SPHERE),   # the paper's 5 x 10 sine pair (982 parameters)
    (1, 1, 10, 5, 2 / 128, O.GEOM_SPHERE),
    (0, 0, 16, 3, 2 / 64, O.GEOM_FLOWER),   # narrow tanh networks
    (1, 1, 32, 2, 2 / 16, O.GEOM_SPHERE),
], ids=["sin10x5-h32", "sin10x5-h128", "tanh16x3", "sin32x2"])
def test_narrow_networks_match_oracle(sol, act, H, L, h, geom):
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=H, precision=nbm.PREC_FP32, h=h,
                        solution=sol, activation=act)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, n_hidden=L, width=H, h=h, solution=sol, activation=act)
    if H == 10 and L == 5:
        assert nbm.param_count(d) == 982
    pts = inputs.mixed_points(600, 400, seed=H + L)
    th = inputs.glorot_params(H, L, seed=29, bias_scale=0.2)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    er = _rel(np.sqrt(r2.cpu().numpy()), np.sqrt(r2_ref))
    eg = _rel(g.cpu().numpy(), g_ref)
    print(f"narrow H {H} L {L} act {act} h {h}: residual {er:.2e} "
          f"loss {abs(loss - L_ref) / L_ref:.2e} grad {eg:.2e}")
    assert er <= 1e-5 and abs(loss - L_ref) <= 1e-5 * L_ref and abs(loss2 - L_ref) <= 1e-5 * L_ref
    assert eg <= 1e-4
    n = 14
    ref = O.eval_grid(o, th.astype(np.float64), n)
    got = prob.eval_grid(tp, n, precision=nbm.PREC_FP32).cpu().numpy()
    assert _rel(got, ref) <= 1e-5


def test_sec41_sine_pair_trains_and_is_deterministic():
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE, n_hidden=5, width=10, precision=nbm.PREC_FP32,
                        h=2 / 32, solution=nbm.SOL_SEC41, activation=nbm.ACT_SIN)
    prob = nbm.Problem(d)
    runs = []
    for _ in range(2):
        params = nbm.xavier_init(d, seed=1, device="cuda")
        m = torch.zeros_like(params)
        v = torch.zeros_like(params)
        hist = torch.zeros(300, device="cuda")
        prob.train_steps(params, m, v, 0, 300, 4096, lr=3e-3, seed=2, loss_hist=hist)
        runs.append((params.clone(), hist.cpu().numpy()))
    assert torch.equal(runs[0][0], runs[1][0])
    h = runs[0][1]
    assert np.all(np.isfinite(h)) and h[-20:].mean() < 0.1 * h[:5].mean()


def test_narrow_and_sine_limits():
    import paper_2210_14907_gb300 as nbm
    bad = [dict(width=10, n_hidden=5, precision=nbm.PREC_BF16),
           dict(width=64, n_hidden=5),
           dict(width=128, n_hidden=3, activation=nbm.ACT_SIN),
           dict(width=10, n_hidden=6),
           dict(solution=2), dict(activation=2)]
    for kw in bad:
        with pytest.raises(nbm.NBMError) as e:
            nbm.Problem(nbm.ProblemDesc(**kw))
        assert e.value.code == 1, kw
