"""Implicit refinement (Sec. 3, Fig. 2; Sec. 4.2): the rows of the cells of
spacing h, h/2, ..., h/2^levels around the same points, stacked into r_p.

The device runs one sample/classify/cut-row/fused pass per level and sums the
levels' losses, per-point residuals and gradients before one Adam update; the
oracle sums its single-level functions over the same spacings.  Tolerances are
those of the path (FP32: residual 1e-5, gradient 1e-4; mixed: 2e-3, 5e-3).
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec,geom,H,L,h,levels,res_tol,grad_tol", [
    (0, O.GEOM_FLOWER, 64, 2, 2 / 32, 2, 1e-5, 1e-4),      # FP32 path: 2/32, 2/64, 2/128
    (1, O.GEOM_SPHERE, 128, 3, 2 / 64, 3, 2e-3, 5e-3),     # BF16: 2/64 .. 2/512 (FP64 rows last)
], ids=["fp32", "bf16"])
def test_refined_loss_residual_gradient_match_oracle(prec, geom, H, L, h, levels, res_tol,
                                                     grad_tol):
    import paper_2210_14907_gb300 as nbm
    d = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=H, precision=prec, mu_minus=1.0,
                        mu_plus=10.0, h=h, refine_levels=levels)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=geom, n_hidden=L, width=H, mu_minus=1.0, mu_plus=10.0, h=h)
    pts = inputs.mixed_points(700, 300, seed=41)
    th = inputs.glorot_params(H, L, seed=13, bias_scale=0.1)
    L_ref, r2_ref = O.loss_levels(o, levels, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad_levels(o, levels, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    er = _rel(np.sqrt(r2.cpu().numpy()), np.sqrt(r2_ref))
    eg = _rel(g.cpu().numpy(), g_ref)
    print(f"levels {levels} prec {prec}: residual {er:.2e} loss {abs(loss - L_ref) / L_ref:.2e} "
          f"grad {eg:.2e}")
    assert er <= res_tol
    assert abs(loss - L_ref) <= res_tol * L_ref and abs(loss2 - L_ref) <= res_tol * L_ref
    assert eg <= grad_tol
    # one level is the single-resolution problem
    d1 = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=H, precision=prec, mu_minus=1.0,
                         mu_plus=10.0, h=h, refine_levels=0)
    l0, _ = nbm.Problem(d1).residual(tp, tx)
    assert abs(l0 - O.loss(o, th.astype(np.float64), pts)) <= res_tol * l0
    assert loss > l0


def test_refined_training_is_deterministic_and_its_first_loss_matches():
    import paper_2210_14907_gb300 as nbm
    d = nbm.config("C2")
    d.h = 2 / 64
    d.refine_levels = 3
    d.band_fraction = 0.25
    prob = nbm.Problem(d)
    n = 16384
    runs = []
    for _ in range(2):
        params = nbm.xavier_init(d, seed=2, device="cuda")
        m = torch.zeros_like(params)
        v = torch.zeros_like(params)
        hist = torch.zeros(30, device="cuda")
        prob.train_steps(params, m, v, 0, 30, n, lr=1e-3, seed=7, loss_hist=hist)
        runs.append((params.clone(), hist.cpu().numpy()))
    assert torch.equal(runs[0][0], runs[1][0])
    h = runs[0][1]
    assert np.all(np.isfinite(h)) and h[-5:].mean() < h[:5].mean()
    # the first step's loss is the refined residual of the initial parameters at
    # the step-1 points (band points drawn within 4 h of the base spacing)
    p0 = nbm.xavier_init(d, seed=2, device="cuda")
    pts = prob.sample_points(n, seed=7, step=1)
    l0, _ = prob.residual(p0, pts)
    assert abs(h[0] - l0) <= 1e-6 * l0


def test_refinement_level_limits():
    import paper_2210_14907_gb300 as nbm
    with pytest.raises(nbm.NBMError) as e:
        nbm.Problem(nbm.ProblemDesc(refine_levels=4))
    assert e.value.code == 1
    with pytest.raises(nbm.NBMError) as e:
        nbm.Problem(nbm.ProblemDesc(h=2 / 4096, refine_levels=2))
    assert e.value.code == 1
