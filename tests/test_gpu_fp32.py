"""Parity of the FP32 CUDA path with the FP64 oracle (through the C ABI).

Tolerances (FP32 path): residual and loss relative error <= 1e-5, gradient
relative error (2-norm) <= 1e-4.  The residual r_p = sqrt(r_p^2) is checked
norm-wise over the batch and point by point (tests/parity.py, at 1e-5 for
both terms of its bound).
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs, parity

pytestmark = pytest.mark.gpu

RES_TOL, LOSS_TOL, GRAD_TOL = 1e-5, 1e-5, 1e-4


def _nbm():
    import paper_2210_14907_gb300 as nbm
    return nbm


def _pair(geom, H, L, h, mu_m=1.0, mu_p=10.0, k_m=0.0, k_p=0.0, prec=0, band=0.0):
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=H, precision=prec, mu_minus=mu_m,
                        mu_plus=mu_p, k_minus=k_m, k_plus=k_p, h=h, band_fraction=band)
    o = O.make_problem(geometry=geom, n_hidden=L, width=H, mu_minus=mu_m, mu_plus=mu_p,
                       k_minus=k_m, k_plus=k_p, h=h)
    return nbm.Problem(d), o


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    # geometry, H, L, h, mu-, mu+, k-, k+, n_uniform, n_shell
    (O.GEOM_SPHERE, 64, 2, 2 / 32, 1.0, 10.0, 0.0, 0.0, 3000, 1000),
    (O.GEOM_FLOWER, 64, 3, 2 / 64, 1.0, 100.0, 0.0, 0.0, 1500, 1500),
    (O.GEOM_SPHERE, 128, 4, 2 / 128, 1.0, 10.0, 0.5, 2.0, 600, 400),
    (O.GEOM_FLOWER, 128, 3, 2 / 256, 1.0, 100.0, 0.0, 0.0, 500, 500),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"g{c[0]}H{c[1]}L{c[2]}n{round(2 / c[3])}")
def test_residual_loss_gradient_match_oracle(case):
    geom, H, L, h, mm, mp, km, kp, nu, ns = case
    prob, o = _pair(geom, H, L, h, mm, mp, km, kp)
    pts = inputs.mixed_points(nu, ns, seed=H + L)
    th = inputs.glorot_params(H, L, seed=7, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)

    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    r2 = r2.cpu().numpy().astype(np.float64)
    assert _rel(np.sqrt(r2), np.sqrt(r2_ref)) <= RES_TOL
    parity.check_points(o, th, pts, r2, r2_ref, RES_TOL, RES_TOL, label=f"fp32 {case[:4]}")
    assert abs(loss - L_ref) / L_ref <= LOSS_TOL
    assert abs(loss2 - L_ref) / L_ref <= LOSS_TOL
    assert _rel(g.cpu().numpy(), g_ref) <= GRAD_TOL


def test_sampler_matches_oracle():
    nbm = _nbm()
    h = 2 / 256
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, n_hidden=2, width=64, h=h, band_fraction=0.3)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_FLOWER, h=h)
    n = 20000
    nb = int(np.floor(0.3 * n + 0.5))
    got = prob.sample_points(n, seed=1, step=3).cpu().numpy().astype(np.float64)
    ref = O.sample_points(o, 1, 3, n, nb)
    assert np.array_equal(got[: n - nb], ref[: n - nb])  # integer lattice draws: bit-exact
    q = np.abs(got[n - nb:] - ref[n - nb:]) / 2.0 ** -22  # FP64 transcendentals: <= 1 quantum
    assert q.max() <= 1.0 and np.mean(q == 0) > 0.999


@pytest.mark.parametrize("n", [1, 7, 9, 63])
def test_tiny_and_ragged_batches(n):
    prob, o = _pair(O.GEOM_SPHERE, 64, 2, 2 / 16)
    pts = inputs.mixed_points(max(n - 6, 0), 0, seed=n)[-n:]
    th = inputs.glorot_params(64, 2, seed=3, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    _, g = prob.loss_grad(tp, tx)
    assert _rel(np.sqrt(r2.cpu().numpy()), np.sqrt(r2_ref)) <= RES_TOL
    parity.check_points(o, th, pts, r2.cpu().numpy(), r2_ref, RES_TOL, RES_TOL, label=f"n={n}")
    assert abs(loss - L_ref) / L_ref <= LOSS_TOL
    assert _rel(g.cpu().numpy(), g_ref) <= GRAD_TOL


def test_single_phase_and_all_cut_batches():
    # no interface: every point in one list, the other network gets zero gradient
    prob, o = _pair(O.GEOM_ALL_MINUS, 64, 2, 2 / 32, mu_m=2.0, k_m=1.0)
    pts = inputs.uniform_points(700, seed=5)
    th = inputs.glorot_params(64, 2, seed=4)
    L_ref, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    loss, g = prob.loss_grad(torch.from_numpy(th).cuda(), torch.from_numpy(pts.astype(np.float32)).cuda())
    g = g.cpu().numpy()
    assert abs(loss - L_ref) / L_ref <= LOSS_TOL and _rel(g, g_ref) <= GRAD_TOL
    assert np.all(g[len(g) // 2:] == 0.0)
    # every cell cut: points hugging the sphere with a coarse cell
    prob, o = _pair(O.GEOM_SPHERE, 64, 2, 2 / 8)
    pts = inputs.shell_points(500, seed=6, r_lo=0.48, r_hi=0.52)
    assert all(O.cell_geometry(o, p)["cut"] for p in pts)
    L_ref, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    loss, g = prob.loss_grad(torch.from_numpy(th).cuda(), torch.from_numpy(pts.astype(np.float32)).cuda())
    assert abs(loss - L_ref) / L_ref <= LOSS_TOL and _rel(g.cpu().numpy(), g_ref) <= GRAD_TOL


def test_train_steps_follow_oracle_trajectory():
    """C1 shape: 20 Adam steps on 4096 sampled points per step, vs the oracle's own loop."""
    nbm = _nbm()
    d = nbm.config("C1")
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=2, width=64, mu_minus=1.0, mu_plus=10.0,
                       h=2 / 32)
    th = inputs.glorot_params(64, 2, seed=0)
    steps, batch = 20, 4096
    th_o = th.astype(np.float64)
    m_o = np.zeros_like(th_o)
    v_o = np.zeros_like(th_o)
    hist_o = O.train(o, th_o, m_o, v_o, 0, steps, batch, 0, lr=1e-3, seed=1)
    tp = torch.from_numpy(th).cuda()
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    hist = torch.zeros(steps, device="cuda")
    st = prob.train_steps(tp, m, v, 0, steps, batch, lr=1e-3, seed=1, loss_hist=hist)
    assert st == steps
    hist = hist.cpu().numpy()
    assert np.max(np.abs(hist - hist_o) / hist_o) < 1e-4
    assert _rel(tp.cpu().numpy(), th_o) < 1e-5
    # resume: 10 + 10 steps reproduce 20 steps bitwise
    tp2 = torch.from_numpy(th).cuda()
    m2 = torch.zeros_like(tp2)
    v2 = torch.zeros_like(tp2)
    s = prob.train_steps(tp2, m2, v2, 0, 10, batch, lr=1e-3, seed=1)
    s = prob.train_steps(tp2, m2, v2, s, 10, batch, lr=1e-3, seed=1)
    assert torch.equal(tp2, tp) and torch.equal(m2, m) and torch.equal(v2, v)


def test_autograd_function_backward_is_libnbm_gradient():
    nbm = _nbm()
    prob, o = _pair(O.GEOM_SPHERE, 64, 2, 2 / 32)
    pts = torch.from_numpy(inputs.mixed_points(300, 100, seed=9).astype(np.float32)).cuda()
    th = torch.from_numpy(inputs.glorot_params(64, 2, seed=2)).cuda().requires_grad_(True)
    loss = nbm.NBMLoss.apply(prob, th, pts)
    loss.backward()
    l2, g = prob.loss_grad(th.detach(), pts)
    assert torch.equal(th.grad, g)
    # no gradient needed: the forward alone (nbm_residual), the same loss
    with torch.no_grad():
        l0 = nbm.NBMLoss.apply(prob, th, pts)
    l1 = nbm.NBMLoss.apply(prob, th.detach(), pts)
    assert not l0.requires_grad and not l1.requires_grad
    assert float(l0) == float(l1) == prob.residual(th.detach(), pts, want_r2=False)[0]
    assert abs(float(l0) - l2) <= 1e-6 * l2
    # the points are not differentiated
    with pytest.raises(ValueError):
        nbm.NBMLoss.apply(prob, th, pts.clone().requires_grad_(True))


def test_invalid_arguments_fail_cleanly():
    nbm = _nbm()
    prob, _ = _pair(O.GEOM_SPHERE, 64, 2, 2 / 32)
    th = torch.zeros(prob.P, device="cuda")
    with pytest.raises(nbm.NBMError) as e:
        prob.loss_grad(th, n=0)
    assert e.value.code == 1
    # one point over the largest batch: refused on the host before any allocation
    with pytest.raises(nbm.NBMError) as e:
        prob.loss_grad(th, n=2**30 + 1)
    assert e.value.code == 1
    with pytest.raises(nbm.NBMError) as e:
        prob.train_steps(th, torch.zeros_like(th), torch.zeros_like(th), 0, 1, 2**30 + 1)
    assert e.value.code == 1
    bad = torch.full((prob.P,), float("nan"), device="cuda")
    with pytest.raises(nbm.NBMError) as e:
        prob.loss_grad(bad, n=256)
    assert e.value.code == 4
    # the problem object stays usable after a rejected call
    loss, _ = prob.loss_grad(torch.from_numpy(inputs.glorot_params(64, 2, 1)).cuda(), n=256)
    assert np.isfinite(loss)


@pytest.mark.parametrize("lobes", [(5.0, 3.0), (4.5, 2.5)], ids=["integer", "fractional"])
def test_flower_lobes_match_oracle(lobes):
    """The flower's angular factor sin(lt theta) cos(lp psi) is evaluated by
    Chebyshev recurrences for integer lobe counts and through the angles
    otherwise; both against the oracle, which always takes the angles."""
    nbm = _nbm()
    lt, lp = lobes
    h = 2 / 64
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, n_hidden=3, width=64, h=h, mu_minus=1.0,
                        mu_plus=100.0, lobes_theta=lt, lobes_psi=lp)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_FLOWER, n_hidden=3, width=64, h=h, mu_minus=1.0,
                       mu_plus=100.0, lobes_theta=lt, lobes_psi=lp)
    pts = inputs.mixed_points(1500, 1500, seed=11)
    th = inputs.glorot_params(64, 3, seed=7, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    r2 = r2.cpu().numpy().astype(np.float64)
    assert _rel(np.sqrt(r2), np.sqrt(r2_ref)) <= RES_TOL
    parity.check_points(o, th, pts, r2, r2_ref, RES_TOL, RES_TOL, label=f"flower lobes {lobes}")
    assert abs(loss - L_ref) / L_ref <= LOSS_TOL
    assert abs(loss2 - L_ref) / L_ref <= LOSS_TOL
    assert _rel(g.cpu().numpy(), g_ref) <= GRAD_TOL


def test_sampler_matches_oracle_fractional_lobes():
    """Band points of a flower whose lobe counts are not integers (the draw's
    angular factor through the angles, on the draw's own azimuth)."""
    nbm = _nbm()
    h = 2 / 256
    d = nbm.ProblemDesc(geometry=nbm.GEOM_FLOWER, n_hidden=2, width=64, h=h, band_fraction=0.3,
                        lobes_theta=4.5, lobes_psi=2.5)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_FLOWER, h=h, lobes_theta=4.5, lobes_psi=2.5)
    n = 20000
    nb = int(np.floor(0.3 * n + 0.5))
    got = prob.sample_points(n, seed=2, step=5).cpu().numpy().astype(np.float64)
    ref = O.sample_points(o, 2, 5, n, nb)
    assert np.array_equal(got[: n - nb], ref[: n - nb])
    q = np.abs(got[n - nb:] - ref[n - nb:]) / 2.0 ** -22
    assert q.max() <= 1.0 and np.mean(q == 0) > 0.999
