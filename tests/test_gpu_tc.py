"""Parity of the BF16 tcgen05 path with the FP64 oracle (through the C ABI).

Tolerances (mixed path): residual and loss relative error <= 2e-3, gradient
relative error (2-norm) <= 5e-3.  The residual r_p is checked norm-wise over the
batch against that bar and point by point against the bound of tests/parity.py
(4 BF16 unit roundoffs relative, plus the rounding of the network values in a
cut cell's jump row).
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs, parity

pytestmark = pytest.mark.gpu

RES_TOL, LOSS_TOL, GRAD_TOL = 2e-3, 2e-3, 5e-3


def _nbm():
    import paper_2210_14907_gb300 as nbm
    return nbm


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _pair(geom, L, h, mu_p, prec, fp64=-1, band=0.0):
    nbm = _nbm()
    d = nbm.ProblemDesc(geometry=geom, n_hidden=L, width=128, precision=prec, mu_minus=1.0,
                        mu_plus=mu_p, h=h, band_fraction=band, fp64_stencil=fp64)
    o = O.make_problem(geometry=geom, n_hidden=L, width=128, mu_minus=1.0, mu_plus=mu_p, h=h)
    return nbm.Problem(d), o


CASES = [
    # geometry, L, h, mu+, n_uniform, n_shell, fp64 rows
    (O.GEOM_SPHERE, 3, 2 / 128, 10.0, 1500, 500, 0),   # C2 architecture
    (O.GEOM_FLOWER, 4, 2 / 256, 100.0, 700, 700, 0),   # C3 architecture, many cut cells
    (O.GEOM_SPHERE, 4, 2 / 1024, 10.0, 600, 200, 1),   # C4 resolution, FP64 rows
    (O.GEOM_SPHERE, 2, 2 / 64, 10.0, 800, 200, 0),     # one hidden GEMM
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"g{c[0]}L{c[1]}n{round(2 / c[2])}")
def test_bf16_residual_loss_gradient_match_oracle(case):
    nbm = _nbm()
    geom, L, h, mu_p, nu, ns, fp64 = case
    prob, o = _pair(geom, L, h, mu_p, nbm.PREC_BF16, fp64)
    pts = inputs.mixed_points(nu, ns, seed=L + 100)
    th = inputs.glorot_params(128, L, seed=8, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts.astype(np.float32)).cuda()
    loss, r2 = prob.residual(tp, tx)
    loss2, g = prob.loss_grad(tp, tx)
    er = _rel(np.sqrt(r2.cpu().numpy()), np.sqrt(r2_ref))
    el = abs(loss - L_ref) / L_ref
    eg = _rel(g.cpu().numpy(), g_ref)
    print(f"bf16 case {case[:3]}: residual {er:.2e} loss {el:.2e} grad {eg:.2e}")
    assert er <= RES_TOL and el <= LOSS_TOL and abs(loss2 - L_ref) / L_ref <= LOSS_TOL
    assert eg <= GRAD_TOL
    parity.check_points(o, th, pts, r2.cpu().numpy(), r2_ref, *parity.bf16_tols(L),
                        label=f"bf16 {case[:3]}")


def test_bf16_ragged_and_tiny_batches():
    nbm = _nbm()
    prob, o = _pair(O.GEOM_SPHERE, 3, 2 / 32, 10.0, nbm.PREC_BF16)
    th = inputs.glorot_params(128, 3, seed=5, bias_scale=0.1)
    for n in (1, 15, 17, 33):
        pts = inputs.mixed_points(max(n - 6, 0), 0, seed=n)[-n:]
        L_ref, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
        loss, g = prob.loss_grad(torch.from_numpy(th).cuda(), torch.from_numpy(pts.astype(np.float32)).cuda())
        assert abs(loss - L_ref) / L_ref <= LOSS_TOL, n
        assert _rel(g.cpu().numpy(), g_ref) <= GRAD_TOL, n


def test_bf16_adam_trajectory_follows_the_oracle():
    """C2 architecture (sphere, h = 2/128, 3 -> 128^3 -> 1), 16,384 device-drawn
    points per step, 10 Adam steps of the mixed path against the oracle's own
    training loop from the same parameters (nbo_train: same Philox points, FP64
    forward, gradient and Adam)."""
    nbm = _nbm()
    d = nbm.config("C2")
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=3, width=128, mu_minus=1.0,
                       mu_plus=10.0, h=2 / 128)
    th = inputs.glorot_params(128, 3, seed=0)
    steps, batch, lr = 10, 16384, 1e-3
    th_o = th.astype(np.float64)
    m_o = np.zeros_like(th_o)
    v_o = np.zeros_like(th_o)
    hist_o = O.train(o, th_o, m_o, v_o, 0, steps, batch, 0, lr=lr, seed=1)
    tp = torch.from_numpy(th).cuda()
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    hist = torch.zeros(steps, device="cuda")
    prob.train_steps(tp, m, v, 0, steps, batch, lr=lr, seed=1, loss_hist=hist)
    hist = hist.cpu().numpy()
    got = tp.cpu().numpy().astype(np.float64)
    # every step's loss within the mixed path's loss tolerance
    assert np.max(np.abs(hist - hist_o) / hist_o) <= LOSS_TOL
    # the parameters after 10 updates: Adam moves each component by about lr per
    # step whatever its gradient's size, so a component whose gradient is within
    # the BF16 error of zero may move the other way (measured: 0.07 % of them by
    # more than lr/2); all together they stay within the gradient tolerance
    assert _rel(got, th_o) <= GRAD_TOL
    moved = np.abs((got - th) - (th_o - th))
    assert np.mean(moved > 0.5 * lr) <= 1e-2
    assert moved.max() <= 2 * steps * lr


def test_bf16_deterministic_and_resumable():
    nbm = _nbm()
    d = nbm.config("C3")
    prob = nbm.Problem(d)
    th = inputs.glorot_params(128, 4, seed=1)
    outs = []
    for split in ((6,), (3, 3)):
        tp = torch.from_numpy(th).cuda()
        m = torch.zeros_like(tp)
        v = torch.zeros_like(tp)
        s = 0
        for k in split:
            s = prob.train_steps(tp, m, v, s, k, 20000, seed=3)
        outs.append((tp, m, v))
    for x, y in zip(outs[0], outs[1]):
        assert torch.equal(x, y)


def test_checkpoint_resume_in_a_new_problem_is_bitwise(tmp_path):
    """Elastic recovery is resume from a checkpoint: 10 steps equal 5 steps, a
    checkpoint written to disk, a fresh problem object and 5 more steps."""
    nbm = _nbm()
    d = nbm.config("C2")
    full = nbm.Problem(d)
    p = nbm.xavier_init(d, seed=4, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    full.train_steps(p, m, v, 0, 10, 16384, seed=9)
    a = nbm.Problem(d)
    q = nbm.xavier_init(d, seed=4, device="cuda")
    mq = torch.zeros_like(q)
    vq = torch.zeros_like(q)
    s = a.train_steps(q, mq, vq, 0, 5, 16384, seed=9)
    nbm.save_checkpoint(tmp_path / "ck.pt", d, q, mq, vq, s, 9)
    del a, q, mq, vq
    d2, q, mq, vq, s, seed = nbm.load_checkpoint(tmp_path / "ck.pt")
    b = nbm.Problem(d2)
    b.train_steps(q, mq, vq, s, 5, 16384, seed=seed)
    for x, y in ((p, q), (m, mq), (v, vq)):
        assert torch.equal(x, y)


@pytest.mark.parametrize("prec,H,L,tol_r,tol_g", [(0, 64, 2, 1e-5, 1e-4), (1, 128, 3, 2e-3, 5e-3)],
                         ids=["fp32", "bf16"])
def test_extreme_points_and_corners_on_the_interface(prec, H, L, tol_r, tol_g):
    """Points at the lattice extremes +-(1 - 2^-22) (stencil neighbours leave the
    cube on up to three axes: Dirichlet faces) and cells with a corner exactly on
    the sphere (phi = 0 counts as Omega-), mixed with ordinary points."""
    nbm = _nbm()
    h = 2 / 16
    d = nbm.ProblemDesc(geometry=O.GEOM_SPHERE, n_hidden=L, width=H, precision=prec,
                        mu_minus=1.0, mu_plus=10.0, h=h)
    prob = nbm.Problem(d)
    o = O.make_problem(geometry=O.GEOM_SPHERE, n_hidden=L, width=H, mu_minus=1.0, mu_plus=10.0,
                       h=h)
    e = 1.0 - 2.0 ** -22
    corners = [[sx * e, sy * e, sz * e] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    edges = [[e, 0.3, -e], [-e, 0.0, 0.5], [0.25, e, 0.0]]
    hh = h / 2
    on_gamma = [[0.5 - hh, hh, hh], [-0.5 + hh, -hh, hh], [hh, 0.5 - hh, -hh], [hh, hh, 0.5 + hh],
                [-hh, -hh, -0.5 - hh]]  # one corner of each cell at a pole of the sphere
    for p in on_gamma:
        t = O.cell_geometry(o, np.array(p), h)
        assert t["cut"] in (0, 1)
    pts = np.concatenate([np.array(corners + edges + on_gamma),
                          inputs.mixed_points(200, 100, seed=77)]).astype(np.float32)
    th = inputs.glorot_params(H, L, seed=19, bias_scale=0.1)
    L_ref, r2_ref = O.loss(o, th.astype(np.float64), pts, want_r2=True)
    _, g_ref = O.loss_grad(o, th.astype(np.float64), pts)
    tp = torch.from_numpy(th).cuda()
    tx = torch.from_numpy(pts).cuda()
    loss, r2 = prob.residual(tp, tx)
    _, g = prob.loss_grad(tp, tx)
    r2 = r2.cpu().numpy()
    assert np.all(np.isfinite(r2))
    assert _rel(np.sqrt(r2), np.sqrt(r2_ref)) <= tol_r
    # every point, the 16 special ones included, within its own bound
    tols = parity.bf16_tols(L) if prec == 1 else (tol_r, tol_r)
    parity.check_points(o, th, pts, r2, r2_ref, *tols, label=f"extreme points prec {prec}")
    assert abs(loss - L_ref) <= tol_r * L_ref
    assert _rel(g.cpu().numpy(), g_ref) <= tol_g
