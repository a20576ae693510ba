"""Parity at the benchmark configurations' full sizes.

The fused kernels run on the full batches in the launch configuration bench.py
times (one persistent CTA per SM, device-side sampling), so every CTA carries
a long chain of half-tiles through the TMEM weight-gradient accumulators and
the cross-group ordering of the shared accumulators (about 215 half-tiles per
CTA for 262,144 points, about 860 for C3's 1,048,576):

- C2 (262,144 points) and C3 (1,048,576 points, 30 % band points): every
  point's residual against the oracle (norm-wise and point by point, see
  tests/parity.py), and the whole gradient against the oracle's gradient.
- C4 (h = 2/1024, FP64 rows): a 262,144-point batch of the C4 problem (the
  same launch configuration and chain length per CTA as C2) with every point
  and the whole gradient, and the full 4,194,304-point batch on a sample of
  points plus properties that hold at any size (the loss is the mean of the
  per-point residuals; loss and gradient finite and nonzero).

The points are read back from the device sampler and fed to the oracle as
inputs (the sampler's own parity is tested separately).
"""
import numpy as np
import pytest
import torch

from oracle import pyoracle as O
from tests import inputs, parity

pytestmark = pytest.mark.gpu

RES_TOL, LOSS_TOL, GRAD_TOL = 2e-3, 2e-3, 5e-3

CFG = {
    "C2": dict(geom=O.GEOM_SPHERE, L=3, h=2 / 128, mu_p=10.0),
    "C3": dict(geom=O.GEOM_FLOWER, L=4, h=2 / 256, mu_p=100.0),
    "C4": dict(geom=O.GEOM_SPHERE, L=4, h=2 / 1024, mu_p=10.0),
}


def _setup(name):
    import paper_2210_14907_gb300 as nbm
    c = CFG[name]
    prob = nbm.Problem(nbm.config(name))
    o = O.make_problem(geometry=c["geom"], n_hidden=c["L"], width=128, mu_minus=1.0,
                       mu_plus=c["mu_p"], h=c["h"])
    th = inputs.glorot_params(128, c["L"], seed=31, bias_scale=0.1)
    return prob, o, th, c["L"]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name, n", [("C2", 262_144), ("C3", 1_048_576), ("C4", 262_144)])
def test_full_batch_every_point_and_gradient_against_oracle(name, n):
    prob, o, th, L = _setup(name)
    tp = torch.from_numpy(th).cuda()
    pts = prob.sample_points(n, seed=1, step=7)
    loss, r2 = prob.residual(tp, pts)
    loss_g, g = prob.loss_grad(tp, pts)
    p = pts.cpu().numpy().astype(np.float64)
    thd = th.astype(np.float64)
    L_ref, r2_ref = O.loss(o, thd, p, want_r2=True)
    r2 = r2.cpu().numpy().astype(np.float64)
    er = _rel(np.sqrt(r2), np.sqrt(r2_ref))
    el = abs(loss - L_ref) / L_ref
    print(f"{name} {n} points: residual {er:.2e}, loss {el:.2e}")
    assert er <= RES_TOL and el <= LOSS_TOL and abs(loss_g - L_ref) / L_ref <= LOSS_TOL
    parity.check_points(o, thd, p, r2, r2_ref, *parity.bf16_tols(L), label=f"{name} {n}")
    _, g_ref = O.loss_grad(o, thd, p)
    eg = _rel(g.cpu().numpy(), g_ref)
    half = len(g_ref) // 2
    print(f"{name} {n} points: gradient {eg:.2e} (net-: {_rel(g.cpu().numpy()[:half], g_ref[:half]):.2e},"
          f" net+: {_rel(g.cpu().numpy()[half:], g_ref[half:]):.2e})")
    assert eg <= GRAD_TOL


def test_c4_full_batch_sampled_against_oracle():
    """The full 4,194,304-point C4 batch: a sample of points (the ones nearest the
    interface over-represented) against the oracle one point at a time, and
    properties that hold at any size."""
    prob, o, th, L = _setup("C4")
    tp = torch.from_numpy(th).cuda()
    n = 4_194_304
    pts = prob.sample_points(n, seed=1, step=7)
    loss, r2 = prob.residual(tp, pts)
    r2 = r2.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(r2)) and np.isfinite(loss)
    assert abs(r2.mean() - loss) <= 1e-5 * loss  # the loss is the mean of the point residuals
    p = pts.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(0)
    idx = rng.choice(n, size=2048, replace=False)
    near = np.argsort(np.abs(np.sqrt((p ** 2).sum(1)) - 0.5))[:512]
    idx = np.unique(np.concatenate([idx, near]))
    thd = th.astype(np.float64)
    ref = np.array([O.point_terms(o, thd, p[i])["r2"] for i in idx])
    got = r2[idx]
    assert _rel(np.sqrt(got), np.sqrt(ref)) <= RES_TOL
    parity.check_points(o, thd, p[idx], got, ref, *parity.bf16_tols(L), label="C4 sample")
    _, g = prob.loss_grad(tp, pts)
    g = g.cpu().numpy()
    half = len(g) // 2
    assert np.all(np.isfinite(g)) and np.abs(g[:half]).max() > 0 and np.abs(g[half:]).max() > 0
