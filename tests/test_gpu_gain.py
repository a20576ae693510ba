"""What the trained surrogate gains over the plain method without it.

The plain method is the grid solve of the same finite-volume scheme at the
same h; between its nodes a user interpolates.  Trilinear interpolation of the
raw node values smears the solution across the interface; the scheme's own
extension of each side across Gamma (a node of the other side carried over by
the node jump J = u+ - u-, nbm_grid_node_jump) does not.  The NBM surrogate
(trained only on residuals of the discretization, Sec. 3) is evaluated
directly at any point with the network of the point's side.

Asserted: near the interface the surrogate's L-infinity error is clearly below
that of the raw interpolation; the jump-aware interpolation is in turn far
below both (the converged grid solve is second order, the surrogate is limited
by its training length); the surrogate takes at least 50x less memory than
the grid solution.  The numbers are printed for each comparison.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _exact(x):
    r = np.sqrt((x ** 2).sum(1))
    um = np.exp(x[:, 0]) * np.cos(x[:, 1]) * np.sin(x[:, 2])
    return np.where(r <= 0.5, um, (x ** 2).sum(1))


def _trilinear(u, n, x, jump=None):
    """Trilinear interpolation of node values; with the node jump J = u+ - u-,
    each corner is first carried to the point's side (sphere r0 = 1/2)."""
    U = u.reshape(n + 1, n + 1, n + 1)
    Jn = None if jump is None else jump.reshape(n + 1, n + 1, n + 1)
    side = (np.sqrt((x ** 2).sum(1)) > 0.5).astype(int)
    t = (x + 1.0) * n / 2.0
    i0 = np.clip(np.floor(t).astype(int), 0, n - 1)
    f = t - i0
    g = -1.0 + np.arange(n + 1) * 2.0 / n
    out = np.zeros(len(x))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                k, j, i = i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx
                val = U[k, j, i]
                if Jn is not None:
                    sq = (np.sqrt(g[i] ** 2 + g[j] ** 2 + g[k] ** 2) > 0.5).astype(int)
                    val = val + np.where(sq == side, 0.0, np.where(side == 1, 1.0, -1.0) * Jn[k, j, i])
                out += w * val
    return out


def test_surrogate_against_the_grid_solve_between_nodes():
    import paper_2210_14907_gb300 as nbm
    d = nbm.config("C2")  # sphere, mu 1/10, h = 2/128, 3->128^3->1, BF16 tensor cores
    prob = nbm.Problem(d)
    params = nbm.xavier_init(d, seed=0, device="cuda")
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    hist = torch.zeros(3000, device="cuda")
    prob.train_steps(params, m, v, 0, 3000, 262_144, lr=1e-3, seed=1, loss_hist=hist)
    h = hist.cpu().numpy()
    assert np.all(np.isfinite(h)) and h[-100:].mean() < 0.01 * h[:10].mean()
    n = 128
    ucg, it, rr, ok = prob.grid_cg_solve(n, rtol=1e-10)
    assert ok
    # the plain method with its own extrapolated jump, and that jump at the nodes
    pj = nbm.Problem(nbm.ProblemDesc(geometry=nbm.GEOM_SPHERE, mu_minus=1.0, mu_plus=10.0,
                                     grid_jump=nbm.JUMP_EXTRAP))
    uj, _, _, ok = pj.grid_cg_solve(n, rtol=1e-10)
    assert ok
    jn = pj.grid_node_jump(n, nbm.JUMP_EXTRAP, uj).cpu().numpy()
    ucg = ucg.cpu().numpy()
    uj = uj.cpu().numpy()
    rng = np.random.default_rng(0)
    dirs = rng.normal(size=(50_000, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    near = dirs * (0.5 + rng.uniform(-4.0 / n, 4.0 / n, len(dirs)))[:, None]
    ex = _exact(near)
    us = prob.eval_points(params, torch.from_numpy(near.astype(np.float32)).cuda()).cpu().numpy()
    es = np.abs(us - ex)
    eg = np.abs(_trilinear(ucg, n, near) - ex)
    ej = np.abs(_trilinear(uj, n, near, jn) - ex)
    print(f"near interface: surrogate linf {es.max():.3f} rmse {np.sqrt((es ** 2).mean()):.3f}; "
          f"grid CG + trilinear linf {eg.max():.3f} rmse {np.sqrt((eg ** 2).mean()):.3f}; "
          f"grid CG (extrapolated jump) + jump-aware trilinear linf {ej.max():.2e} "
          f"rmse {np.sqrt((ej ** 2).mean()):.2e}")
    assert es.max() < 0.5 * eg.max()
    assert ej.max() < 0.1 * es.max()
    assert params.numel() * 4 * 50 < (n + 1) ** 3 * 8  # >= 50x less memory than the grid solution


def test_eval_points_matches_eval_grid_on_nodes():
    import paper_2210_14907_gb300 as nbm
    d = nbm.config("C3")
    prob = nbm.Problem(d)
    params = nbm.xavier_init(d, seed=4, device="cuda")
    n = 16  # dyadic: node coordinates are exact in FP32 on both sides
    g = -1.0 + np.arange(n + 1) * 2.0 / n
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    pts = torch.from_numpy(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1).astype(np.float32)).cuda()
    for prec in (nbm.PREC_FP32, nbm.PREC_FP16):
        a = prob.eval_grid(params, n, precision=prec)
        b = prob.eval_points(params, pts, precision=prec)
        assert torch.equal(a, b)
