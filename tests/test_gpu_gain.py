"""What the trained surrogate gains over the plain method without it.

The plain method is the grid CG solve of the same finite-volume scheme at the
same h (nbm_grid_cg_solve); between its nodes a user interpolates, and
trilinear interpolation smears the solution across the interface.  The NBM
surrogate (trained only on residuals of the discretization, Sec. 3) is
evaluated directly at any point with the network of the point's side.  Near
the interface (the paper's motivation: smoothing "introduces unphysical
characteristics") the surrogate's L-infinity error must be clearly lower, at a
small fraction of the memory.  Away from the interface the converged grid
solution is more accurate; that is reported, not asserted.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _exact(x):
    r = np.sqrt((x ** 2).sum(1))
    um = np.exp(x[:, 0]) * np.cos(x[:, 1]) * np.sin(x[:, 2])
    return np.where(r <= 0.5, um, (x ** 2).sum(1))


def _trilinear(u, n, x):
    U = u.reshape(n + 1, n + 1, n + 1)
    t = (x + 1.0) * n / 2.0
    i0 = np.clip(np.floor(t).astype(int), 0, n - 1)
    f = t - i0
    out = np.zeros(len(x))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                     * (f[:, 2] if dz else 1 - f[:, 2]))
                out += w * U[i0[:, 2] + dz, i0[:, 1] + dy, i0[:, 0] + dx]
    return out


def test_surrogate_beats_interpolated_grid_solve_near_interface():
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
    ucg = ucg.cpu().numpy()
    rng = np.random.default_rng(0)
    dirs = rng.normal(size=(50_000, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    near = dirs * (0.5 + rng.uniform(-4.0 / n, 4.0 / n, len(dirs)))[:, None]
    ex = _exact(near)
    us = prob.eval_points(params, torch.from_numpy(near.astype(np.float32)).cuda()).cpu().numpy()
    es = np.abs(us - ex)
    eg = np.abs(_trilinear(ucg, n, near) - ex)
    print(f"near interface: surrogate linf {es.max():.3f} rmse {np.sqrt((es ** 2).mean()):.3f}; "
          f"grid CG + trilinear linf {eg.max():.3f} rmse {np.sqrt((eg ** 2).mean()):.3f}")
    assert es.max() < 0.5 * eg.max()
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
