"""Per-point residual parity between a CUDA path and the FP64 oracle.

For every collocation point i the CUDA residual r_i = sqrt(r_i^2) must satisfy

    |r_i - r_i^ref| <= tol * max(r_i^ref, FLOOR * rms(r^ref)) + tol_jump * s_i,

where r^ref is the oracle's residual, rms(r^ref) its root mean square over the
batch, and s_i = |U+(x_G)| + |U-(x_G)| + |alpha(x_G)| for a cut cell with a
value-jump row (0 for every other point), all from the oracle.

Why the two terms:
- Every row except the jump row is computed from difference-form columns
  (centre value, O(h^2) symmetric and O(h) antisymmetric increments), so its
  rounding error is relative to the row itself; the floor (1 % of the batch's
  rms) only matters for points whose residual happens to vanish.
- The jump row J = U+(x_G) - U-(x_G) - alpha(x_G) subtracts O(1) network values,
  so its error is the rounding of those values, not a fraction of J.

Tolerances: the FP32 path takes the benchmark's FP32 bar 1e-5 for both terms.
The BF16 path rounds every hidden GEMM operand (weights and activations) to
BF16, unit roundoff u = 2^-9: tol = 4u per point (the norm-wise bar of 2e-3 over
the batch stays, and is checked separately) and tol_jump = 4 L u for L hidden
layers (two rounded operands per layer, in each of the two networks).
"""
import numpy as np

from oracle import pyoracle as O

FLOOR = 0.01
U_BF16 = 2.0 ** -9


def bf16_tols(n_hidden):
    return 4 * U_BF16, 4 * n_hidden * U_BF16


def jump_scale(o, theta, pts):
    """s_i of the bound above for every point: |U+(x_G)| + |U-(x_G)| + |alpha(x_G)|
    for cut cells with an interface (S > 0), else 0.  Only points within a few
    cells of the interface can be cut; the others are skipped by a cheap radius
    test first (the sphere's and the flower's phi are r - R with R in
    [r0 - amp, r0 + amp])."""
    theta = np.asarray(theta, np.float64)
    pts = np.asarray(pts, np.float64)
    s = np.zeros(len(pts))
    h = o.h
    reach = 4 * h
    rad = np.sqrt((pts ** 2).sum(1))
    if o.geometry == O.GEOM_SPHERE:
        near = np.abs(rad - o.r0) < reach
    elif o.geometry == O.GEOM_FLOWER:
        near = np.abs(rad - o.r0) < abs(o.amp) + reach
    else:  # any other level set: every point
        near = np.ones(len(pts), bool)
    pn = O.params_per_net(o)
    for i in np.where(near)[0]:
        g = O.cell_geometry(o, pts[i])
        if g["cut"] and g["S"] > 0:
            xg = g["xg"]
            s[i] = (abs(O.mlp_eval(o, theta[:pn], xg)) + abs(O.mlp_eval(o, theta[pn:], xg))
                    + abs(O.alpha(o, xg)))
    return s


def worst_ratio(r2_gpu, r2_ref, s, tol, tol_jump):
    """max over the points of |r_i - r_i^ref| / bound_i (the check passes at <= 1)."""
    r = np.sqrt(np.asarray(r2_gpu, np.float64))
    rr = np.sqrt(np.asarray(r2_ref, np.float64))
    rms = np.sqrt(np.mean(rr ** 2))
    bound = tol * np.maximum(rr, FLOOR * rms) + tol_jump * s
    return float(np.max(np.abs(r - rr) / bound))


def check_points(o, theta, pts, r2_gpu, r2_ref, tol, tol_jump, label=""):
    q = worst_ratio(r2_gpu, r2_ref, jump_scale(o, theta, pts), tol, tol_jump)
    print(f"{label} per-point residual: worst |r - r_ref| / bound = {q:.3f}")
    assert q <= 1.0, f"{label}: a point's residual is off by {q:.2f} x its bound"
    return q
