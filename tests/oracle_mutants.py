"""Mutation check of the oracle's CPU pins: does a plausible mistake fail one?

Each mutant plants one mistake (a dropped term, a wrong sign, index or
operand, a changed convention) in a temporary copy of oracle/.  The script
then runs the oracle pins on that copy.  A mutant is "killed" when at least
one pin fails.  Mutants marked equivalent change nothing on any input the
oracle supports; the reason is given with each.

    python tests/oracle_mutants.py [-j JOBS] [NAME ...]

Exit status 0 when every non-equivalent mutant is killed.  The script runs
the CPU tests only, on copies; it does not touch oracle/ itself.  pytest does
not collect it (no test_ prefix): the full run takes a few minutes.
"""
import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = "oracle/nbm_oracle.c"
P = "oracle/pyoracle.py"
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_conventions.py",
        "tests/test_grid_identities.py"]

# The Sec. 4.1 pair has grad mu . grad u = 0 on both sides: mu- varies in x, y
# where u- = e^z does not; mu+ = e^-z varies in z where u+ = cos x sin y does not.
SEC41_ORTH = "grad mu . grad u vanishes identically for the Sec. 4.1 pair"

# (name, file, text, replacement, reason if equivalent)
MUTANTS = [
    # Philox and the sampler
    ("philox_key1", C, "k1 += W1;", "k1 += W0;", None),
    ("philox_xor", C, "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c1 ^ k1;", None),
    ("sample_lattice", C, "uint64_t k = 1 + (((uint64_t)r[j] * 8388607ull) >> 32);",
     "uint64_t k = 1 + (((uint64_t)r[j] * 8388606ull) >> 32);", None),
    ("sample_ctr", C, "uint32_t ctr[4] = {(uint32_t)i, (uint32_t)step,",
     "uint32_t ctr[4] = {(uint32_t)i + 1, (uint32_t)step,", None),
    ("sample_band_width", C, "double t = (2.0 * u[2] - 1.0) * 4.0 * pr->h;",
     "double t = (2.0 * u[2] - 1.0) * 2.0 * pr->h;", None),
    ("sample_band_cth", C, "double cth = 1.0 - 2.0 * u[0];", "double cth = 1.0 - u[0];", None),
    ("sample_split", C, "if (i < n_uniform || !has_iface) {", "if (i <= n_uniform || !has_iface) {",
     None),
    ("quantize_round", C, "double k = floor((v + 1.0) * 4194304.0 + 0.5);",
     "double k = floor((v + 1.0) * 4194304.0);",
     "moves a band point by less than one lattice step, the stated parity bound of band points"),
    # level sets and manufactured data
    ("grid_phi_gy", C, "g[1] = sc * ((c10 - c00) * (1.0 - f[2]) + (c11 - c01) * f[2]);",
     "g[1] = sc * ((c10 - c00) * (1.0 - f[2]) + (c11 - c01) * f[1]);", None),
    ("grid_phi_interp", C, "c1 = c01 * (1.0 - f[1]) + c11 * f[1];",
     "c1 = c01 * (1.0 - f[1]) + c11 * f[0];", None),
    ("flower_sign", C, "return r - pr->r0 - pr->amp * sin(", "return r - pr->r0 + pr->amp * sin(",
     None),
    ("flower_theta", C, "double theta = atan2(sqrt(x[0] * x[0] + x[1] * x[1]), x[2]);",
     "double theta = atan2(x[2], sqrt(x[0] * x[0] + x[1] * x[1]));", None),
    ("flower_dth", C, "-rho / (r * r)};", "rho / (r * r)};", None),
    ("flower_dps", C, "double dphi_dps = a * lp * sin(lt * theta) * sin(lp * psi);",
     "double dphi_dps = -a * lp * sin(lt * theta) * sin(lp * psi);", None),
    ("phase_tie", C, "return nbo_phi(pr, x) <= 0.0 ? 0 : 1;", "return nbo_phi(pr, x) < 0.0 ? 0 : 1;",
     None),
    ("grad_u_y", C, "g[1] = -e * sin(x[1]) * sin(x[2]);", "g[1] = e * sin(x[1]) * sin(x[2]);", None),
    ("lap_sec41", C, "return -2.0 * cos(x[0]) * sin(x[1]);", "return -cos(x[0]) * sin(x[1]);", None),
    ("mu_grad_x", C, "g[0] = x[1] * x[1] / (x[0] + 2.0);", "g[0] = x[1] / (x[0] + 2.0);", SEC41_ORTH),
    ("rhs_gradmu", C, "- nbo_mu(pr, s, x) * exact_laplacian(pr, s, x) -",
     "- nbo_mu(pr, s, x) * exact_laplacian(pr, s, x) +", SEC41_ORTH),
    ("alpha_sign", C, "return nbo_exact_u(pr, 1, x) - nbo_exact_u(pr, 0, x);",
     "return nbo_exact_u(pr, 0, x) - nbo_exact_u(pr, 1, x);", None),
    ("beta_mu", C, "b += (mp * gp[i] - mm * gm[i]) * gphi[i] / nn;",
     "b += (mm * gp[i] - mp * gm[i]) * gphi[i] / nn;", None),
    ("dirichlet_side", C, "int s = (pr->geometry == NBO_GEOM_ALL_MINUS) ? 0 : 1;", "int s = 0;", None),
    # cell geometry
    ("tri_1minus", C, "return 1.0 - (f[c] / (f[c] - f[a])) * (f[c] / (f[c] - f[b]));",
     "return (f[c] / (f[c] - f[a])) * (f[c] / (f[c] - f[b]));", None),
    ("tri_corner", C, "return (f[a] / (f[a] - f[b])) * (f[a] / (f[a] - f[c]));",
     "return (f[a] / (f[a] - f[b])) * (f[a] / (f[a] - f[b]));", None),
    ("tet_22", C, "(C + Dd) * A * B * (A + B)", "(C + Dd) * A * B * (A - B)", None),
    ("tet_lone", C, "prod *= f[lone] / (f[lone] - f[i]);", "prod *= f[lone] / (f[lone] + f[i]);",
     None),
    ("geom_vol", C, "/ 6.0;\n    double ta", "/ 5.0;\n    double ta", None),
    ("geom_face_split", C, "nbo_tri_fraction(F[c00], F[c01], F[c11]));",
     "nbo_tri_fraction(F[c00], F[c01], F[c10]));", None),
    ("geom_S", C, "out->S = area / (h * h);", "out->S = area / h;", None),
    ("geom_newton", C, "for (int i = 0; i < 3; ++i) x[i] -= ph * g[i] / gg;",
     "for (int i = 0; i < 3; ++i) x[i] += ph * g[i] / gg;", None),
    ("edge_cross_t", C, "double t = fu / (fu - fv);", "double t = fv / (fv - fu);", None),
    ("tet_quad_order", C, "tri_area_centroid(Q[0], Q[2], Q[3], &a2, c2);",
     "tri_area_centroid(Q[0], Q[1], Q[3], &a2, c2);", None),
    ("tri_area_half", C, "*area = 0.5 * norm3(cr);", "*area = norm3(cr);", None),
    ("centroid", C, "cen[i] = (a[i] + b[i] + c[i]) / 3.0;", "cen[i] = (a[i] + b[i]) / 2.0;", None),
    # networks
    ("act_dtanh", C, "*dz = 1.0 - t * t;", "*dz = 1.0 - t;", None),
    ("act_dsin", C, "*dz = cos(z);", "*dz = -cos(z);", None),
    ("mlp_w1_index", C, "for (int j = 0; j < 3; ++j) z += W[3 * n + j] * x[j];",
     "for (int j = 0; j < 3; ++j) z += W[n + H * j] * x[j];", None),
    ("mlp_fwd_transpose", C, "for (int k = 0; k < H; ++k) z += Wl[(int64_t)n * H + k] * cur[k];",
     "for (int k = 0; k < H; ++k) z += Wl[(int64_t)k * H + n] * cur[k];", None),
    ("mlp_out_bias", C, "double u = q[H];", "double u = 0.0;", None),
    ("mlp_bwd_transpose", C, "for (int n = 0; n < H; ++n) s += Wl[(int64_t)n * H + k] * gz[n];",
     "for (int n = 0; n < H; ++n) s += Wl[(int64_t)k * H + n] * gz[n];", None),
    ("mlp_bwd_b1", C, "grad[3 * H + n] += gz1;", "grad[3 * H + n] += g[n];", None),
    ("mlp_bwd_bout", C, "grad[off_out + H] += c;", "grad[off_out + H] += 0.0 * c;", None),
    ("mlp_bwd_actderiv", C, "for (int n = 0; n < H; ++n) gz[n] = g[n] * dout[n];",
     "for (int n = 0; n < H; ++n) gz[n] = g[n];", None),
    # point residual, loss and gradient
    ("B_rhs_sign", C, "B += h * h * cell.V[s] * (k * U[s][0] - nbo_rhs_f(pr, s, p));",
     "B += h * h * cell.V[s] * (k * U[s][0] + nbo_rhs_f(pr, s, p));", None),
    ("B_flux_sign", C, "B -= cell.A[s][f] * muf[s][f] * (U[s][1 + f] - U[s][0]);",
     "B += cell.A[s][f] * muf[s][f] * (U[s][1 + f] - U[s][0]);", None),
    ("B_beta_sign", C, "if (has_jump) B += h * cell.S * nbo_beta(pr, cell.xg);",
     "if (has_jump) B -= h * cell.S * nbo_beta(pr, cell.xg);", None),
    ("B_beta_h", C, "if (has_jump) B += h * cell.S * nbo_beta(pr, cell.xg);",
     "if (has_jump) B += h * h * cell.S * nbo_beta(pr, cell.xg);", None),
    ("J_alpha_sign", C, "J = U[1][7] - U[0][7] - nbo_alpha(pr, cell.xg);",
     "J = U[1][7] - U[0][7] + nbo_alpha(pr, cell.xg);", None),
    ("J_at_centroid", C, "for (int i = 0; i < 3; ++i) Q[7][i] = cell.xg[i];",
     "for (int i = 0; i < 3; ++i) Q[7][i] = cell.centroid[i];", None),
    ("D_mu", C, "D += cell.A[s][f] * muf[s][f];", "D += cell.A[s][f];", None),
    ("D_k", C, "D += h * h * cell.V[s] * k;", "D += h * cell.V[s] * k;", None),
    ("mu_face", C, "c[f / 2] += (f & 1) ? 0.5 * h : -0.5 * h;",
     "c[f / 2] += (f & 1) ? -0.5 * h : 0.5 * h;", None),
    ("r2_lambda", C, "double r2 = rB * rB + pr->lambda_jump * J * J;", "double r2 = rB * rB + J * J;",
     None),
    ("dirichlet_both", C,
     "if (e >= 1 && e <= 6 && !inside[e - 1]) {\n        U[s][e] = nbo_dirichlet_g(pr, Q[e]);",
     "if (e >= 1 && e <= 6 && !inside[e - 1]) {\n        U[s][e] = nbo_exact_u(pr, s, Q[e]);",
     "the cube boundary lies in Omega+ for every geometry, so g = u+ there and the minus "
     "network's weight at a boundary vertex is zero"),
    ("outside_strict", C, "return fabs(q[0]) >= 1.0 || fabs(q[1]) >= 1.0 || fabs(q[2]) >= 1.0;",
     "return fabs(q[0]) > 1.0 || fabs(q[1]) > 1.0 || fabs(q[2]) > 1.0;", None),
    ("grad_cB", C, "double cB = scale * 2.0 * rB / D;", "double cB = scale * rB / D;", None),
    ("grad_cJ_sign", C, "c[7] = has_jump ? (s == 1 ? cJ : -cJ) : 0.0;",
     "c[7] = has_jump ? (s == 1 ? -cJ : cJ) : 0.0;", None),
    ("grad_c0", C, "c[0] += cell.A[s][f] * muf[s][f];\n        c[1 + f]",
     "c[0] -= cell.A[s][f] * muf[s][f];\n        c[1 + f]", None),
    ("loss_mean", C, "  free(part);\n  return s / (double)n;\n}\n\n/* The loss and its gradient",
     "  free(part);\n  return s / (double)(n + 1);\n}\n\n/* The loss and its gradient", None),
    ("loss_grad_scale", C, "double scale = 1.0 / (double)n;", "double scale = 2.0 / (double)n;", None),
    ("levels_h", P, "q.h = pr.h / 2.0 ** level", "q.h = pr.h / 2.0 ** (level + 1)", None),
    ("levels_count", P, "for lv in range(levels + 1):\n        L, r2 = loss(",
     "for lv in range(levels):\n        L, r2 = loss(", None),
    ("levels_grad", P, "L, gl = loss_grad(level_problem(pr, lv), theta, pts, n_threads)",
     "L, gl = loss_grad(level_problem(pr, 0), theta, pts, n_threads)", None),
    # Adam and the training loop
    ("adam_c2", C, "double c2 = 1.0 - pow(beta2, (double)t);",
     "double c2 = 1.0 - pow(beta2, (double)(t + 1));", None),
    ("adam_vhat", C, "theta[i] -= lr * mh / (sqrt(vh) + eps);",
     "theta[i] -= lr * mh / (sqrt(v[i]) + eps);", None),
    ("adam_eps", C, "theta[i] -= lr * mh / (sqrt(vh) + eps);", "theta[i] -= lr * mh / sqrt(vh + eps);",
     None),
    ("adam_m", C, "m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];",
     "m[i] = beta1 * m[i] + (1.0 - beta2) * grad[i];", None),
    ("train_step_t", C, "int64_t t = step0 + k + 1;", "int64_t t = step0 + k + 2;", None),
    # grid evaluation, grid rows, CG, node jumps, error metrics
    ("eval_phase", C, "u_out[id] = mlp_forward(pr, theta + s * Pn, x, NULL);",
     "u_out[id] = mlp_forward(pr, theta, x, NULL);", None),
    ("eval_order", C,
     "double x[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};\n    int s = nbo_phase(pr, x);",
     "double x[3] = {-1.0 + k * hg, -1.0 + j * hg, -1.0 + i * hg};\n    int s = nbo_phase(pr, x);",
     None),
    ("grow_jump_sign", C, "if (sp == 1) cp[0] = -jmp; else cp[1] = jmp;",
     "if (sp == 1) cp[0] = jmp; else cp[1] = -jmp;", None),
    ("grow_known_sign", C, "known -= a * (cq[s] - cp[s]);", "known += a * (cq[s] - cp[s]);", None),
    ("grow_beta_sign", C,
     "if (cell.cut && cell.S > 0.0) known += hg * cell.S * nbo_beta(pg, cell.xg);",
     "if (cell.cut && cell.S > 0.0) known -= hg * cell.S * nbo_beta(pg, cell.xg);", None),
    ("grow_dirichlet", C, "known -= wf * nbo_dirichlet_g(pg, q);",
     "known += wf * nbo_dirichlet_g(pg, q);", None),
    ("grow_mu_face", C, "fc[ax] += 0.5 * sg * hg;", "fc[ax] -= 0.5 * sg * hg;", None),
    ("grow_jump_node", C,
     "double jq = Jn ? Jn[node_id(n, nb[0], nb[1], nb[2])] : nbo_alpha(pg, q);",
     "double jq = Jn ? Jn[node_id(n, i, j, k)] : nbo_alpha(pg, q);", None),
    ("cg_beta", C, "double beta = rz_new / rz;", "double beta = rz_new / (rz * 1.1);", None),
    ("cg_precond", C, "    z[r] = rr[r] / rows[r].diag;\n    pp[r] = z[r];",
     "    z[r] = rr[r];\n    pp[r] = z[r];", None),
    ("cg_stop", C, "if (rnorm <= rtol * bnorm) {", "if (rnorm <= 1e3 * rtol * bnorm) {", None),
    ("cg_warm_r0", C, "rr[r] = rows[r].rhs - s;", "rr[r] = rows[r].rhs - 0.0 * s;", None),
    ("cg_bnorm", C, "bnorm2 += rows[r].rhs * rows[r].rhs;", "bnorm2 += rr[r] * rr[r];", None),
    ("nodes_boundary", C, "u_out[id] = nbo_dirichlet_g(pg, q);",
     "u_out[id] = 0.0 * nbo_dirichlet_g(pg, q);", None),
    ("jx_newton", C, "for (int i = 0; i < 3; ++i) xg[i] -= f * gg[i] / q;",
     "for (int i = 0; i < 3; ++i) xg[i] += f * gg[i] / q;", None),
    ("jx_lag_sign", C, "G = beta / mup - (use_lag ? (1.0 - mum / mup) * dn_small : 0.0);",
     "G = beta / mup + (use_lag ? (1.0 - mum / mup) * dn_small : 0.0);", None),
    ("jx_lag_ratio", C, "G = beta / mum + (use_lag ? (1.0 - mup / mum) * dn_small : 0.0);",
     "G = beta / mum + (use_lag ? (1.0 - mum / mup) * dn_small : 0.0);", None),
    ("jx_d_sign", C, "*J = nbo_alpha(pr, xg) + d * G;", "*J = nbo_alpha(pr, xg) - d * G;", None),
    ("jx_band", C, "fabs(ph / gn) > 3.0 * h * (1.0 + 1e-9)", "fabs(ph / gn) > 1.0 * h * (1.0 + 1e-9)",
     None),
    ("jumps_lag_flag", C, "nbo_jump_extrap(pg, x, hg, 1, dn, &J, xg, nrm, &ss);",
     "nbo_jump_extrap(pg, x, hg, 0, dn, &J, xg, nrm, &ss);", None),
    ("fit_side", C, "double xc = xg[i] + (s == 0 ? -hg : hg) * nrm[i];",
     "double xc = xg[i] + (s == 0 ? hg : -hg) * nrm[i];", None),
    ("fit_nearest", C, "c[i] = (int)floor((xc + 1.0) / hg + 0.5 + 1e-6);",
     "c[i] = (int)floor((xc + 1.0) / hg + 1e-6);", None),
    ("fit_phase", C, "if (nbo_phase(pr, xq) != s) continue;", "if (0) continue;", None),
    ("fit_scale", C, "*dn = (cf[1] * nrm[0] + cf[2] * nrm[1] + cf[3] * nrm[2]) / hg;",
     "*dn = (cf[1] * nrm[0] + cf[2] * nrm[1] + cf[3] * nrm[2]);", None),
    ("fit_chol", C, "for (int k = a + 1; k < 4; ++k) t -= L[k][a] * cf[k];",
     "for (int k = a + 1; k < 4; ++k) t -= L[a][k] * cf[k];", None),
    ("gs_warm", C,
     "      status = grid_cg_core(rows, m1, x, rtol, max_iter, nt, &it, &rr);\n"
     "      it_total += it;\n      grid_write_nodes(&pg, n, x, u_out);\n      if (status",
     "      for (int64_t z = 0; z < m; ++z) x[z] = 0.0;\n"
     "      status = grid_cg_core(rows, m1, x, rtol, max_iter, nt, &it, &rr);\n"
     "      it_total += it;\n      grid_write_nodes(&pg, n, x, u_out);\n      if (status", None),
    ("gs_fallback", C,
     "      grid_jumps(&pg, n, NULL, Jn, nt);\n      grid_rows_all(&pg, n, Jn, rows, nt);\n"
     "      status = grid_cg_core",
     "      grid_rows_all(&pg, n, Jn, rows, nt);\n      status = grid_cg_core", None),
    ("gerr_phase", C, "double e = fabs(u[node_id(n, i, j, k)] - nbo_exact_u(pr, s, q));",
     "double e = fabs(u[node_id(n, i, j, k)] - nbo_exact_u(pr, 1, q));", None),
    ("gerr_rms", C, "*rmse = cnt ? sqrt(s2 / cnt) : 0.0;", "*rmse = cnt ? sqrt(s2) / cnt : 0.0;",
     None),
    ("gerr_interior", C,
     "      for (int i = 1; i < n; ++i) {\n"
     "        double q[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};\n"
     "        int s = nbo_phase(pr, q);\n        double e",
     "      for (int i = 0; i <= n; ++i) {\n"
     "        double q[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};\n"
     "        int s = nbo_phase(pr, q);\n        double e", None),
    ("py_grid_error", P, "return a.value, b.value\n", "return b.value, a.value\n", None),
    # argument marshalling of the Python wrappers
    ("py_sample_args", P, "lib().nbo_sample_points(C.byref(pr), seed, step, n, n_band, _dp(pts))",
     "lib().nbo_sample_points(C.byref(pr), step, seed, n, n_band, _dp(pts))", None),
    ("py_terms_D", P, '"D": t.D,', '"D": t.B,', None),
    ("py_adam_t", P, "len(theta), t, lr, beta1,", "len(theta), t + 1, lr, beta1,", None),
    ("py_jump_lag", P, "0 if dn_small is None else 1,", "0,", None),
    ("py_fit_side", P, "_dp(_vec(u)), s, _dp(_vec(xg))", "_dp(_vec(u)), 1 - s, _dp(_vec(xg))", None),
    # degenerate cases
    ("flower_axis", C, "if (rho == 0.0) return;", "if (rho < 0.0) return;", None),
    ("loss_empty", C,
     "  if (n <= 0) return 0.0;\n  int nt = pick_threads(n_threads);\n"
     "  double* part = (double*)calloc(nt, sizeof(double));\n#pragma omp",
     "  int nt = pick_threads(n_threads);\n"
     "  double* part = (double*)calloc(nt, sizeof(double));\n#pragma omp", None),
    ("fit_chol_guard", C, "if (!(t > 1e-8 * M[0][0])) return 1;", "if (!(t > 0.0)) return 1;",
     None),
    ("fit_count", C, "if (cnt < 4) return 1;", "if (cnt < 1) return 1;",
     "fewer than four nodes cannot span an affine basis, so the Cholesky guard refuses them"),
]


def run_one(m, timeout):
    name, rel, old, new, equiv = m
    with tempfile.TemporaryDirectory(prefix=f"nbm_mutant_{name}_") as d:
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
        shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"),
                        ignore=shutil.ignore_patterns("__pycache__"))
        path = os.path.join(d, rel)
        with open(path) as f:
            src = f.read()
        if src.count(old) != 1:
            return name, "pattern", f"{src.count(old)} matches in {rel}", equiv
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        env = dict(os.environ, OMP_NUM_THREADS="2")
        try:
            r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu",
                                "-p", "no:cacheprovider", *PINS], cwd=d, env=env,
                               capture_output=True, text=True, timeout=timeout)
        except subprocess.TimeoutExpired:
            return name, "killed", "timeout", equiv
        lines = r.stdout.strip().splitlines()
        failed = [ln for ln in lines if ln.startswith(("FAILED", "ERROR"))]
        if r.returncode == 0:
            return name, "survived", lines[-1] if lines else "", equiv
        return name, "killed", failed[0] if failed else (lines[-1] if lines else ""), equiv


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("names", nargs="*", help="run only these mutants")
    ap.add_argument("-j", "--jobs", type=int, default=4)
    ap.add_argument("--timeout", type=float, default=900.0)
    args = ap.parse_args()
    chosen = [m for m in MUTANTS if not args.names or m[0] in args.names]
    bad = 0
    counts = {"killed": 0, "equivalent": 0, "survived": 0, "pattern": 0}
    with cf.ThreadPoolExecutor(args.jobs) as ex:
        for name, status, why, equiv in ex.map(lambda m: run_one(m, args.timeout), chosen):
            if status == "survived" and equiv:
                status, why = "equivalent", equiv
            counts[status] += 1
            bad += status in ("survived", "pattern")
            print(f"{name:20s} {status:10s} {why[:100]}", flush=True)
    print(", ".join(f"{k} {v}" for k, v in counts.items()), f"of {len(chosen)} mutants")
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
