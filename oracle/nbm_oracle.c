/*
 * nbm_oracle.c -- plain FP64 CPU oracle of the NBM collocation-residual step.
 *
 * TEST INFRASTRUCTURE ONLY (see nbm_oracle.h).  Written for readability
 * against the paper (arXiv 2210.14907, Sec. 2-3, Fig. 2), not for speed:
 * every network evaluation at every stencil vertex is a separate plain
 * forward pass, and the gradient is plain reverse mode through each one.
 * OpenMP parallelises over collocation points only.
 */
#include "nbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NBO_PI 3.14159265358979323846

/* ======================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies with
 * a Weyl-sequence key schedule.
 * ==================================================================== */
void nbo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* ======================================================================
 * Geometry (Sec. 3: the level set lives on a separate coarse
 * mesh; here it is analytic, or such a mesh).
 * ==================================================================== */
/* Level set stored on a coarse mesh (Sec. 3): the trilinear interpolant of the
 * node values in the mesh cell that contains x (cell index floor((x+1) n/2),
 * clamped to the last cell on the upper faces); g (if not NULL) receives its
 * gradient in that cell. */
static double grid_phi(const nbo_problem* pr, const double x[3], double g[3]) {
  const int n = pr->phi_n;
  const int64_t N1 = n + 1;
  const double sc = 0.5 * n;
  int i[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    double t = (x[a] + 1.0) * sc;
    int c = (int)floor(t);
    if (c < 0) c = 0;
    if (c > n - 1) c = n - 1;
    i[a] = c;
    f[a] = t - c;
  }
  const double* c = pr->phi_grid;
#define NBO_C(di, dj, dk) c[(i[0] + (di)) + N1 * ((i[1] + (dj)) + N1 * (int64_t)(i[2] + (dk)))]
  const double c000 = NBO_C(0, 0, 0), c100 = NBO_C(1, 0, 0), c010 = NBO_C(0, 1, 0),
               c110 = NBO_C(1, 1, 0), c001 = NBO_C(0, 0, 1), c101 = NBO_C(1, 0, 1),
               c011 = NBO_C(0, 1, 1), c111 = NBO_C(1, 1, 1);
#undef NBO_C
  const double c00 = c000 * (1.0 - f[0]) + c100 * f[0], c10 = c010 * (1.0 - f[0]) + c110 * f[0];
  const double c01 = c001 * (1.0 - f[0]) + c101 * f[0], c11 = c011 * (1.0 - f[0]) + c111 * f[0];
  const double c0 = c00 * (1.0 - f[1]) + c10 * f[1], c1 = c01 * (1.0 - f[1]) + c11 * f[1];
  if (g) {
    g[0] = sc * (((c100 - c000) * (1.0 - f[1]) + (c110 - c010) * f[1]) * (1.0 - f[2]) +
                 ((c101 - c001) * (1.0 - f[1]) + (c111 - c011) * f[1]) * f[2]);
    g[1] = sc * ((c10 - c00) * (1.0 - f[2]) + (c11 - c01) * f[2]);
    g[2] = sc * (c1 - c0);
  }
  return c0 * (1.0 - f[2]) + c1 * f[2];
}

/* The level set, Omega- = {phi <= 0}: the sphere |x| = r0 of Sec. 4.1, the
 * flower (that sphere with an angular perturbation amp sin(lt theta) cos(lp psi),
 * the benchmark interface), the no-interface cases, or a mesh level set. */
double nbo_phi(const nbo_problem* pr, const double x[3]) {
  if (pr->geometry == NBO_GEOM_GRID) return grid_phi(pr, x, NULL);
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  switch (pr->geometry) {
    case NBO_GEOM_SPHERE:
      return r - pr->r0;
    case NBO_GEOM_FLOWER: {
      if (r == 0.0) return -pr->r0;
      /* theta: polar angle from +z, written atan2(rho, z) (well conditioned
       * at the poles, same angle as acos(z/r)); psi: azimuth. */
      double theta = atan2(sqrt(x[0] * x[0] + x[1] * x[1]), x[2]);
      double psi = atan2(x[1], x[0]);
      return r - pr->r0 - pr->amp * sin(pr->lobes_theta * theta) * cos(pr->lobes_psi * psi);
    }
    case NBO_GEOM_ALL_PLUS:
      return 1.0;
    case NBO_GEOM_ALL_MINUS:
      return -1.0;
  }
  return 1.0;
}

/* grad phi in closed form; for the flower, the radial part plus the chain
 * rule through the polar angle theta and the azimuth psi. */
void nbo_grad_phi(const nbo_problem* pr, const double x[3], double g[3]) {
  if (pr->geometry == NBO_GEOM_GRID) {
    grid_phi(pr, x, g);
    return;
  }
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  g[0] = g[1] = g[2] = 0.0;
  if (pr->geometry == NBO_GEOM_ALL_PLUS || pr->geometry == NBO_GEOM_ALL_MINUS) return;
  if (r == 0.0) return;
  for (int i = 0; i < 3; ++i) g[i] = x[i] / r; /* grad r */
  if (pr->geometry != NBO_GEOM_FLOWER) return;
  double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
  if (rho == 0.0) return; /* the flower has a conical point on the z axis */
  double theta = atan2(rho, x[2]), psi = atan2(x[1], x[0]);
  double lt = pr->lobes_theta, lp = pr->lobes_psi, a = pr->amp;
  /* d(theta)/dx = z x / (r^2 rho), d/dy = z y / (r^2 rho), d/dz = -rho / r^2 */
  double dth[3] = {x[2] * x[0] / (r * r * rho), x[2] * x[1] / (r * r * rho), -rho / (r * r)};
  /* d(psi)/dx = -y / rho^2, d/dy = x / rho^2 */
  double dps[3] = {-x[1] / (rho * rho), x[0] / (rho * rho), 0.0};
  double dphi_dth = -a * lt * cos(lt * theta) * cos(lp * psi);
  double dphi_dps = a * lp * sin(lt * theta) * sin(lp * psi);
  for (int i = 0; i < 3; ++i) g[i] += dphi_dth * dth[i] + dphi_dps * dps[i];
}

int nbo_phase(const nbo_problem* pr, const double x[3]) {
  /* reading: phi = 0 belongs to Omega- (interior) */
  return nbo_phi(pr, x) <= 0.0 ? 0 : 1;
}

/* Manufactured pairs.
 * Solution 0 (the benchmark configurations), constant mu^s:
 *   u- = exp(x) cos(y) sin(z)   (Laplacian u- = -u-)
 *   u+ = x^2 + y^2 + z^2        (Laplacian u+ = 6)
 * Solution 1 (Sec. 4.1):
 *   u- = exp(z),  u+ = cos(x) sin(y),
 *   mu- = y^2 ln(x + 2) + 4,  mu+ = exp(-z).                             */
double nbo_exact_u(const nbo_problem* pr, int s, const double x[3]) {
  if (pr->solution == 1) {
    if (s == 0) return exp(x[2]);
    return cos(x[0]) * sin(x[1]);
  }
  if (s == 0) return exp(x[0]) * cos(x[1]) * sin(x[2]);
  return x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
}

void nbo_exact_grad_u(const nbo_problem* pr, int s, const double x[3], double g[3]) {
  if (pr->solution == 1) {
    if (s == 0) {
      g[0] = 0.0;
      g[1] = 0.0;
      g[2] = exp(x[2]);
    } else {
      g[0] = -sin(x[0]) * sin(x[1]);
      g[1] = cos(x[0]) * cos(x[1]);
      g[2] = 0.0;
    }
    return;
  }
  if (s == 0) {
    double e = exp(x[0]);
    g[0] = e * cos(x[1]) * sin(x[2]);
    g[1] = -e * sin(x[1]) * sin(x[2]);
    g[2] = e * cos(x[1]) * cos(x[2]);
  } else {
    g[0] = 2.0 * x[0];
    g[1] = 2.0 * x[1];
    g[2] = 2.0 * x[2];
  }
}

static double exact_laplacian(const nbo_problem* pr, int s, const double x[3]) {
  if (pr->solution == 1) {
    if (s == 0) return exp(x[2]);
    return -2.0 * cos(x[0]) * sin(x[1]);
  }
  if (s == 0) return -nbo_exact_u(pr, 0, x);
  return 6.0;
}

double nbo_mu(const nbo_problem* pr, int s, const double x[3]) {
  if (pr->solution == 1) {
    if (s == 0) return x[1] * x[1] * log(x[0] + 2.0) + 4.0;
    return exp(-x[2]);
  }
  return s == 0 ? pr->mu_minus : pr->mu_plus;
}

static void mu_grad(const nbo_problem* pr, int s, const double x[3], double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  if (pr->solution != 1) return;
  if (s == 0) {
    g[0] = x[1] * x[1] / (x[0] + 2.0);
    g[1] = 2.0 * x[1] * log(x[0] + 2.0);
  } else {
    g[2] = -exp(-x[2]);
  }
}

/* f^s = k^s u^s - div(mu^s grad u^s) = k^s u^s - mu^s Lap(u^s) - grad(mu^s).grad(u^s)
 * (Sec. 2 with k^s constant). */
double nbo_rhs_f(const nbo_problem* pr, int s, const double x[3]) {
  double k = s == 0 ? pr->k_minus : pr->k_plus;
  double gu[3], gm[3];
  nbo_exact_grad_u(pr, s, x, gu);
  mu_grad(pr, s, x, gm);
  return k * nbo_exact_u(pr, s, x) - nbo_mu(pr, s, x) * exact_laplacian(pr, s, x) -
         (gm[0] * gu[0] + gm[1] * gu[1] + gm[2] * gu[2]);
}

/* [u] = u+ - u- (reading: jumps are plus side minus minus side). */
double nbo_alpha(const nbo_problem* pr, const double x[3]) {
  return nbo_exact_u(pr, 1, x) - nbo_exact_u(pr, 0, x);
}

/* [mu d_n u] = mu+ grad u+ . n - mu- grad u- . n, n = grad phi / |grad phi|
 * pointing from Omega- into Omega+. */
double nbo_beta(const nbo_problem* pr, const double x[3]) {
  double gp[3], gm[3], gphi[3];
  nbo_exact_grad_u(pr, 1, x, gp);
  nbo_exact_grad_u(pr, 0, x, gm);
  nbo_grad_phi(pr, x, gphi);
  double nn = sqrt(gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2]);
  if (nn == 0.0) return 0.0;
  double b = 0.0;
  const double mp = nbo_mu(pr, 1, x), mm = nbo_mu(pr, 0, x);
  for (int i = 0; i < 3; ++i) b += (mp * gp[i] - mm * gm[i]) * gphi[i] / nn;
  return b;
}

/* Dirichlet data on the cube boundary: the outer solution (Sec. 2). */
double nbo_dirichlet_g(const nbo_problem* pr, const double x[3]) {
  int s = (pr->geometry == NBO_GEOM_ALL_MINUS) ? 0 : 1;
  return nbo_exact_u(pr, s, x);
}

/* ======================================================================
 * Implicit compute cell C_p = p + [-h/2, h/2]^3 (Fig. 2: an implicit
 * cell at each point, cut by the interface).  Reading: phi is taken
 * linear on each tetrahedron of the Freudenthal-Kuhn six-tetrahedron split
 * of the cube, so every fraction has a closed form.
 * ==================================================================== */

/* Fraction of a triangle where the linear interpolant of (f0,f1,f2) is <= 0. */
double nbo_tri_fraction(double f0, double f1, double f2) {
  double f[3] = {f0, f1, f2};
  int neg[3], nn = 0;
  for (int i = 0; i < 3; ++i) {
    neg[i] = f[i] <= 0.0;
    nn += neg[i];
  }
  if (nn == 0) return 0.0;
  if (nn == 3) return 1.0;
  if (nn == 1) {
    int a = neg[0] ? 0 : (neg[1] ? 1 : 2);
    int b = (a + 1) % 3, c = (a + 2) % 3;
    /* corner triangle cut at t_b = fa/(fa-fb), t_c = fa/(fa-fc) */
    return (f[a] / (f[a] - f[b])) * (f[a] / (f[a] - f[c]));
  }
  int c = !neg[0] ? 0 : (!neg[1] ? 1 : 2);
  int a = (c + 1) % 3, b = (c + 2) % 3;
  return 1.0 - (f[c] / (f[c] - f[a])) * (f[c] / (f[c] - f[b]));
}

/* Fraction of a tetrahedron where the linear interpolant is <= 0. */
double nbo_tet_fraction(double f0, double f1, double f2, double f3) {
  double f[4] = {f0, f1, f2, f3};
  int neg[4], nn = 0;
  for (int i = 0; i < 4; ++i) {
    neg[i] = f[i] <= 0.0;
    nn += neg[i];
  }
  if (nn == 0) return 0.0;
  if (nn == 4) return 1.0;
  if (nn == 1 || nn == 3) {
    int lone = -1;
    for (int i = 0; i < 4; ++i)
      if (neg[i] == (nn == 1)) lone = i;
    double prod = 1.0;
    for (int i = 0; i < 4; ++i)
      if (i != lone) prod *= f[lone] / (f[lone] - f[i]);
    return nn == 1 ? prod : 1.0 - prod;
  }
  /* two below, two above: closed form of the divided difference of
   * (-s)_+^3 over the four values, written without cancellation.        */
  double A = 0, B = 0, C = 0, Dd = 0;
  int gotn = 0, gotp = 0;
  for (int i = 0; i < 4; ++i) {
    if (neg[i]) {
      if (gotn++ == 0) A = -f[i]; else B = -f[i];
    } else {
      if (gotp++ == 0) C = f[i]; else Dd = f[i];
    }
  }
  double num = C * Dd * (A * A + A * B + B * B) + (C + Dd) * A * B * (A + B) + A * A * B * B;
  double den = (C + A) * (Dd + A) * (C + B) * (Dd + B);
  return num / den;
}

static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* crossing point of the zero level on edge u(neg) -> v(pos) */
static void edge_cross(const double xu[3], double fu, const double xv[3], double fv, double out[3]) {
  double t = fu / (fu - fv);
  for (int i = 0; i < 3; ++i) out[i] = xu[i] + t * (xv[i] - xu[i]);
}

static void tri_area_centroid(const double a[3], const double b[3], const double c[3],
                              double* area, double cen[3]) {
  double e1[3], e2[3], cr[3];
  for (int i = 0; i < 3; ++i) {
    e1[i] = b[i] - a[i];
    e2[i] = c[i] - a[i];
  }
  cross3(e1, e2, cr);
  *area = 0.5 * norm3(cr);
  for (int i = 0; i < 3; ++i) cen[i] = (a[i] + b[i] + c[i]) / 3.0;
}

/* interface polygon of one tetrahedron: area and area-weighted centroid sum */
static void tet_interface(const double X[4][3], const double f[4], double* area, double wc[3]) {
  int neg[4], nn = 0;
  for (int i = 0; i < 4; ++i) {
    neg[i] = f[i] <= 0.0;
    nn += neg[i];
  }
  *area = 0.0;
  wc[0] = wc[1] = wc[2] = 0.0;
  if (nn == 0 || nn == 4) return;
  if (nn == 1 || nn == 3) {
    int lone = -1;
    for (int i = 0; i < 4; ++i)
      if (neg[i] == (nn == 1)) lone = i;
    double P[3][3];
    int k = 0;
    for (int i = 0; i < 4; ++i) {
      if (i == lone) continue;
      if (neg[lone]) edge_cross(X[lone], f[lone], X[i], f[i], P[k]);
      else edge_cross(X[i], f[i], X[lone], f[lone], P[k]);
      ++k;
    }
    double cen[3];
    tri_area_centroid(P[0], P[1], P[2], area, cen);
    for (int i = 0; i < 3; ++i) wc[i] = *area * cen[i];
    return;
  }
  int a = -1, b = -1, c = -1, d = -1;
  for (int i = 0; i < 4; ++i) {
    if (neg[i]) { if (a < 0) a = i; else b = i; }
    else { if (c < 0) c = i; else d = i; }
  }
  /* cyclic order of the quadrilateral: ac, ad, bd, bc */
  double Q[4][3];
  edge_cross(X[a], f[a], X[c], f[c], Q[0]);
  edge_cross(X[a], f[a], X[d], f[d], Q[1]);
  edge_cross(X[b], f[b], X[d], f[d], Q[2]);
  edge_cross(X[b], f[b], X[c], f[c], Q[3]);
  double a1, a2, c1[3], c2[3];
  tri_area_centroid(Q[0], Q[1], Q[2], &a1, c1);
  tri_area_centroid(Q[0], Q[2], Q[3], &a2, c2);
  *area = a1 + a2;
  for (int i = 0; i < 3; ++i) wc[i] = a1 * c1[i] + a2 * c2[i];
}

/* Geometry of the cell p + [-h/2, h/2]^3 (Fig. 2): volume fractions V^s, face
 * fractions A^s_f, interface area fraction S and interface point x_G. */
void nbo_cell_geometry(const nbo_problem* pr, const double p[3], double h, nbo_cell* out) {
  memset(out, 0, sizeof(*out));
  /* corner c has offsets ((c&1), (c>>1)&1, (c>>2)&1) - 1/2, times h */
  double X[8][3], F[8];
  int nneg = 0;
  for (int c = 0; c < 8; ++c) {
    for (int i = 0; i < 3; ++i) X[c][i] = p[i] + h * ((double)((c >> i) & 1) - 0.5);
    F[c] = nbo_phi(pr, X[c]);
    nneg += F[c] <= 0.0;
  }
  if (nneg == 0 || nneg == 8) {
    int s = nneg == 0 ? 1 : 0;
    out->cut = 0;
    out->phase = s;
    out->V[s] = 1.0;
    for (int f = 0; f < 6; ++f) out->A[s][f] = 1.0;
    out->S = 0.0;
    for (int i = 0; i < 3; ++i) out->centroid[i] = out->xg[i] = p[i];
    return;
  }
  out->cut = 1;
  out->phase = nbo_phase(pr, p);
  /* six tetrahedra 0 -> e_a -> e_a+e_b -> 7 for every permutation (a,b,c) */
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  double vneg = 0.0, area = 0.0, wc[3] = {0, 0, 0};
  for (int t = 0; t < 6; ++t) {
    int v1 = 1 << perms[t][0];
    int v2 = v1 | (1 << perms[t][1]);
    int idx[4] = {0, v1, v2, 7};
    double Xt[4][3], ft[4];
    for (int k = 0; k < 4; ++k) {
      for (int i = 0; i < 3; ++i) Xt[k][i] = X[idx[k]][i];
      ft[k] = F[idx[k]];
    }
    vneg += nbo_tet_fraction(ft[0], ft[1], ft[2], ft[3]) / 6.0;
    double ta, tw[3];
    tet_interface((const double(*)[3])Xt, ft, &ta, tw);
    area += ta;
    for (int i = 0; i < 3; ++i) wc[i] += tw[i];
  }
  out->V[0] = vneg;
  out->V[1] = 1.0 - vneg;
  /* faces: axis i, side sd; split along the diagonal from the face's
   * lowest to its highest corner (the split the tetrahedra induce). */
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3, k = (i + 2) % 3;
    for (int sd = 0; sd < 2; ++sd) {
      int base = sd << i;
      int c00 = base, c10 = base | (1 << j), c01 = base | (1 << k), c11 = base | (1 << j) | (1 << k);
      double fr = 0.5 * (nbo_tri_fraction(F[c00], F[c10], F[c11]) +
                         nbo_tri_fraction(F[c00], F[c01], F[c11]));
      out->A[0][2 * i + sd] = fr;
      out->A[1][2 * i + sd] = 1.0 - fr;
    }
  }
  out->S = area / (h * h);
  if (area > 0.0) {
    double x[3];
    for (int i = 0; i < 3; ++i) x[i] = out->centroid[i] = wc[i] / area;
    /* project onto phi = 0: at most three Newton steps along grad phi */
    for (int it = 0; it < 3; ++it) {
      double g[3];
      double ph = nbo_phi(pr, x);
      nbo_grad_phi(pr, x, g);
      double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
      if (gg <= 1e-300) break;
      for (int i = 0; i < 3; ++i) x[i] -= ph * g[i] / gg;
    }
    for (int i = 0; i < 3; ++i) out->xg[i] = x[i];
  } else {
    for (int i = 0; i < 3; ++i) out->centroid[i] = out->xg[i] = p[i];
  }
}

/* ======================================================================
 * Networks (Sec. 3: one network for the
 * solution on each side of the interface): a_0 = x, z_l = W_l a_{l-1} + b_l,
 * a_l = act(z_l) for the hidden layers (tanh, or sin for the sine-activated
 * networks of Sec. 4.1), u = w . a_L + b.
 * Layout per net: W1[H][3], b1[H], then (W_l[H][H], b_l[H]) for
 * l = 2..n_hidden, then w[H], b.  Net minus first, then net plus.
 * ==================================================================== */
int64_t nbo_params_per_net(const nbo_problem* pr) {
  int64_t H = pr->width;
  return 4 * H + (int64_t)(pr->n_hidden - 1) * (H * H + H) + H + 1;
}

/* activation and its derivative at z */
static double act_fn(const nbo_problem* pr, double z, double* dz) {
  if (pr->activation == 1) {
    *dz = cos(z);
    return sin(z);
  }
  double t = tanh(z);
  *dz = 1.0 - t * t;
  return t;
}

/* forward; acts (if given, 2 n_hidden H values) receives the hidden
 * activations act(z_l) followed by their derivatives act'(z_l) */
static double mlp_forward(const nbo_problem* pr, const double* th, const double x[3], double* acts) {
  int H = pr->width, L = pr->n_hidden;
  double* a = acts;
  double buf[2][512], dbuf[512];
  double* cur = buf[0];
  const double* W = th;
  const double* b = th + 3 * H;
  for (int n = 0; n < H; ++n) {
    double z = b[n];
    for (int j = 0; j < 3; ++j) z += W[3 * n + j] * x[j];
    cur[n] = act_fn(pr, z, &dbuf[n]);
  }
  if (a) {
    memcpy(a, cur, sizeof(double) * H);
    memcpy(a + (int64_t)L * H, dbuf, sizeof(double) * H);
  }
  const double* q = th + 4 * H;
  for (int l = 1; l < L; ++l) {
    double* nxt = buf[l & 1];
    const double* Wl = q;
    const double* bl = q + (int64_t)H * H;
    for (int n = 0; n < H; ++n) {
      double z = bl[n];
      for (int k = 0; k < H; ++k) z += Wl[(int64_t)n * H + k] * cur[k];
      nxt[n] = act_fn(pr, z, &dbuf[n]);
    }
    cur = nxt;
    if (a) {
      memcpy(a + (int64_t)l * H, cur, sizeof(double) * H);
      memcpy(a + (int64_t)(L + l) * H, dbuf, sizeof(double) * H);
    }
    q += (int64_t)H * H + H;
  }
  double u = q[H];
  for (int n = 0; n < H; ++n) u += q[n] * cur[n];
  return u;
}

/* one network's output at x (parameter layout as above) */
double nbo_mlp_eval(const nbo_problem* pr, const double* theta_net, const double x[3]) {
  return mlp_forward(pr, theta_net, x, NULL);
}

/* reverse mode of one evaluation: grad += c * du/dtheta */
static void mlp_backward(const nbo_problem* pr, const double* th, const double x[3], double c,
                         const double* acts, double* grad) {
  int H = pr->width, L = pr->n_hidden;
  double g[512], gz[512];
  /* offsets of each layer */
  int64_t off_out = 4 * H + (int64_t)(L - 1) * (H * H + H);
  const double* w = th + off_out;
  const double* aL = acts + (int64_t)(L - 1) * H;
  for (int n = 0; n < H; ++n) {
    grad[off_out + n] += c * aL[n];
    g[n] = c * w[n];
  }
  grad[off_out + H] += c;
  for (int l = L - 1; l >= 1; --l) {
    /* layer l+1 in 1-based numbering: input acts[l-1], output acts[l] */
    int64_t off = 4 * H + (int64_t)(l - 1) * (H * H + H);
    const double* Wl = th + off;
    const double* dout = acts + (int64_t)(L + l) * H;  /* act'(z) of layer l+1 */
    const double* ain = acts + (int64_t)(l - 1) * H;
    for (int n = 0; n < H; ++n) gz[n] = g[n] * dout[n];
    for (int n = 0; n < H; ++n) {
      for (int k = 0; k < H; ++k) grad[off + (int64_t)n * H + k] += gz[n] * ain[k];
      grad[off + (int64_t)H * H + n] += gz[n];
    }
    for (int k = 0; k < H; ++k) {
      double s = 0.0;
      for (int n = 0; n < H; ++n) s += Wl[(int64_t)n * H + k] * gz[n];
      g[k] = s;
    }
  }
  const double* d1 = acts + (int64_t)L * H;
  for (int n = 0; n < H; ++n) {
    double gz1 = g[n] * d1[n];
    for (int j = 0; j < 3; ++j) grad[3 * n + j] += gz1 * x[j];
    grad[3 * H + n] += gz1;
  }
}

/* ======================================================================
 * Collocation points (random points, Sec. 3).  Uniform points
 * lie on the lattice -1 + k 2^-22, k in [1, 2^23-1], so p +- h is exact for
 * power-of-two h.  Band points (|phi| < 4h) are placed along rays from the
 * origin at a uniform offset t in (-4h, 4h) from the interface radius.
 * Counter of point i at step t: {i, t_lo, t_hi, 0x4E424D31}; key = seed.
 * ==================================================================== */
static double quantize_coord(double v) {
  double k = floor((v + 1.0) * 4194304.0 + 0.5);
  if (k < 1.0) k = 1.0;
  if (k > 8388607.0) k = 8388607.0;
  return -1.0 + k / 4194304.0;
}

void nbo_sample_points(const nbo_problem* pr, uint64_t seed, int64_t step, int64_t n,
                       int64_t n_band, double* pts) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int has_iface = pr->geometry == NBO_GEOM_SPHERE || pr->geometry == NBO_GEOM_FLOWER;
  int64_t n_uniform = n - n_band;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0x4E424D31u};
    uint32_t r[4];
    nbo_philox4x32_10(ctr, key, r);
    double* x = pts + 3 * i;
    if (i < n_uniform || !has_iface) {
      for (int j = 0; j < 3; ++j) {
        uint64_t k = 1 + (((uint64_t)r[j] * 8388607ull) >> 32);
        x[j] = -1.0 + (double)k / 4194304.0;
      }
    } else {
      double u[3];
      for (int j = 0; j < 3; ++j) u[j] = ((double)(r[j] >> 8) + 0.5) / 16777216.0;
      double cth = 1.0 - 2.0 * u[0];
      double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
      double psi = 2.0 * NBO_PI * u[1];
      double t = (2.0 * u[2] - 1.0) * 4.0 * pr->h;
      double R = pr->r0;
      if (pr->geometry == NBO_GEOM_FLOWER)
        R += pr->amp * sin(pr->lobes_theta * acos(cth)) * cos(pr->lobes_psi * psi);
      double dir[3] = {sth * cos(psi), sth * sin(psi), cth};
      for (int j = 0; j < 3; ++j) x[j] = quantize_coord((R + t) * dir[j]);
    }
  }
}

/* ======================================================================
 * Point residual (Sec. 3 and Fig. 2; the equation itself is missing from
 * the text, so this is the reading).  Integrating the PDE over both parts
 * of the cell and using the flux-jump condition on the interface gives,
 * after division by h,
 *   B = h^2 sum_s V^s (k^s U^s(p) - f^s(p))
 *       - sum_faces sum_s A^s_f mu^s_f (U^s(p + sigma h e_i) - U^s(p))
 *       + h S beta(x_G)
 * with U^s(q) = g(q) whenever q leaves the cube (Dirichlet data) and
 * mu^s_f = mu^s at the face centre p + sigma (h/2) e_i (constant for the
 * benchmark pair).
 * Jacobi preconditioner M = diag(A):  D = sum_f sum_s A^s_f mu^s_f + h^2 sum_s V^s k^s.
 * Value jump (cut cells with S > 0):  J = U+(x_G) - U-(x_G) - alpha(x_G).
 * r_p^2 = (B/D)^2 + lambda J^2.
 * ==================================================================== */
static double k_of(const nbo_problem* pr, int s) { return s == 0 ? pr->k_minus : pr->k_plus; }

static int outside_box(const double q[3]) {
  return fabs(q[0]) >= 1.0 || fabs(q[1]) >= 1.0 || fabs(q[2]) >= 1.0;
}

/* One point: all evaluations, the rows, and (if grad != NULL) the gradient
 * of (scale * r^2) accumulated into grad.  mode 1 substitutes exact u^s. */
static void point_core(const nbo_problem* pr, const double* theta, const double p[3], int mode,
                       double scale, double* grad, nbo_point_terms* out) {
  const double h = pr->h;
  int64_t Pn = nbo_params_per_net(pr);
  nbo_cell cell;
  nbo_cell_geometry(pr, p, h, &cell);
  int L = pr->n_hidden, H = pr->width;
  /* U[s][0] at p, U[s][1+f] at the neighbour across face f, U[s][7] at x_G */
  double U[2][8];
  int inside[6];
  double Q[8][3];
  for (int i = 0; i < 3; ++i) Q[0][i] = p[i];
  for (int f = 0; f < 6; ++f) {
    int ax = f / 2;
    double sg = (f & 1) ? 1.0 : -1.0;
    for (int i = 0; i < 3; ++i) Q[1 + f][i] = p[i] + (i == ax ? sg * h : 0.0);
    inside[f] = !outside_box(Q[1 + f]);
  }
  for (int i = 0; i < 3; ++i) Q[7][i] = cell.xg[i];
  int has_jump = cell.cut && cell.S > 0.0;
  int used[2];
  double* acts = NULL;
  if (grad) acts = (double*)malloc(sizeof(double) * 2 * 8 * 2 * L * H);
  for (int s = 0; s < 2; ++s) {
    double any = cell.V[s];
    for (int f = 0; f < 6; ++f) any += cell.A[s][f];
    used[s] = any > 0.0 || has_jump;
    for (int e = 0; e < 8; ++e) {
      U[s][e] = 0.0;
      if (!used[s]) continue;
      if (e == 7 && !has_jump) continue;
      if (e >= 1 && e <= 6 && !inside[e - 1]) {
        U[s][e] = nbo_dirichlet_g(pr, Q[e]);
        continue;
      }
      if (mode == 1) {
        U[s][e] = nbo_exact_u(pr, s, Q[e]);
      } else {
        const double* th = theta + s * Pn;
        U[s][e] = mlp_forward(pr, th, Q[e], acts ? acts + ((int64_t)s * 8 + e) * 2 * L * H : NULL);
      }
    }
  }
  /* mu^s at the six face centres p + sigma (h/2) e_i */
  double muf[2][6];
  for (int f = 0; f < 6; ++f) {
    double c[3] = {p[0], p[1], p[2]};
    c[f / 2] += (f & 1) ? 0.5 * h : -0.5 * h;
    for (int s = 0; s < 2; ++s) muf[s][f] = nbo_mu(pr, s, c);
  }
  double B = 0.0, D = 0.0;
  for (int s = 0; s < 2; ++s) {
    double k = k_of(pr, s);
    B += h * h * cell.V[s] * (k * U[s][0] - nbo_rhs_f(pr, s, p));
    D += h * h * cell.V[s] * k;
    for (int f = 0; f < 6; ++f) {
      B -= cell.A[s][f] * muf[s][f] * (U[s][1 + f] - U[s][0]);
      D += cell.A[s][f] * muf[s][f];
    }
  }
  if (has_jump) B += h * cell.S * nbo_beta(pr, cell.xg);
  double J = 0.0;
  if (has_jump) J = U[1][7] - U[0][7] - nbo_alpha(pr, cell.xg);
  double rB = B / D;
  double r2 = rB * rB + pr->lambda_jump * J * J;
  if (out) {
    out->B = B;
    out->D = D;
    out->J = J;
    out->r2 = r2;
    out->has_jump = has_jump;
    out->cut = cell.cut;
  }
  if (grad && mode == 0) {
    /* d(scale r^2)/dU for each evaluation, then reverse mode through it */
    double cB = scale * 2.0 * rB / D;
    double cJ = scale * 2.0 * pr->lambda_jump * J;
    for (int s = 0; s < 2; ++s) {
      if (!used[s]) continue;
      double k = k_of(pr, s);
      double c[8] = {0};
      c[0] = h * h * cell.V[s] * k;
      for (int f = 0; f < 6; ++f) {
        c[0] += cell.A[s][f] * muf[s][f];
        c[1 + f] = -cell.A[s][f] * muf[s][f];
      }
      for (int e = 0; e < 7; ++e) c[e] *= cB;
      c[7] = has_jump ? (s == 1 ? cJ : -cJ) : 0.0;
      for (int e = 0; e < 8; ++e) {
        if (c[e] == 0.0) continue;
        if (e >= 1 && e <= 6 && !inside[e - 1]) continue;
        if (e == 7 && !has_jump) continue;
        mlp_backward(pr, theta + s * Pn, Q[e], c[e], acts + ((int64_t)s * 8 + e) * 2 * L * H,
                     grad + s * Pn);
      }
    }
  }
  free(acts);
}

/* B, D, J and r_p^2 of one point (Sec. 3), without the gradient */
void nbo_point_terms_eval(const nbo_problem* pr, const double* theta, const double p[3], int mode,
                          nbo_point_terms* out) {
  point_core(pr, theta, p, mode, 0.0, NULL, out);
}

static int pick_threads(int n_threads) {
#ifdef _OPENMP
  return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
  (void)n_threads;
  return 1;
#endif
}

int nbo_default_threads(void) { return pick_threads(0); }

/* The loss: the mean of r_p^2 over the points (Sec. 3 aggregates the point
 * residuals into one loss; the mean of squares is the reading taken).
 * r2_out (if not NULL) receives every r_p^2. */
double nbo_loss(const nbo_problem* pr, const double* theta, const double* pts, int64_t n,
                double* r2_out, int n_threads) {
  if (n <= 0) return 0.0;
  int nt = pick_threads(n_threads);
  double* part = (double*)calloc(nt, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double acc = 0.0;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      nbo_point_terms t;
      point_core(pr, theta, pts + 3 * i, 0, 0.0, NULL, &t);
      if (r2_out) r2_out[i] = t.r2;
      acc += t.r2;
    }
    part[tid] = acc;
  }
  double s = 0.0;
  for (int t = 0; t < nt; ++t) s += part[t];
  free(part);
  return s / (double)n;
}

/* The loss and its gradient with respect to both networks' parameters, by
 * the reverse mode of point_core (Sec. 3: the gradient passes through the
 * NBM kernels). */
double nbo_loss_grad(const nbo_problem* pr, const double* theta, const double* pts, int64_t n,
                     double* grad, int n_threads) {
  int64_t P = 2 * nbo_params_per_net(pr);
  memset(grad, 0, sizeof(double) * P);
  if (n <= 0) return 0.0;
  int nt = pick_threads(n_threads);
  double* part = (double*)calloc(nt, sizeof(double));
  double* gpart = (double*)calloc((size_t)nt * P, sizeof(double));
  double scale = 1.0 / (double)n;
#pragma omp parallel num_threads(nt)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double acc = 0.0;
    double* g = gpart + (size_t)tid * P;
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      nbo_point_terms t;
      point_core(pr, theta, pts + 3 * i, 0, scale, g, &t);
      acc += t.r2;
    }
    part[tid] = acc;
  }
  double s = 0.0;
  for (int t = 0; t < nt; ++t) {
    s += part[t];
    for (int64_t j = 0; j < P; ++j) grad[j] += gpart[(size_t)t * P + j];
  }
  free(part);
  free(gpart);
  return s / (double)n;
}

/* Adam (Kingma & Ba 2015), bias-corrected, step t >= 1, no weight decay. */
void nbo_adam_step(double* theta, double* m, double* v, const double* grad, int64_t n, int64_t t,
                   double lr, double beta1, double beta2, double eps) {
  double c1 = 1.0 - pow(beta1, (double)t);
  double c2 = 1.0 - pow(beta2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    theta[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* n_steps training steps (Sec. 3): step t = step0 + k + 1 samples its batch
 * at Philox counter t, takes the loss gradient there and applies Adam with
 * the bias correction of step t. */
void nbo_train(const nbo_problem* pr, double* theta, double* m, double* v, int64_t step0,
               int n_steps, int64_t batch, int64_t n_band, double lr, double beta1, double beta2,
               double eps, uint64_t seed, double* loss_hist, int n_threads) {
  int64_t P = 2 * nbo_params_per_net(pr);
  double* pts = (double*)malloc(sizeof(double) * 3 * batch);
  double* g = (double*)malloc(sizeof(double) * P);
  for (int k = 0; k < n_steps; ++k) {
    int64_t t = step0 + k + 1;
    nbo_sample_points(pr, seed, t, batch, n_band, pts);
    double L = nbo_loss_grad(pr, theta, pts, batch, g, n_threads);
    if (loss_hist) loss_hist[k] = L;
    nbo_adam_step(theta, m, v, g, P, t, lr, beta1, beta2, eps);
  }
  free(pts);
  free(g);
}

/* ======================================================================
 * Grid evaluation and the grid scheme (the plain mesh-based method that
 * NBM lifts off the grid, Sec. 1 and Sec. 3).  Nodes -1 + i h_g,
 * i = 0..n, h_g = 2/n; node (i,j,k) at index i + (n+1)(j + (n+1)k).
 * ==================================================================== */
static int64_t node_id(int n, int i, int j, int k) {
  return (int64_t)i + (int64_t)(n + 1) * ((int64_t)j + (int64_t)(n + 1) * k);
}

/* The trained pair on the (n+1)^3 nodes, each node with the network of its
 * phase (the use of a trained model in Fig. 1); node (i,j,k) at
 * i + (n+1)(j + (n+1)k). */
void nbo_eval_grid(const nbo_problem* pr, const double* theta, int n, double* u_out, int n_threads) {
  int64_t Pn = nbo_params_per_net(pr);
  double hg = 2.0 / n;
  int nt = pick_threads(n_threads);
  int64_t total = (int64_t)(n + 1) * (n + 1) * (n + 1);
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t id = 0; id < total; ++id) {
    int i = (int)(id % (n + 1)), j = (int)((id / (n + 1)) % (n + 1)), k = (int)(id / ((int64_t)(n + 1) * (n + 1)));
    double x[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};
    int s = nbo_phase(pr, x);
    u_out[id] = mlp_forward(pr, theta + s * Pn, x, NULL);
  }
}

/* Grid rows: the same balance row B_p at every interior node, with one
 * unknown u_q per node.  A net-s value at a node of the other phase is
 * u_q +- J(q), J(q) the value jump u+ - u- carried to the node: with Jn ==
 * NULL the manufactured pair's own u+(q) - u-(q) (the "exact jump"
 * extension), else Jn[node] (the extrapolated jump below).  Every jump term
 * moves to the RHS and A stays symmetric: A_pp = D_p, A_pq = -w_f,
 * w_f = sum_s A^s_f mu^s. */
typedef struct {
  double diag;
  double w[6];
  double rhs;
} grid_row;

static void grid_row_build(const nbo_problem* pg, int n, int i, int j, int k, const double* Jn,
                           grid_row* row) {
  double hg = pg->h;
  int idx[3] = {i, j, k};
  double p[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};
  nbo_cell cell;
  nbo_cell_geometry(pg, p, hg, &cell);
  int sp = nbo_phase(pg, p);
  /* c^s(q): correction so that U^s(q) = u_q + c^s(q) */
  double cp[2] = {0, 0};
  {
    double jmp = Jn ? Jn[node_id(n, i, j, k)] : nbo_alpha(pg, p);
    if (sp == 1) cp[0] = -jmp; else cp[1] = jmp;
  }
  row->diag = 0.0;
  row->rhs = 0.0;
  double known = 0.0; /* terms of B that do not involve the unknowns */
  for (int s = 0; s < 2; ++s) {
    double k_s = k_of(pg, s);
    row->diag += hg * hg * cell.V[s] * k_s;
    known += hg * hg * cell.V[s] * (k_s * cp[s] - nbo_rhs_f(pg, s, p));
  }
  for (int f = 0; f < 6; ++f) {
    int ax = f / 2, sg = (f & 1) ? 1 : -1;
    int nb[3] = {idx[0], idx[1], idx[2]};
    nb[ax] += sg;
    double q[3] = {-1.0 + nb[0] * hg, -1.0 + nb[1] * hg, -1.0 + nb[2] * hg};
    int bnd = nb[ax] == 0 || nb[ax] == n;
    int sq = nbo_phase(pg, q);
    double cq[2] = {0, 0};
    if (!bnd) {
      /* boundary neighbours carry g(q) for both networks, as in B_p */
      double jq = Jn ? Jn[node_id(n, nb[0], nb[1], nb[2])] : nbo_alpha(pg, q);
      if (sq == 1) cq[0] = -jq; else cq[1] = jq;
    }
    double fc[3] = {p[0], p[1], p[2]};  /* face centre, shared with the neighbour's row */
    fc[ax] += 0.5 * sg * hg;
    double wf = 0.0;
    for (int s = 0; s < 2; ++s) {
      double a = cell.A[s][f] * nbo_mu(pg, s, fc);
      wf += a;
      known -= a * (cq[s] - cp[s]);
    }
    row->diag += wf;
    if (bnd) {
      /* Dirichlet node: its value g(q) is known */
      known -= wf * nbo_dirichlet_g(pg, q);
      row->w[f] = 0.0;
    } else {
      row->w[f] = wf;
    }
  }
  if (cell.cut && cell.S > 0.0) known += hg * cell.S * nbo_beta(pg, cell.xg);
  /* B = diag u_p - sum w_f u_q + known = 0  ->  A u = -known */
  row->rhs = -known;
}

/* the grid system as a dense matrix (small n only), exact node jump */
int nbo_grid_assemble_dense(const nbo_problem* pr, int n, double* A, double* b) {
  nbo_problem pg = *pr;
  pg.h = 2.0 / n;
  int m1 = n - 1;
  int64_t m = (int64_t)m1 * m1 * m1;
  memset(A, 0, sizeof(double) * m * m);
  for (int k = 1; k < n; ++k)
    for (int j = 1; j < n; ++j)
      for (int i = 1; i < n; ++i) {
        grid_row row;
        grid_row_build(&pg, n, i, j, k, NULL, &row);
        int64_t r = (i - 1) + (int64_t)m1 * ((j - 1) + (int64_t)m1 * (k - 1));
        A[r * m + r] = row.diag;
        b[r] = row.rhs;
        for (int f = 0; f < 6; ++f) {
          if (row.w[f] == 0.0) continue;
          int ax = f / 2, sg = (f & 1) ? 1 : -1;
          int nb[3] = {i, j, k};
          nb[ax] += sg;
          int64_t c = (nb[0] - 1) + (int64_t)m1 * ((nb[1] - 1) + (int64_t)m1 * (nb[2] - 1));
          A[r * m + c] -= row.w[f];
        }
      }
  return 0;
}

/* Jacobi-preconditioned conjugate gradients on the interior nodes from the
 * start vector x (warm start); stops at ||b - A x|| <= rtol ||b|| with the
 * recursively updated residual.  Returns 0 on convergence, 1 otherwise. */
static int grid_cg_core(const grid_row* rows, int m1, double* x, double rtol, int max_iter,
                        int nt, int* iters_out, double* relres_out) {
  int64_t m = (int64_t)m1 * m1 * m1;
  int64_t strides[3] = {1, m1, (int64_t)m1 * m1};
  double* rr = (double*)malloc(sizeof(double) * m);
  double* z = (double*)malloc(sizeof(double) * m);
  double* pp = (double*)malloc(sizeof(double) * m);
  double* Ap = (double*)malloc(sizeof(double) * m);
  double bnorm2 = 0.0;
  for (int64_t r = 0; r < m; ++r) {
    double s = rows[r].diag * x[r];
    for (int f = 0; f < 6; ++f)
      if (rows[r].w[f] != 0.0) s -= rows[r].w[f] * x[r + ((f & 1) ? 1 : -1) * strides[f / 2]];
    rr[r] = rows[r].rhs - s;
    bnorm2 += rows[r].rhs * rows[r].rhs;
  }
  double bnorm = sqrt(bnorm2);
  double rz = 0.0, rn2 = 0.0;
  for (int64_t r = 0; r < m; ++r) {
    z[r] = rr[r] / rows[r].diag;
    pp[r] = z[r];
    rz += rr[r] * z[r];
    rn2 += rr[r] * rr[r];
  }
  int it = 0;
  double rnorm = sqrt(rn2);
  int status = rnorm <= rtol * bnorm ? 0 : 1;
  while (status != 0 && it < max_iter) {
    double pAp = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : pAp) num_threads(nt)
    for (int64_t r = 0; r < m; ++r) {
      double s = rows[r].diag * pp[r];
      for (int f = 0; f < 6; ++f)
        if (rows[r].w[f] != 0.0) s -= rows[r].w[f] * pp[r + ((f & 1) ? 1 : -1) * strides[f / 2]];
      Ap[r] = s;
      pAp += pp[r] * s;
    }
    double alpha = rz / pAp;
    double rz_new = 0.0;
    rn2 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz_new, rn2) num_threads(nt)
    for (int64_t r = 0; r < m; ++r) {
      x[r] += alpha * pp[r];
      rr[r] -= alpha * Ap[r];
      z[r] = rr[r] / rows[r].diag;
      rz_new += rr[r] * z[r];
      rn2 += rr[r] * rr[r];
    }
    ++it;
    rnorm = sqrt(rn2);
    if (rnorm <= rtol * bnorm) {
      status = 0;
      break;
    }
    double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t r = 0; r < m; ++r) pp[r] = z[r] + beta * pp[r];
  }
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = bnorm > 0 ? rnorm / bnorm : 0.0;
  free(rr);
  free(z);
  free(pp);
  free(Ap);
  return status;
}

/* the rows of every interior node (OpenMP over rows) */
static void grid_rows_all(const nbo_problem* pg, int n, const double* Jn, grid_row* rows, int nt) {
  int m1 = n - 1;
  int64_t m = (int64_t)m1 * m1 * m1;
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t r = 0; r < m; ++r) {
    int i = 1 + (int)(r % m1), j = 1 + (int)((r / m1) % m1), k = 1 + (int)(r / ((int64_t)m1 * m1));
    grid_row_build(pg, n, i, j, k, Jn, &rows[r]);
  }
}

/* the full node array: interior unknowns, Dirichlet data on the boundary */
static void grid_write_nodes(const nbo_problem* pg, int n, const double* x, double* u_out) {
  int m1 = n - 1;
  double hg = 2.0 / n;
  for (int k = 0; k <= n; ++k)
    for (int j = 0; j <= n; ++j)
      for (int i = 0; i <= n; ++i) {
        int64_t id = node_id(n, i, j, k);
        if (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n) {
          double q[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};
          u_out[id] = nbo_dirichlet_g(pg, q);
        } else {
          u_out[id] = x[(i - 1) + (int64_t)m1 * ((j - 1) + (int64_t)m1 * (k - 1))];
        }
      }
}

/* The grid method the NBM is bootstrapped from (Sec. 1, Sec. 3): the rows
 * above on the grid of spacing 2/n with the exact node jump, solved by Jacobi
 * PCG from zero to ||b - A x|| <= rtol ||b||. */
int nbo_grid_cg_solve(const nbo_problem* pr, int n, double rtol, int max_iter, double* u_out,
                      int* iters_out, double* relres_out, int n_threads) {
  nbo_problem pg = *pr;
  pg.h = 2.0 / n;
  int nt = pick_threads(n_threads);
  int m1 = n - 1;
  int64_t m = (int64_t)m1 * m1 * m1;
  grid_row* rows = (grid_row*)malloc(sizeof(grid_row) * m);
  grid_rows_all(&pg, n, NULL, rows, nt);
  double* x = (double*)calloc(m, sizeof(double));
  int status = grid_cg_core(rows, m1, x, rtol, max_iter, nt, iters_out, relres_out);
  grid_write_nodes(&pg, n, x, u_out);
  free(rows);
  free(x);
  return status;
}

/* ======================================================================
 * Extrapolated value jump at the grid nodes (the grid scheme's reading of
 * carrying u+ - u- off Gamma to a node of the other side).  For a node x:
 *   x_G = x moved onto phi = 0 by three Newton steps along grad phi,
 *   d   = phi(x) / |grad phi(x)|   (signed distance, > 0 in Omega+),
 *   n   = grad phi(x_G) / |grad phi(x_G)|,
 *   J(x) = alpha(x_G) + d G,   G = [d_n u] = d_n u+ - d_n u-  at x_G
 * (Taylor in d: J(x) - (u+(x) - u-(x)) = O(d^2)).  The flux jump
 * beta = mu+ d_n u+ - mu- d_n u- fixes G once the normal derivative of one
 * side is known; the side with the smaller mu, s*, is lagged:
 *   mu- <= mu+:  G = beta/mu+ - (1 - mu-/mu+) d_n u-
 *   mu+ <  mu-:  G = beta/mu- + (1 - mu+/mu-) d_n u+
 * (all coefficients at x_G).  Dropping the lag term gives G = beta/mu_big,
 * which is first order in h.  Nodes with |d| > 3h, or where grad phi
 * vanishes, get J = 0: no row weights them (a face or cell touches the
 * other phase only within about h of Gamma).
 * ==================================================================== */
int nbo_jump_extrap(const nbo_problem* pr, const double x[3], double h, int use_lag,
                    double dn_small, double* J, double xg[3], double nrm[3], int* small_side) {
  double g[3];
  double ph = nbo_phi(pr, x);
  nbo_grad_phi(pr, x, g);
  double gn = norm3(g);
  *J = 0.0;
  *small_side = 0;
  for (int i = 0; i < 3; ++i) xg[i] = x[i], nrm[i] = 0.0;
  /* the band edge sits 1e-9 outside 3h so that nodes at exactly 3h (lattice
   * points on a sphere) fall inside whatever the rounding of d */
  if (!(gn > 1e-300) || fabs(ph / gn) > 3.0 * h * (1.0 + 1e-9)) return 1;
  double d = ph / gn;
  for (int it = 0; it < 3; ++it) {
    double gg[3];
    double f = nbo_phi(pr, xg);
    nbo_grad_phi(pr, xg, gg);
    double q = gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2];
    if (q <= 1e-300) break;
    for (int i = 0; i < 3; ++i) xg[i] -= f * gg[i] / q;
  }
  double gx[3];
  nbo_grad_phi(pr, xg, gx);
  double gxn = norm3(gx);
  if (!(gxn > 1e-300)) return 1;
  for (int i = 0; i < 3; ++i) nrm[i] = gx[i] / gxn;
  double mum = nbo_mu(pr, 0, xg), mup = nbo_mu(pr, 1, xg), beta = nbo_beta(pr, xg);
  double G;
  if (mum <= mup) {
    *small_side = 0;
    G = beta / mup - (use_lag ? (1.0 - mum / mup) * dn_small : 0.0);
  } else {
    *small_side = 1;
    G = beta / mum + (use_lag ? (1.0 - mup / mum) * dn_small : 0.0);
  }
  *J = nbo_alpha(pr, xg) + d * G;
  return 0;
}

/* Normal derivative of side s at x_G from the node values u (the full
 * (n+1)^3 array of an iterate): least-squares fit of a linear function
 * a + g.(q - x_G) to the interior nodes q of phase s in the 3x3x3 block
 * around the node nearest x_G - h n (s = minus) or x_G + h n (s = plus)
 * (a midway point takes the upper node),
 * i.e. one spacing into side s, so that the block holds at least two layers
 * of side-s nodes (normal equations, Cholesky), dn = g . nrm.
 * Returns 1 (no value) with fewer than 4 such nodes or a degenerate fit. */
int nbo_fit_dn(const nbo_problem* pr, int n, const double* u, int s, const double xg[3],
               const double nrm[3], double* dn) {
  double hg = 2.0 / n;
  int c[3];
  for (int i = 0; i < 3; ++i) {
    double xc = xg[i] + (s == 0 ? -hg : hg) * nrm[i];
    /* nearest node; a point midway between two nodes (symmetric interfaces
     * put x_G there) takes the upper one, by a margin far above rounding */
    c[i] = (int)floor((xc + 1.0) / hg + 0.5 + 1e-6);
    if (c[i] < 2) c[i] = 2;
    if (c[i] > n - 2) c[i] = n - 2;
  }
  double M[4][4] = {{0}}, rhs[4] = {0};
  int cnt = 0;
  for (int dk = -1; dk <= 1; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        int q[3] = {c[0] + di, c[1] + dj, c[2] + dk};
        if (q[0] < 1 || q[1] < 1 || q[2] < 1 || q[0] > n - 1 || q[1] > n - 1 || q[2] > n - 1)
          continue;  /* interior nodes only (reached for n < 4) */
        double xq[3] = {-1.0 + q[0] * hg, -1.0 + q[1] * hg, -1.0 + q[2] * hg};
        if (nbo_phase(pr, xq) != s) continue;
        double bv[4] = {1.0, (xq[0] - xg[0]) / hg, (xq[1] - xg[1]) / hg, (xq[2] - xg[2]) / hg};
        double uq = u[node_id(n, q[0], q[1], q[2])];
        for (int a = 0; a < 4; ++a) {
          rhs[a] += bv[a] * uq;
          for (int b = 0; b < 4; ++b) M[a][b] += bv[a] * bv[b];
        }
        ++cnt;
      }
  if (cnt < 4) return 1;
  /* Cholesky M = L L^T (M is SPD when the nodes span an affine basis) */
  double L[4][4] = {{0}};
  for (int a = 0; a < 4; ++a) {
    for (int b = 0; b <= a; ++b) {
      double t = M[a][b];
      for (int k = 0; k < b; ++k) t -= L[a][k] * L[b][k];
      if (a == b) {
        if (!(t > 1e-8 * M[0][0])) return 1;
        L[a][a] = sqrt(t);
      } else {
        L[a][b] = t / L[b][b];
      }
    }
  }
  double y[4], cf[4];
  for (int a = 0; a < 4; ++a) {
    double t = rhs[a];
    for (int k = 0; k < a; ++k) t -= L[a][k] * y[k];
    y[a] = t / L[a][a];
  }
  for (int a = 3; a >= 0; --a) {
    double t = y[a];
    for (int k = a + 1; k < 4; ++k) t -= L[k][a] * cf[k];
    cf[a] = t / L[a][a];
  }
  *dn = (cf[1] * nrm[0] + cf[2] * nrm[1] + cf[3] * nrm[2]) / hg;
  return 0;
}

/* J at every node: lagged from the iterate u (u != NULL), or first order */
static void grid_jumps(const nbo_problem* pg, int n, const double* u, double* Jn, int nt) {
  int64_t N1 = n + 1, total = N1 * N1 * N1;
  double hg = 2.0 / n;
#pragma omp parallel for schedule(static) num_threads(nt)
  for (int64_t id = 0; id < total; ++id) {
    int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
    Jn[id] = 0.0;
    if (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n) continue;
    double x[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg}, xg[3], nrm[3], J, dn = 0.0;
    int ss;
    if (nbo_jump_extrap(pg, x, hg, 0, 0.0, &J, xg, nrm, &ss)) continue;
    if (u && nbo_fit_dn(pg, n, u, ss, xg, nrm, &dn) == 0)
      nbo_jump_extrap(pg, x, hg, 1, dn, &J, xg, nrm, &ss);
    Jn[id] = J;
  }
}

/* Grid solve with a choice of node jump (jump_mode): 0 exact (as
 * nbo_grid_cg_solve), 2 extrapolated first order (one solve), 1 extrapolated
 * with the lagged normal derivative: pass 1 is the first-order solve, each
 * later pass refits the lag from the previous solution, rebuilds the RHS and
 * re-solves from the previous solution, until
 *   max |J_new - J| <= jtol max(1, max |J_new|)
 * (converged, returns 0).  If max_passes go by without that, the solve falls
 * back to the first-order jump (re-solved from the last solution) and
 * returns 2.  Returns 1 if a CG solve does not converge.  passes_out counts
 * the lagged passes (1 for modes 0 and 2), dj_out the last max |J_new - J|. */
int nbo_grid_solve_jump(const nbo_problem* pr, int n, int jump_mode, double rtol, int max_iter,
                        int max_passes, double jtol, double* u_out, int* iters_out,
                        double* relres_out, int* passes_out, double* dj_out, int n_threads) {
  nbo_problem pg = *pr;
  pg.h = 2.0 / n;
  int nt = pick_threads(n_threads);
  int m1 = n - 1;
  int64_t m = (int64_t)m1 * m1 * m1, total = (int64_t)(n + 1) * (n + 1) * (n + 1);
  grid_row* rows = (grid_row*)malloc(sizeof(grid_row) * m);
  double* x = (double*)calloc(m, sizeof(double));
  double* Jn = NULL;
  double* Jnew = NULL;
  if (jump_mode != 0) {
    Jn = (double*)malloc(sizeof(double) * total);
    Jnew = (double*)malloc(sizeof(double) * total);
    grid_jumps(&pg, n, NULL, Jn, nt);
  }
  grid_rows_all(&pg, n, Jn, rows, nt);
  int it_total = 0, it = 0, passes = 1;
  double rr = 0.0, dj = 0.0;
  int status = grid_cg_core(rows, m1, x, rtol, max_iter, nt, &it, &rr);
  it_total += it;
  grid_write_nodes(&pg, n, x, u_out);
  if (jump_mode == 1 && status == 0) {
    int converged = 0;
    while (passes < max_passes && !converged) {
      grid_jumps(&pg, n, u_out, Jnew, nt);
      double jmax = 0.0;
      dj = 0.0;
      for (int64_t id = 0; id < total; ++id) {
        double e = fabs(Jnew[id] - Jn[id]);
        if (e > dj) dj = e;
        if (fabs(Jnew[id]) > jmax) jmax = fabs(Jnew[id]);
      }
      double* t = Jn;
      Jn = Jnew;
      Jnew = t;
      grid_rows_all(&pg, n, Jn, rows, nt);
      ++passes;
      status = grid_cg_core(rows, m1, x, rtol, max_iter, nt, &it, &rr);
      it_total += it;
      grid_write_nodes(&pg, n, x, u_out);
      if (status != 0) break;
      converged = dj <= jtol * (jmax > 1.0 ? jmax : 1.0);
    }
    if (status == 0 && !converged) {  /* stalled: the first-order jump instead */
      grid_jumps(&pg, n, NULL, Jn, nt);
      grid_rows_all(&pg, n, Jn, rows, nt);
      status = grid_cg_core(rows, m1, x, rtol, max_iter, nt, &it, &rr);
      it_total += it;
      grid_write_nodes(&pg, n, x, u_out);
      status = status == 0 ? 2 : 1;
    }
  }
  if (iters_out) *iters_out = it_total;
  if (relres_out) *relres_out = rr;
  if (passes_out) *passes_out = passes;
  if (dj_out) *dj_out = dj;
  free(rows);
  free(x);
  free(Jn);
  free(Jnew);
  return status;
}

/* L-infinity and RMS error against the exact solution of the node's phase
 * over the interior nodes (the paper's metrics, Table 1). */
void nbo_grid_error(const nbo_problem* pr, int n, const double* u, double* linf, double* rmse) {
  double hg = 2.0 / n, mx = 0.0, s2 = 0.0;
  int64_t cnt = 0;
  for (int k = 1; k < n; ++k)
    for (int j = 1; j < n; ++j)
      for (int i = 1; i < n; ++i) {
        double q[3] = {-1.0 + i * hg, -1.0 + j * hg, -1.0 + k * hg};
        int s = nbo_phase(pr, q);
        double e = fabs(u[node_id(n, i, j, k)] - nbo_exact_u(pr, s, q));
        if (e > mx) mx = e;
        s2 += e * e;
        ++cnt;
      }
  *linf = mx;
  *rmse = cnt ? sqrt(s2 / cnt) : 0.0;
}
