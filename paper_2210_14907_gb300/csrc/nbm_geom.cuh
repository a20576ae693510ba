// nbm_geom.cuh -- geometry of the implicit compute cell (arXiv
// 2210.14907, Fig. 2: where the interface crosses the cell): the level set is taken
// linear on each tetrahedron of the Freudenthal-Kuhn six-tetrahedron split of
// the cube, which gives closed forms for the volume fractions, the face
// fractions (each face split along the diagonal from its lowest to its
// highest corner, the split the tetrahedra induce) and the interface polygon.
#pragma once

#include "nbm_device.cuh"

namespace nbm {

// The closed forms below are templated on the real type T: FP64 for the grid
// rows and the FP64-row mode; FP32 (on cell-local coordinates, where the
// corners are exactly +-1/2) for the cut cells of the FP32-row mode.

// fraction of the triangle (corner values a, b, c; phi linear) with phi <= 0
template <typename T>
__device__ inline T frac_tri(T a, T b, T c) {
  int na = a <= T(0), nb = b <= T(0), nc = c <= T(0);
  int k = na + nb + nc;
  if (k == 0) return T(0);
  if (k == 3) return T(1);
  if (k == 1) {
    T l = na ? a : (nb ? b : c);
    T o1 = na ? b : a, o2 = nc ? b : c;  // the two positive values
    return (l / (l - o1)) * (l / (l - o2));
  }
  T l = !na ? a : (!nb ? b : c);
  T o1 = !na ? b : a, o2 = !nc ? b : c;  // the two non-positive values
  return T(1) - (l / (l - o1)) * (l / (l - o2));
}

// Element i of a 4-array and row i of a 4 x 3 array by selects, so that the
// arrays stay in registers: a run-time index into a register array would put
// it in local memory (the scans below pick vertices by their signs).
template <typename T>
__device__ __forceinline__ T sel4(const T a[4], int i) {
  return i == 0 ? a[0] : i == 1 ? a[1] : i == 2 ? a[2] : a[3];
}
template <typename T>
__device__ __forceinline__ void sel4_row(const T X[4][3], int i, T o[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) o[c] = i == 0 ? X[0][c] : i == 1 ? X[1][c] : i == 2 ? X[2][c] : X[3][c];
}

// The vertex alone on its side of a tetrahedron with `neg` (1 or 3) corner
// values <= 0: the last one in vertex order whose sign is the minority's.
template <typename T>
__device__ __forceinline__ int lone_vertex(const T f[4], bool want_neg) {
  int lone = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if ((f[i] <= T(0)) == want_neg) lone = i;
  return lone;
}

// fraction of the tetrahedron (corner values f; phi linear) with phi <= 0
template <typename T>
__device__ inline T frac_tet(const T f[4]) {
  int neg = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) neg += f[i] <= T(0);
  if (neg == 0) return T(0);
  if (neg == 4) return T(1);
  if (neg == 1 || neg == 3) {
    const int lone = lone_vertex<T>(f, neg == 1);
    const T fl = sel4<T>(f, lone);
    T prod = T(1);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i != lone) prod *= fl / (fl - f[i]);
    return neg == 1 ? prod : T(1) - prod;
  }
  // two on each side: A, B = -values below, C, D = values above
  T A = T(-1), B = T(-1), C = T(-1), D = T(-1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (f[i] <= T(0)) {
      if (A < T(0)) A = -f[i]; else B = -f[i];
    } else {
      if (C < T(0)) C = f[i]; else D = f[i];
    }
  }
  T num = C * D * (A * A + A * B + B * B) + (C + D) * A * B * (A + B) + A * A * B * B;
  return num / ((C + A) * (D + A) * (C + B) * (D + B));
}

// zero of phi on the edge u -> v
template <typename T>
__device__ inline void lerp_zero(const T* xu, T fu, const T* xv, T fv, T* o) {
  T t = fu / (fu - fv);
  for (int i = 0; i < 3; ++i) o[i] = xu[i] + t * (xv[i] - xu[i]);
}

// area of the triangle a b c; adds area x centroid to wc
template <typename T>
__device__ inline T tri_area_acc(const T* a, const T* b, const T* c, T* wc) {
  T e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  T e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  T cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
    cz = e1[0] * e2[1] - e1[1] * e2[0];
  T ar = T(0.5) * sqrt(cx * cx + cy * cy + cz * cz);
  for (int i = 0; i < 3; ++i) wc[i] += ar * (a[i] + b[i] + c[i]) / T(3);
  return ar;
}

// area of the interface polygon inside the tetrahedron (vertices X, values f);
// adds area x centroid to wc
template <typename T>
__device__ inline T tet_iface(const T X[4][3], const T f[4], T* wc) {
  int neg = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) neg += f[i] <= T(0);
  if (neg == 0 || neg == 4) return T(0);
  if (neg == 1 || neg == 3) {
    // a triangle: the zeros on the edges from the lone vertex to the other
    // three, taken in vertex order, each edge oriented from its <= 0 end
    const bool want_neg = neg == 1;
    const int lone = lone_vertex<T>(f, want_neg);
    const int o[3] = {lone == 0 ? 1 : 0, lone <= 1 ? 2 : 1, lone <= 2 ? 3 : 2};
    T xl[3];
    sel4_row<T>(X, lone, xl);
    const T fl = sel4<T>(f, lone);
    T Pp[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T xi[3];
      sel4_row<T>(X, o[k], xi);
      const T fi = sel4<T>(f, o[k]);
      if (want_neg) lerp_zero<T>(xl, fl, xi, fi, Pp[k]);
      else lerp_zero<T>(xi, fi, xl, fl, Pp[k]);
    }
    return tri_area_acc<T>(Pp[0], Pp[1], Pp[2], wc);
  }
  // a quadrilateral: vertices a < b with phi <= 0, c < d above
  int a = -1, b = -1, c = -1, d = -1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (f[i] <= T(0)) { if (a < 0) a = i; else b = i; }
    else { if (c < 0) c = i; else d = i; }
  }
  T xa[3], xb[3], xc[3], xd[3];
  sel4_row<T>(X, a, xa);
  sel4_row<T>(X, b, xb);
  sel4_row<T>(X, c, xc);
  sel4_row<T>(X, d, xd);
  const T fa = sel4<T>(f, a), fb = sel4<T>(f, b), fc = sel4<T>(f, c), fd = sel4<T>(f, d);
  T Q[4][3];
  lerp_zero<T>(xa, fa, xc, fc, Q[0]);
  lerp_zero<T>(xa, fa, xd, fd, Q[1]);
  lerp_zero<T>(xb, fb, xd, fd, Q[2]);
  lerp_zero<T>(xb, fb, xc, fc, Q[3]);
  return tri_area_acc<T>(Q[0], Q[1], Q[2], wc) + tri_area_acc<T>(Q[0], Q[2], Q[3], wc);
}

struct CellGeo {
  double Vm;      // volume fraction of Omega-
  double Am[6];   // face fractions of Omega-, face f = 2 axis + (side > 0)
  double S;       // interface area / h^2
  double xg[3];   // area-weighted interface centroid projected onto phi = 0
  int has_jump;   // S > 0
  int cut;        // corners on both sides
};

// Geometry of the cell p + [-h/2, h/2]^3.  Uncut cells (all corners on one
// side, phi = 0 counted as minus) get fractions exactly 0 or 1.
__device__ inline void cell_geometry_d(const ProbDev& P, const double p[3], double h, CellGeo& g) {
  double C[8][3], F[8];
  int nneg = 0;
  for (int c = 0; c < 8; ++c) {
    for (int a = 0; a < 3; ++a) C[c][a] = p[a] + h * ((double)((c >> a) & 1) - 0.5);
    F[c] = phi_d(P, C[c][0], C[c][1], C[c][2]);
    nneg += F[c] <= 0.0;
  }
  g.S = 0.0;
  g.has_jump = 0;
  for (int a = 0; a < 3; ++a) g.xg[a] = p[a];
  if (nneg == 0 || nneg == 8) {
    const double v = nneg == 8 ? 1.0 : 0.0;
    g.Vm = v;
    for (int f = 0; f < 6; ++f) g.Am[f] = v;
    g.cut = 0;
    return;
  }
  g.cut = 1;
  double vneg = 0.0, area = 0.0, wc[3] = {0.0, 0.0, 0.0};
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
#pragma unroll
  for (int t = 0; t < 6; ++t) {  // unrolled: every index below is a constant
    int v1 = 1 << perm[t][0];
    int v2 = v1 | (1 << perm[t][1]);
    int idx[4] = {0, v1, v2, 7};
    double Xt[4][3], ft[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      for (int a = 0; a < 3; ++a) Xt[k][a] = C[idx[k]][a];
      ft[k] = F[idx[k]];
    }
    vneg += frac_tet<double>(ft) / 6.0;
    area += tet_iface<double>(Xt, ft, wc);
  }
  g.Vm = vneg;
  for (int a = 0; a < 3; ++a) {
    int j = (a + 1) % 3, k = (a + 2) % 3;
    for (int sd = 0; sd < 2; ++sd) {
      int b0 = sd << a;
      int c00 = b0, c10 = b0 | (1 << j), c01 = b0 | (1 << k), c11 = c10 | (1 << k);
      g.Am[2 * a + sd] =
          0.5 * (frac_tri<double>(F[c00], F[c10], F[c11]) + frac_tri<double>(F[c00], F[c01], F[c11]));
    }
  }
  g.S = area / (h * h);
  g.has_jump = area > 0.0;
  if (area > 0.0) {
    for (int a = 0; a < 3; ++a) g.xg[a] = wc[a] / area;
    for (int it = 0; it < 3; ++it) {  // Newton projection onto phi = 0
      double gr[3];
      double ph = phi_d(P, g.xg[0], g.xg[1], g.xg[2]);
      grad_phi_d(P, g.xg, gr);
      double gg = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
      if (gg <= 1e-300) break;
      for (int a = 0; a < 3; ++a) g.xg[a] -= ph * gr[a] / gg;
    }
  }
}

}  // namespace nbm
