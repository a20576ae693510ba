// nbm_cg.cu -- the plain mesh-based method the NBM is bootstrapped from
// (arXiv 2210.14907, Sec. 1 and Sec. 3): the same finite-volume balance row on
// the nodes of a grid of spacing h = 2/n, one unknown per interior node, solved
// by Jacobi-preconditioned conjugate gradients in FP64 (nbm_grid_cg_solve; run
// as CG on the Jacobi-scaled system D^-1/2 A D^-1/2, the same iterates in
// exact arithmetic with fewer bytes), or to the same FP64 residual test by
// FP32 inner PCG corrections of FP64 residuals (nbm_grid_solve_refined).  In
// FP64 the SpMV is bound by GB300's narrow FP64 pipe, in FP32 the kernels by
// HBM.
//
// Row of interior node p (cell p + [-h/2, h/2]^3, fractions as in nbm_geom.cuh):
//   sum_f w_f (u_p - u_q) + h^2 sum_s V^s k^s u_p = -known_p,
//   w_f = sum_s A^s_f mu^s  (shared by the two cells of the face: A is SPD),
// where the value of network/side s at a node q of the other side is u_q plus
// the value jump J(q) = u+ - u- carried to q: the manufactured pair's own
// u+(q) - u-(q) (the exact jump), or alpha(x_G) + d [d_n u] extrapolated from
// the interface (k_node_jump; the normal derivative of the small-mu side
// lagged from the previous solve, or dropped); all such terms, the source,
// the interface flux h S beta and the Dirichlet data move to the right-hand
// side.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "nbm_device.cuh"
#include "nbm_geom.cuh"

namespace nbm {
namespace {

constexpr int kB = 256;

struct Grid {
  int n, m1;      // cells per axis, interior nodes per axis
  int64_t m;      // interior nodes
  double h;
};

// grid node coordinate -1 + i h with the product rounded before the sum (no
// fused multiply-add), so that nodes on a symmetry plane of the level set
// (x = 0 at i = n/2) lie exactly on it
__device__ inline double node_coord(int i, double h) { return __dadd_rn(-1.0, __dmul_rn((double)i, h)); }

__device__ inline void node_xyz(const Grid& G, int64_t r, int& i, int& j, int& k, double x[3]) {
  i = 1 + (int)(r % G.m1);
  j = 1 + (int)((r / G.m1) % G.m1);
  k = 1 + (int)(r / ((int64_t)G.m1 * G.m1));
  x[0] = node_coord(i, G.h);
  x[1] = node_coord(j, G.h);
  x[2] = node_coord(k, G.h);
}

__device__ inline int phase_d(const ProbDev& P, const double x[3]) {
  return phi_d(P, x[0], x[1], x[2]) <= 0.0 ? 0 : 1;
}

// jump correction of side s at a node of side sx: U^s = u + c[s]
__device__ inline void jump_corr(double jmp, int sx, double c[2]) {
  c[0] = sx == 1 ? -jmp : 0.0;
  c[1] = sx == 0 ? jmp : 0.0;
}

// Rows of every interior node.  Jn (interior-node array) holds the node jump
// J = u+ - u- carried to each node; NULL takes the manufactured pair's own
// u+(x) - u-(x) (the exact jump).
__global__ void __launch_bounds__(kB) k_grid_rows(ProbDev P, Grid G, const double* Jn,
                                                  double* diag, double* wx, double* wy, double* wz,
                                                  double* rhs) {
  pdl_enter();
  const int64_t r = (int64_t)blockIdx.x * kB + threadIdx.x;
  if (r >= G.m) return;
  int idx[3];
  double p[3];
  node_xyz(G, r, idx[0], idx[1], idx[2], p);
  const double h = G.h;
  CellGeo cg;
  cell_geometry_d(P, p, h, cg);
  const int sp = phase_d(P, p);
  double cp[2];
  jump_corr(Jn ? Jn[r] : alpha_d(P, p), sp, cp);
  double dg = 0.0, known = 0.0;
  for (int s = 0; s < 2; ++s) {
    const double V = s ? 1.0 - cg.Vm : cg.Vm;
    dg += h * h * V * P.k[s];
    known += h * h * V * (P.k[s] * cp[s] - rhs_f<double>(P, s, p[0], p[1], p[2]));
  }
  double wplus[3] = {0.0, 0.0, 0.0};
  for (int f = 0; f < 6; ++f) {
    const int ax = f >> 1, sg = (f & 1) ? 1 : -1;
    int nb[3] = {idx[0], idx[1], idx[2]};
    nb[ax] += sg;
    const double q[3] = {node_coord(nb[0], h), node_coord(nb[1], h), node_coord(nb[2], h)};
    const bool bnd = nb[ax] == 0 || nb[ax] == G.n;
    double cq[2] = {0.0, 0.0};
    if (!bnd) {
      const int64_t rq = (nb[0] - 1) + (int64_t)G.m1 * ((nb[1] - 1) + (int64_t)G.m1 * (nb[2] - 1));
      jump_corr(Jn ? Jn[rq] : alpha_d(P, q), phase_d(P, q), cq);
    }
    // face centre: the same point for both cells of the face, so the face
    // weight (and the matrix) stays symmetric with variable mu
    double fc[3] = {p[0], p[1], p[2]};
    fc[ax] += 0.5 * sg * h;
    double wf = 0.0;
    for (int s = 0; s < 2; ++s) {
      const double A = s ? 1.0 - cg.Am[f] : cg.Am[f];
      const double a = A * mu_at<double>(P, s, fc[0], fc[1], fc[2]);
      wf += a;
      known -= a * (cq[s] - cp[s]);
    }
    dg += wf;
    if (bnd) known -= wf * dirichlet_g<double>(P, q[0], q[1], q[2]);
    else if (sg > 0) wplus[ax] = wf;
  }
  if (cg.cut && cg.has_jump) known += h * cg.S * beta_d(P, cg.xg);
  diag[r] = dg;
  wx[r] = wplus[0];
  wy[r] = wplus[1];
  wz[r] = wplus[2];
  rhs[r] = -known;
}

// The Jacobi-scaled system D^-1/2 A D^-1/2 x^ = D^-1/2 b, x = D^-1/2 x^ (D =
// diag A): unit diagonal, face weights w / sqrt(d_p d_q), in place.  CG on it
// is Jacobi-preconditioned CG on A in exact arithmetic, and it reads neither
// the diagonal nor its inverse in the SpMV or the direction update.
__global__ void __launch_bounds__(kB) k_scale_rows(Grid G, const double* diag,
                                                   double* wx, double* wy, double* wz, double* b) {
  pdl_enter();
  const int64_t s1 = G.m1, s2 = (int64_t)G.m1 * G.m1;
  for (int64_t r = (int64_t)blockIdx.x * kB + threadIdx.x; r < G.m; r += (int64_t)gridDim.x * kB) {
    const int i = (int)(r % G.m1), j = (int)((r / G.m1) % G.m1), k = (int)(r / s2);
    const double dr = diag[r];
    if (i + 1 < G.m1) wx[r] /= sqrt(dr * diag[r + 1]);
    if (j + 1 < G.m1) wy[r] /= sqrt(dr * diag[r + s1]);
    if (k + 1 < G.m1) wz[r] /= sqrt(dr * diag[r + s2]);
    b[r] /= sqrt(dr);
  }
}

// Block partial sums: each thread's NV values are summed over the warp in T
// (FP32 or FP64), then over the block's warps in FP64 by thread 0, which
// writes part[v * stride + idx].
template <typename T, int NV>
__device__ inline void block_partials(T (&v)[NV], double* part, int64_t idx, int64_t stride) {
  __shared__ double red[NV][kB / 32];
  const int t = threadIdx.x + blockDim.x * threadIdx.y;  // blocks of kB threads, 1-D or 2-D
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((t & 31) == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q][t >> 5] = (double)v[q];
  __syncthreads();
  if (t == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < kB / 32; ++w) s += red[q][w];
      part[q * stride + idx] = s;
    }
}

// scalars[]: 0 rz, 1 pAp, 2 alpha, 3 rz_new, 4 rr, 5 beta (the CG recurrence
// on the Jacobi-scaled system); 6 ||r|| and 7 1/||r|| (the FP64 residual of the
// refined solve, unscaled norm), 8 sum d r^2 (= ||r||^2), 9 sum d b^2
// (= ||b||^2), 12 max |dJ|, 13 max |J| (node jump).  After the sums, POST_ALPHA
// sets alpha = rz / pAp, POST_BETA sets beta = rz_new / rz and rz = rz_new,
// POST_NORM sets ||r|| and its inverse; POST_SKIP leaves the partials unused.
enum { POST_SKIP = -1, POST_ALPHA = 1, POST_BETA = 2, POST_NORM = 3 };
constexpr int kMaxVec = 2;

// Fixed-order sum of nvec (<= 2) partial vectors of nparts entries by one
// block of kB threads into sc[slot + q], then the post step.  `l2`: read the
// partials from L2 (other blocks of the same launch wrote them).
__device__ void sum_partials(const double* part, int nparts, int nvec, double* sc, int slot,
                             int post, bool l2) {
  __shared__ double red[kMaxVec][kB];
  const int t = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll
  for (int q = 0; q < kMaxVec; ++q) {
    double s = 0.0;
    if (q < nvec)
      for (int b = t; b < nparts; b += kB)
        s += l2 ? __ldcg(part + (int64_t)q * nparts + b) : part[(int64_t)q * nparts + b];
    red[q][t] = s;
  }
  __syncthreads();
  for (int o = kB / 2; o > 0; o >>= 1) {
    if (t < o)
#pragma unroll
      for (int q = 0; q < kMaxVec; ++q) red[q][t] += red[q][t + o];
    __syncthreads();
  }
  if (t == 0) {
    for (int q = 0; q < nvec; ++q) sc[slot + q] = red[q][0];
    if (post == POST_ALPHA) sc[2] = sc[0] / sc[1];
    if (post == POST_BETA) {
      sc[5] = sc[3] / sc[0];
      sc[0] = sc[3];
    }
    if (post == POST_NORM) {  // residual norm of the refined solve
      sc[6] = sqrt(sc[8]);
      sc[7] = 1.0 / sc[6];
    }
  }
}

// The sum over a launch's block partials, done by its last block: each block
// takes a ticket after a device-scope fence (its partials are written); the
// block that draws the last ticket adds every partial in a fixed order and
// re-arms the ticket.  With no ticket (large grids) a separate
// k_reduce_parts launch does the sum.
__device__ void fold_partials(const double* part, int nparts, int nvec, double* sc, int slot,
                              int post, int* ticket) {
  if (!ticket) return;
  __shared__ int last;
  const int t = threadIdx.x + blockDim.x * threadIdx.y;
  __syncthreads();  // the block's partials are written (by thread 0)
  if (t == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1) == nparts - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  sum_partials(part, nparts, nvec, sc, slot, post, true);
  if (t == 0) *ticket = 0;
}

// The same sum as fold_partials as a separate one-block launch.  A fold costs
// every block a device-scope fence before it retires; on large grids that
// costs more than the extra launch, so they use this kernel instead.
__global__ void __launch_bounds__(kB) k_reduce_parts(const double* part, int nparts,
                                                     int nvec, double* sc, int slot, int post) {
  pdl_enter();
  sum_partials(part, nparts, nvec, sc, slot, post, false);
}

// y = A v on the interior nodes: the Jacobi-scaled operator (UNIT: unit
// diagonal, `diag` unused) or the unscaled one; v . y summed into sc[1]
// (post = POST_ALPHA)
// or not at all (POST_SKIP).  Blocks of kB threads: blockDim.x nodes of a row
// times blockDim.y rows; grid z = slabs of kz planes.  Each thread walks its
// (i, j) column through the slab, keeping the z neighbours in registers, so
// node indices need no integer division and each thread reduces once.
// (FP32: 8 blocks, i.e. 2048 threads, per SM; at most 32 registers)
template <typename T, bool UNIT>
__global__ void __launch_bounds__(kB, sizeof(T) == 4 ? 8 : 6) k_spmv_dot(Grid G, int kz,
                                                 const T* diag,
                                                 const T* wx,
                                                 const T* wy,
                                                 const T* wz,
                                                 const T* v, T* y,
                                                 double* part, double* sc, int post, int* ticket) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k0 = blockIdx.z * kz, k1 = min(k0 + kz, G.m1);
  const int64_t s1 = G.m1, s2 = (int64_t)G.m1 * G.m1;
  T d[1] = {T(0)};
  if (i < G.m1 && j < G.m1) {
    int64_t r = i + s1 * j + s2 * k0;
    T vm = k0 > 0 ? v[r - s2] : T(0), wzm = k0 > 0 ? wz[r - s2] : T(0);
    T vc = v[r];
    for (int k = k0; k < k1; ++k, r += s2) {
      const T vp = k + 1 < G.m1 ? v[r + s2] : T(0);
      const T wzc = wz[r];  // zero on the last interior plane
      T acc = UNIT ? vc : diag[r] * vc;
      if (i + 1 < G.m1) acc -= wx[r] * v[r + 1];
      if (i > 0) acc -= wx[r - 1] * v[r - 1];
      if (j + 1 < G.m1) acc -= wy[r] * v[r + s1];
      if (j > 0) acc -= wy[r - s1] * v[r - s1];
      acc -= wzc * vp;
      acc -= wzm * vm;
      y[r] = acc;
      d[0] += vc * acc;
      vm = vc;
      vc = vp;
      wzm = wzc;
    }
  }
  if (post == POST_SKIP) return;
  const int nparts = (int)(gridDim.x * gridDim.y * gridDim.z);
  block_partials<T, 1>(d, part, blockIdx.x + gridDim.x * ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z), 0);
  fold_partials(part, nparts, 1, sc, 1, post, ticket);
}

// x += alpha p; r -= alpha Ap; partials of the recurrence's r.z and of the
// stopping norm ||r||^2 of the unscaled system.  UNIT (scaled system, dv = D):
// r.z = r^.r^ and ||r||^2 = sum d r^2.  Otherwise (Jacobi PCG, dv = 1/D):
// r.z = sum r^2 / d and ||r||^2 = r.r.  The scalars stay FP64 and each thread
// strides over the nodes, reducing once.
template <typename T, bool UNIT>
__global__ void __launch_bounds__(kB) k_update(Grid G, double* sc, const T* dv,
                                               const T* p,
                                               const T* Ap, T* x, T* r,
                                               double* part, int* ticket) {
  pdl_enter();
  T acc[2] = {T(0), T(0)};
  const T a = (T)sc[2];
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < G.m; i += (int64_t)gridDim.x * kB) {
    x[i] += a * p[i];
    const T ri = r[i] - a * Ap[i];
    r[i] = ri;
    const T rr = ri * ri;
    acc[0] += UNIT ? rr : rr * dv[i];
    acc[1] += UNIT ? dv[i] * rr : rr;
  }
  block_partials<T, 2>(acc, part, blockIdx.x, gridDim.x);
  fold_partials(part, gridDim.x, 2, sc, 3, POST_BETA, ticket);
}

// p = z + beta p with z = r (UNIT) or r / D (`inv_diag`; Jacobi PCG)
// (beta = 0: p = z for the first direction)
template <typename T, bool UNIT>
__global__ void __launch_bounds__(kB) k_pupdate(Grid G, const double* sc, int first,
                                                const T* inv_diag,
                                                const T* r, T* p) {
  pdl_enter();
  const T beta = first ? T(0) : (T)sc[5];
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < G.m; i += (int64_t)gridDim.x * kB) {
    const T z = UNIT ? r[i] : r[i] * inv_diag[i];
    p[i] = first ? z : z + beta * p[i];
  }
}

// ---- refined solve: FP64 residuals, FP32 inner PCG ----

// FP32 copies of the unscaled operator for the inner Jacobi PCG of the
// refined solve: D, 1/D and the face weights w = w^ sqrt(d_p d_q)
__global__ void __launch_bounds__(kB) k_to_f32(Grid G, const double* diag,
                                               const double* wx,
                                               const double* wy,
                                               const double* wz, float* d32,
                                               float* idg32, float* wx32, float* wy32,
                                               float* wz32) {
  pdl_enter();
  const int64_t s1 = G.m1, s2 = (int64_t)G.m1 * G.m1;
  for (int64_t r = (int64_t)blockIdx.x * kB + threadIdx.x; r < G.m; r += (int64_t)gridDim.x * kB) {
    const int i = (int)(r % G.m1), j = (int)((r / G.m1) % G.m1), k = (int)(r / s2);
    const double dr = diag[r];
    d32[r] = (float)dr;
    idg32[r] = (float)(1.0 / dr);
    wx32[r] = i + 1 < G.m1 ? (float)(wx[r] * sqrt(dr * diag[r + 1])) : 0.f;
    wy32[r] = j + 1 < G.m1 ? (float)(wy[r] * sqrt(dr * diag[r + s1])) : 0.f;
    wz32[r] = k + 1 < G.m1 ? (float)(wz[r] * sqrt(dr * diag[r + s2])) : 0.f;
  }
}

// r^ = b^ - r^ (r^ holds A^ x^ on entry); partials of sum d r^2 (= ||r||^2)
// and sum d b^2 (= ||b||^2), summed into sc[8], sc[9] (POST_NORM)
__global__ void __launch_bounds__(kB) k_defect(Grid G, const double* d,
                                               const double* b, double* r,
                                               double* part, double* sc, int* ticket) {
  pdl_enter();
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < G.m; i += (int64_t)gridDim.x * kB) {
    const double bi = b[i], ri = bi - r[i], di = d[i];
    r[i] = ri;
    acc[0] += di * ri * ri;
    acc[1] += di * bi * bi;
  }
  block_partials<double, 2>(acc, part, blockIdx.x, gridDim.x);
  fold_partials(part, gridDim.x, 2, sc, 8, POST_NORM, ticket);
}

// start of an inner solve (FP32 Jacobi PCG on the unscaled operator) of
// A e = r / ||r|| with r = D^1/2 r^: e = 0, r32 = r / ||r|| (norm 1),
// p32 = r32 / D; partials of r32.p32 and r32.r32
__global__ void __launch_bounds__(kB) k_inner_init(Grid G, double* sc,
                                                   const double* r64,
                                                   const float* d32,
                                                   const float* idg32, float* r32,
                                                   float* e32, float* p32, double* part,
                                                   int* ticket) {
  pdl_enter();
  float acc[2] = {0.f, 0.f};
  const double inv = sc[7];
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < G.m; i += (int64_t)gridDim.x * kB) {
    const float ri = (float)(r64[i] * inv) * sqrtf(d32[i]);
    const float z = ri * idg32[i];
    r32[i] = ri;
    e32[i] = 0.f;
    p32[i] = z;
    acc[0] += ri * z;
    acc[1] += ri * ri;
  }
  block_partials<float, 2>(acc, part, blockIdx.x, gridDim.x);
  fold_partials(part, gridDim.x, 2, sc, 3, POST_BETA, ticket);
}

// ---- extrapolated node jump ----

// d_n u_s at x_G from the interior iterate x^ of the scaled system (node
// values x^ / sqrt(d)): least-squares fit of
// a + g.(q - x_G) over the interior side-s nodes of the 3x3x3 block around
// the node nearest x_G -+ h n (one spacing into side s; a midway point takes
// the upper node), normal equations by
// Cholesky; false with fewer than 4 such nodes or a degenerate fit.
// `val(q, rq)` returns the node value at grid node q (rq: its interior index).
template <class Val>
__device__ bool fit_dn(const ProbDev& P, const Grid& G, Val val, int s, const double xg[3],
                       const double nrm[3], double* dn) {
  const double h = G.h;
  int c[3];
  for (int a = 0; a < 3; ++a) {
    const double xc = xg[a] + (s == 0 ? -h : h) * nrm[a];
    int ci = (int)floor((xc + 1.0) / h + 0.5 + 1e-6);  // a midway point takes the upper node
    ci = ci < 2 ? 2 : ci;
    c[a] = ci > G.n - 2 ? G.n - 2 : ci;
  }
  double M[4][4] = {}, rhs[4] = {};
  int cnt = 0;
  for (int dk = -1; dk <= 1; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int q[3] = {c[0] + di, c[1] + dj, c[2] + dk};
        if (q[0] < 1 || q[1] < 1 || q[2] < 1 || q[0] > G.n - 1 || q[1] > G.n - 1 ||
            q[2] > G.n - 1)
          continue;
        const double xq[3] = {node_coord(q[0], h), node_coord(q[1], h), node_coord(q[2], h)};
        if (phase_d(P, xq) != s) continue;
        const double bv[4] = {1.0, (xq[0] - xg[0]) / h, (xq[1] - xg[1]) / h, (xq[2] - xg[2]) / h};
        const int64_t rq = (q[0] - 1) + (int64_t)G.m1 * ((q[1] - 1) + (int64_t)G.m1 * (q[2] - 1));
        const double uq = val(q, rq);
        for (int a = 0; a < 4; ++a) {
          rhs[a] += bv[a] * uq;
          for (int b = 0; b < 4; ++b) M[a][b] += bv[a] * bv[b];
        }
        ++cnt;
      }
  if (cnt < 4) return false;
  double L[4][4] = {};
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b <= a; ++b) {
      double t = M[a][b];
      for (int k = 0; k < b; ++k) t -= L[a][k] * L[b][k];
      if (a == b) {
        if (!(t > 1e-8 * M[0][0])) return false;
        L[a][a] = sqrt(t);
      } else {
        L[a][b] = t / L[b][b];
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
  *dn = (cf[1] * nrm[0] + cf[2] * nrm[1] + cf[3] * nrm[2]) / h;
  return true;
}

// Node jump J(x) = alpha(x_G) + d G at a node x within 3h of Gamma (0
// elsewhere): x_G by three Newton steps from the node, d = phi / |grad phi| at
// the node, G = [d_n u] from the flux jump with the small-mu side's d_n fitted
// from the node values val (lag = 1) or dropped (lag = 0).
template <class Val>
__device__ double node_jump(const ProbDev& P, const Grid& G, const double p[3], int lag, Val val) {
  double g[3];
  const double ph = phi_d(P, p[0], p[1], p[2]);
  grad_phi_d(P, p, g);
  const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double jn = 0.0;
  if (gn > 1e-300 && fabs(ph / gn) <= 3.0 * G.h * (1.0 + 1e-9)) {  // nodes at 3h: inside
    const double d = ph / gn;
    double xg[3] = {p[0], p[1], p[2]};
    for (int it = 0; it < 3; ++it) {
      double gg[3];
      const double f = phi_d(P, xg[0], xg[1], xg[2]);
      grad_phi_d(P, xg, gg);
      const double q = gg[0] * gg[0] + gg[1] * gg[1] + gg[2] * gg[2];
      if (q <= 1e-300) break;
      for (int a = 0; a < 3; ++a) xg[a] -= f * gg[a] / q;
    }
    double gx[3];
    grad_phi_d(P, xg, gx);
    const double gxn = sqrt(gx[0] * gx[0] + gx[1] * gx[1] + gx[2] * gx[2]);
    if (gxn > 1e-300) {
      const double nrm[3] = {gx[0] / gxn, gx[1] / gxn, gx[2] / gxn};
      const double mum = mu_at<double>(P, 0, xg[0], xg[1], xg[2]);
      const double mup = mu_at<double>(P, 1, xg[0], xg[1], xg[2]);
      const double beta = beta_d(P, xg);
      const int ss = mum <= mup ? 0 : 1;
      double dn = 0.0;
      const bool have = lag && fit_dn(P, G, val, ss, xg, nrm, &dn);
      const double Gj = ss == 0 ? beta / mup - (have ? (1.0 - mum / mup) * dn : 0.0)
                                : beta / mum + (have ? (1.0 - mup / mum) * dn : 0.0);
      jn = alpha_d(P, xg) + d * Gj;
    }
  }
  return jn;
}

// node_jump on every interior node, updated in place, from the iterate x^ of
// the scaled system (node values x^ / sqrt(d)).  Block partials of
// max |J_new - J| and max |J_new| go to part[] and part[gridDim.x + ...].
__global__ void __launch_bounds__(kB) k_node_jump(ProbDev P, Grid G, int lag,
                                                  const double* x,
                                                  const double* diag, double* J,
                                                  double* part) {
  pdl_enter();
  __shared__ double red[2][kB / 32];
  double mx[2] = {0.0, 0.0};
  auto val = [&](const int*, int64_t rq) { return x[rq] / sqrt(diag[rq]); };
  for (int64_t r = (int64_t)blockIdx.x * kB + threadIdx.x; r < G.m; r += (int64_t)gridDim.x * kB) {
    int i, j, k;
    double p[3];
    node_xyz(G, r, i, j, k, p);
    const double jn = node_jump(P, G, p, lag, val);
    mx[0] = fmax(mx[0], fabs(jn - J[r]));
    mx[1] = fmax(mx[1], fabs(jn));
    J[r] = jn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    for (int q = 0; q < 2; ++q) mx[q] = fmax(mx[q], __shfl_xor_sync(0xffffffffu, mx[q], o));
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 2; ++q) red[q][threadIdx.x >> 5] = mx[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < 2; ++q) {
      double m = 0.0;
      for (int w = 0; w < kB / 32; ++w) m = fmax(m, red[q][w]);
      part[q * (int64_t)gridDim.x + blockIdx.x] = m;
    }
}

// The node jump of grid_jump mode `mode` on all (n+1)^3 nodes (x fastest), from
// the node values u (read only by the lagged mode's fit): the exact jump
// alpha(x) = u+(x) - u-(x) of the manufactured pair, or node_jump (first
// order: lag 0; lagged: lag 1).
__global__ void __launch_bounds__(kB) k_node_jump_all(ProbDev P, Grid G, int mode,
                                                      const double* u, double* J) {
  pdl_enter();
  const int64_t n1 = G.n + 1, nodes = n1 * n1 * n1;
  auto val = [&](const int* q, int64_t) { return u[q[0] + n1 * (q[1] + n1 * (int64_t)q[2])]; };
  for (int64_t e = (int64_t)blockIdx.x * kB + threadIdx.x; e < nodes;
       e += (int64_t)gridDim.x * kB) {
    const int i = (int)(e % n1), j = (int)((e / n1) % n1), k = (int)(e / (n1 * n1));
    const double p[3] = {node_coord(i, G.h), node_coord(j, G.h), node_coord(k, G.h)};
    J[e] = mode == NBM_JUMP_EXACT ? alpha_d(P, p)
                                  : node_jump(P, G, p, mode == NBM_JUMP_EXTRAP ? 1 : 0, val);
  }
}

// sc[slot], sc[slot + 1] = maxima of the two partial vectors
__global__ void k_reduce_max2(const double* part, int nparts, double* sc, int slot) {
  pdl_enter();
  __shared__ double red[2][256];
  double m0 = 0.0, m1 = 0.0;
  for (int b = threadIdx.x; b < nparts; b += 256) {
    m0 = fmax(m0, part[b]);
    m1 = fmax(m1, part[nparts + b]);
  }
  red[0][threadIdx.x] = m0;
  red[1][threadIdx.x] = m1;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + o]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sc[slot] = red[0][0];
    sc[slot + 1] = red[1][0];
  }
}

// x^ += ||r|| D^1/2 e   (FP64; e is the inner solve's unscaled correction)
__global__ void __launch_bounds__(kB) k_correct(Grid G, const double* sc,
                                                const float* d32,
                                                const float* e32, double* x) {
  pdl_enter();
  const double s = sc[6];
  for (int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x; i < G.m; i += (int64_t)gridDim.x * kB)
    x[i] += s * (double)(e32[i] * sqrtf(d32[i]));
}

// the (n+1)^3 node array: x = x^ / sqrt(d) inside, Dirichlet data on the boundary
__global__ void __launch_bounds__(kB) k_write_nodes(ProbDev P, Grid G, const double* x,
                                                    const double* diag, double* u) {
  pdl_enter();
  const int64_t N1 = G.n + 1;
  const int64_t id = (int64_t)blockIdx.x * kB + threadIdx.x;
  if (id >= N1 * N1 * N1) return;
  const int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
  if (i == 0 || j == 0 || k == 0 || i == G.n || j == G.n || k == G.n) {
    u[id] = dirichlet_g<double>(P, node_coord(i, G.h), node_coord(j, G.h), node_coord(k, G.h));
  } else {
    const int64_t r = (i - 1) + (int64_t)G.m1 * ((j - 1) + (int64_t)G.m1 * (k - 1));
    u[id] = x[r] / sqrt(diag[r]);
  }
}

}  // namespace
}  // namespace nbm

using namespace nbm;

namespace nbm {
namespace {

// Grids up to this many unknowns fold each reduction into the kernel that
// produces the partials (measured: 12 % faster at 128^3, 3 % slower at 256^3).
constexpr int64_t kFoldMaxUnknowns = 8'000'000;

// problem, grid and launch shapes shared by the two solvers
struct CgSetup {
  ProbDev P;
  Grid G;
  int nb;      // one-node-per-thread blocks (row assembly)
  int nu;      // blocks of the strided vector kernels
  int kz;      // planes per thread in the SpMV
  dim3 sblock; // SpMV block: a run of a row times rows (kB threads)
  dim3 sgrid;  // SpMV grid
  int nsp;     // SpMV partials
  int64_t nodes;
  bool fold;   // reductions folded into the producing kernels (small grids)
};

int cg_setup(nbm_problem* p, int n, double rtol, int max_iter, const double* u_out, const char* who,
             CgSetup& S) {
  char msg[256];
  if (!p || !u_out) {
    set_error_message("NULL argument");
    return NBM_ERR_INVALID_ARG;
  }
  if (int rc = check_aligned(u_out, 8, "u_out")) return rc;
  if (n < 2 || n > 2048 || !(rtol > 0.0) || max_iter < 0) {
    snprintf(msg, sizeof(msg), "%s needs 2 <= n <= 2048, rtol > 0, max_iter >= 0 (n=%d)", who, n);
    set_error_message(msg);
    return NBM_ERR_INVALID_ARG;
  }
  nbm_problem_desc d = problem_desc(p);
  d.h = 2.0 / n;
  make_prob_dev(d, S.P);
  if (int rc = attach_level_set(p, S.P)) return rc;
  Grid& G = S.G;
  G.n = n;
  G.m1 = n - 1;
  G.m = (int64_t)G.m1 * G.m1 * G.m1;
  G.h = 2.0 / n;
  S.nb = (int)((G.m + kB - 1) / kB);
  const int resident = 8 * problem_num_sms(p);  // 2048 threads per SM
  S.nu = S.nb < resident ? S.nb : resident;
  // SpMV blocks: a power-of-two run of a row (32 ... kB nodes) times kB / run
  // rows; slabs of kz planes, kz chosen to keep about two threads per
  // resident thread slot (2048 per SM), between 2 and 16 planes
  int run = 32;  // a power of two, so that run x (kB / run) is exactly kB threads
  while (run < G.m1 && run < kB) run *= 2;
  S.sblock = dim3((unsigned)run, (unsigned)(kB / run), 1);
  const int gx = (G.m1 + run - 1) / run, gy = (G.m1 + (int)S.sblock.y - 1) / (int)S.sblock.y;
  const int64_t threads_per_plane = (int64_t)gx * run * gy * S.sblock.y;
  const int64_t slots = 2048LL * problem_num_sms(p);
  int64_t kz = threads_per_plane * G.m1 / (2 * slots);
  S.kz = (int)(kz < 2 ? 2 : kz > 16 ? 16 : kz);
  S.sgrid = dim3((unsigned)gx, (unsigned)gy, (unsigned)((G.m1 + S.kz - 1) / S.kz));
  S.nsp = (int)(S.sgrid.x * S.sgrid.y * S.sgrid.z);
  S.nodes = (int64_t)(n + 1) * (n + 1) * (n + 1);
  S.fold = G.m <= kFoldMaxUnknowns;
  return NBM_OK;
}

// device buffers of one solve, freed together
struct CgBuffers {
  void* ptr[24] = {};
  int n = 0;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T* get(size_t count) {
    void* q = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&q, sizeof(T) * (count > 0 ? count : 1));
    if (err == cudaSuccess) ptr[n++] = q;
    return (T*)q;
  }
  ~CgBuffers() {
    for (int i = 0; i < n; ++i) cudaFree(ptr[i]);
  }
};

int cg_cuda_fail(const char* who, cudaError_t err) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", who, cudaGetErrorString(err));
  set_error_message(msg);
  return err == cudaErrorMemoryAllocation ? (int)NBM_ERR_OOM : (int)NBM_ERR_CUDA;
}

int cg_report(const char* who, bool converged, int it, double rnorm, double bnorm, double rtol,
              int* iters_out, double* relres_out) {
  char msg[256];
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  if (!(rnorm == rnorm)) {
    snprintf(msg, sizeof(msg), "%s: residual is not finite", who);
    set_error_message(msg);
    return NBM_ERR_NONFINITE;
  }
  if (!converged) {
    snprintf(msg, sizeof(msg), "%s: %d iterations, relative residual %.3e > %.3e", who, it,
             bnorm > 0 ? rnorm / bnorm : 0.0, rtol);
    set_error_message(msg);
    return NBM_ERR_NOT_CONVERGED;
  }
  return NBM_OK;
}

}  // namespace
}  // namespace nbm

using namespace nbm;

namespace nbm {
namespace {

constexpr double kInnerTol = 1e-5;  // relative residual target of one FP32 inner solve
constexpr int kCheckEvery = 10;     // inner iterations between host convergence checks
constexpr int kMaxStall = 3;        // outer steps in a row that gain less than 10 %
constexpr int kMaxPasses = 10;      // solves with a lagged jump
constexpr double kJumpTol = 1e-6;   // max |J_new - J| <= kJumpTol max(1, max |J|)

struct JumpInfo {
  int passes = 0;
  double dj = 0.0;
  int fell_back = 0;
};
thread_local JumpInfo g_jump_info;

// Device state of one grid solve (either solver) and its outer jump loop.
struct GridSolve {
  const char* who;
  CgSetup S;
  cudaStream_t st;
  CgBuffers B;
  bool refined;
  // diag: D = diag A; wx, wy, wz, b, x, r: the Jacobi-scaled system's face
  // weights, right-hand side, iterate x^ = D^1/2 x and residual
  double *diag, *wx, *wy, *wz, *b, *x, *r, *J = nullptr, *part, *sc;
  int* ticket = nullptr;  // last-block counter of the folded reductions
  double *pv = nullptr, *Ap = nullptr;                        // FP64 CG
  float *d32 = nullptr, *idg32 = nullptr, *wx32 = nullptr, *wy32 = nullptr, *wz32 = nullptr,
        *r32 = nullptr, *e32 = nullptr, *p32 = nullptr, *Ap32 = nullptr;  // refined
  double host_sc[16];
  double rnorm = 0.0, bnorm = 0.0;
  int iters = 0;

  int* tk() const { return S.fold ? ticket : nullptr; }
  // the separate reduction of a launch's partials when they are not folded
  void reduce(int nparts, int nvec, int slot, int post) {
    if (!S.fold) launch_pdl(k_reduce_parts, dim3(1),
                            dim3(kB), 0, st, part, nparts, nvec, sc, slot, post);
  }

  cudaError_t read_sc() {
    cudaError_t e = cudaMemcpyAsync(host_sc, sc, sizeof(host_sc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }

  // r^ = b^ - A^ x^ for the current x^; sc cleared, then sc[8] = ||r||^2,
  // sc[9] = ||b||^2 and (POST_NORM) sc[6] = ||r||, sc[7] = 1 / ||r||
  void defect() {
    const Grid& G = S.G;
    cudaMemsetAsync(sc, 0, sizeof(double) * 16, st);
    launch_pdl(k_spmv_dot<double, true>, dim3(S.sgrid),
               dim3(S.sblock), 0, st, G, S.kz, nullptr, wx, wy, wz, x, r, part, sc, POST_SKIP,
               nullptr);
    launch_pdl(k_defect, dim3(S.nu), dim3(kB), 0, st, G, diag, b, r, part, sc, tk());
    reduce(S.nu, 2, 8, POST_NORM);
  }

  // FP64 CG on the Jacobi-scaled system (Jacobi PCG on A) from the current x^;
  // stops at ||r|| <= rtol ||b|| in the unscaled norm.  0,
  // NBM_ERR_NOT_CONVERGED or NONFINITE, or -1 for a CUDA error (message in `e`).
  int solve_fp64(double rtol, int max_iter, cudaError_t& e) {
    const Grid& G = S.G;
    defect();
    cudaMemsetAsync(pv, 0, sizeof(double) * G.m, st);
    cudaMemsetAsync(Ap, 0, sizeof(double) * G.m, st);
    // rz = r^.r^, rr = ||r||^2 (an update with alpha = sc[2] = 0), p = r^
    launch_pdl(k_update<double, true>, dim3(S.nu), dim3(kB), 0, st, G, sc, diag, pv, Ap, x, r, part,
               tk());
    reduce(S.nu, 2, 3, POST_BETA);
    launch_pdl(k_pupdate<double, true>, dim3(S.nu), dim3(kB), 0, st, G, sc, 1, nullptr, r, pv);
    if ((e = read_sc()) != cudaSuccess) return -1;
    bnorm = sqrt(host_sc[9]);
    rnorm = sqrt(host_sc[4]);
    int it = 0;
    bool converged = rnorm <= rtol * bnorm;
    while (!converged && it < max_iter && rnorm == rnorm) {
      launch_pdl(k_spmv_dot<double, true>, dim3(S.sgrid), dim3(S.sblock), 0, st, G, S.kz, nullptr,
                 wx, wy, wz, pv, Ap, part, sc, POST_ALPHA, tk());
      reduce(S.nsp, 1, 1, POST_ALPHA);
      launch_pdl(k_update<double, true>, dim3(S.nu), dim3(kB), 0, st, G, sc, diag, pv, Ap, x, r,
                 part, tk());
      reduce(S.nu, 2, 3, POST_BETA);
      launch_pdl(k_pupdate<double, true>, dim3(S.nu), dim3(kB), 0, st, G, sc, 0, nullptr, r, pv);
      ++it;
      if (it % kCheckEvery == 0 || it == max_iter) {
        if ((e = read_sc()) != cudaSuccess) return -1;
        rnorm = sqrt(host_sc[4]);
        converged = rnorm <= rtol * bnorm;
      }
    }
    iters += it;
    if (!(rnorm == rnorm)) return NBM_ERR_NONFINITE;
    return converged ? NBM_OK : NBM_ERR_NOT_CONVERGED;
  }

  // FP64 residuals of the scaled system, FP32 inner Jacobi-PCG corrections on
  // the unscaled operator, from the current x^
  int solve_refined(double rtol, int max_iter, cudaError_t& e) {
    const Grid& G = S.G;
    defect();
    if ((e = read_sc()) != cudaSuccess) return -1;
    bnorm = sqrt(host_sc[9]);
    rnorm = sqrt(host_sc[8]);
    int it = 0, stall = 0;
    bool converged = rnorm <= rtol * bnorm;
    while (!converged && it < max_iter && rnorm == rnorm && stall < kMaxStall) {
      // inner FP32 Jacobi PCG on A e = D^1/2 r^ / ||r|| (initial residual norm
      // 1), stopped at kInnerTol or where the outer target needs no more
      double tau = 0.5 * rtol * bnorm / rnorm;
      tau = tau < kInnerTol ? kInnerTol : tau > 0.5 ? 0.5 : tau;
      launch_pdl(k_inner_init, dim3(S.nu), dim3(kB), 0, st, G, sc, r, d32, idg32, r32, e32, p32,
                 part, tk());
      reduce(S.nu, 2, 3, POST_BETA);
      for (int inner = 1; it < max_iter; ++inner) {
        launch_pdl(k_spmv_dot<float, false>, dim3(S.sgrid), dim3(S.sblock), 0, st, G, S.kz, d32,
                   wx32, wy32, wz32, p32, Ap32, part, sc, POST_ALPHA, tk());
        reduce(S.nsp, 1, 1, POST_ALPHA);
        launch_pdl(k_update<float, false>, dim3(S.nu), dim3(kB), 0, st, G, sc, idg32, p32, Ap32,
                   e32, r32, part, tk());
        reduce(S.nu, 2, 3, POST_BETA);
        launch_pdl(k_pupdate<float, false>, dim3(S.nu), dim3(kB), 0, st, G, sc, 0, idg32, r32, p32);
        ++it;
        if (inner % kCheckEvery == 0 || it == max_iter) {
          if ((e = read_sc()) != cudaSuccess) return -1;
          const double rin = sqrt(host_sc[4]);
          if (!(rin == rin) || rin <= tau) break;
        }
      }
      // x^ += ||r|| D^1/2 e in FP64, then the FP64 residual r^ = b^ - A^ x^
      launch_pdl(k_correct, dim3(S.nu), dim3(kB), 0, st, G, sc, d32, e32, x);
      defect();
      if ((e = read_sc()) != cudaSuccess) return -1;
      const double rnew = sqrt(host_sc[8]);
      stall = rnew > 0.9 * rnorm ? stall + 1 : 0;
      rnorm = rnew;
      converged = rnorm <= rtol * bnorm;
    }
    iters += it;
    if (!(rnorm == rnorm)) return NBM_ERR_NONFINITE;
    return converged ? NBM_OK : NBM_ERR_NOT_CONVERGED;
  }

  int solve(double rtol, int max_iter, cudaError_t& e) {
    return refined ? solve_refined(rtol, max_iter, e) : solve_fp64(rtol, max_iter, e);
  }

  // the rows of the current jumps, then the scaled system
  void rows() {
    launch_pdl(k_grid_rows, dim3(S.nb), dim3(kB), 0, st, S.P, S.G, J, diag, wx, wy, wz, b);
    launch_pdl(k_scale_rows, dim3(S.nu), dim3(kB), 0, st, S.G, diag, wx, wy, wz, b);
  }

  // J from the current x (lag 1) or first order (lag 0); sc[12] = max |dJ|,
  // sc[13] = max |J|
  void jumps(int lag) {
    launch_pdl(k_node_jump, dim3(S.nu), dim3(kB), 0, st, S.P, S.G, lag, x, diag, J, part);
    launch_pdl(k_reduce_max2, dim3(1), dim3(256), 0, st, part, S.nu, sc, 12);
  }
};

int grid_solve(nbm_problem* p, int n, double rtol, int max_iter, double* u_out, int* iters_out,
               double* relres_out, nbm_stream_t stream, bool refined) {
  GridSolve W;
  W.who = refined ? "refined grid solve" : "grid CG";
  W.refined = refined;
  g_jump_info = JumpInfo();
  if (int rc = cg_setup(p, n, rtol, max_iter, u_out, W.who, W.S)) return rc;
  const Grid& G = W.S.G;
  const int mode = problem_desc(p).grid_jump;
  W.st = (cudaStream_t)stream;
  CgBuffers& B = W.B;
  W.diag = B.get<double>(G.m);
  W.wx = B.get<double>(G.m);
  W.wy = B.get<double>(G.m);
  W.wz = B.get<double>(G.m);
  W.b = B.get<double>(G.m);
  W.x = B.get<double>(G.m);
  W.r = B.get<double>(G.m);
  if (mode != NBM_JUMP_EXACT) W.J = B.get<double>(G.m);
  if (refined) {
    W.d32 = B.get<float>(G.m);
    W.idg32 = B.get<float>(G.m);
    W.wx32 = B.get<float>(G.m);
    W.wy32 = B.get<float>(G.m);
    W.wz32 = B.get<float>(G.m);
    W.r32 = B.get<float>(G.m);
    W.e32 = B.get<float>(G.m);
    W.p32 = B.get<float>(G.m);
    W.Ap32 = B.get<float>(G.m);
  } else {
    W.pv = B.get<double>(G.m);
    W.Ap = B.get<double>(G.m);
  }
  W.part = B.get<double>(kMaxVec * (size_t)(W.S.nu > W.S.nsp ? W.S.nu : W.S.nsp));
  W.sc = B.get<double>(16);
  W.ticket = B.get<int>(1);
  if (B.err != cudaSuccess) return cg_cuda_fail(W.who, B.err);

  cudaStream_t st = W.st;
  cudaMemsetAsync(W.ticket, 0, sizeof(int), st);
  cudaMemsetAsync(W.x, 0, sizeof(double) * G.m, st);
  if (W.J) {
    cudaMemsetAsync(W.J, 0, sizeof(double) * G.m, st);
    W.jumps(0);
  }
  W.rows();
  if (refined)  // the operator is the same for every pass: round it once
    launch_pdl(k_to_f32, dim3(W.S.nu),
               dim3(kB), 0, st, G, W.diag, W.wx, W.wy, W.wz, W.d32, W.idg32, W.wx32, W.wy32,
               W.wz32);
  cudaError_t e = cudaSuccess;
  int status = W.solve(rtol, max_iter, e);
  JumpInfo info;
  info.passes = 1;
  if (mode == NBM_JUMP_EXTRAP && status == NBM_OK) {
    bool converged = false;
    while (info.passes < kMaxPasses && !converged) {
      W.jumps(1);
      if ((e = W.read_sc()) != cudaSuccess) {
        status = -1;
        break;
      }
      info.dj = W.host_sc[12];
      const double jmax = W.host_sc[13];
      W.rows();
      ++info.passes;
      status = W.solve(rtol, max_iter, e);
      if (status != NBM_OK) break;
      converged = info.dj <= kJumpTol * (jmax > 1.0 ? jmax : 1.0);
    }
    if (status == NBM_OK && !converged) {  // stalled: the first-order jump instead
      W.jumps(0);
      W.rows();
      status = W.solve(rtol, max_iter, e);
      info.fell_back = 1;
    }
  }
  if (status < 0) return cg_cuda_fail(W.who, e);
  launch_pdl(k_write_nodes, dim3((int)((W.S.nodes + kB - 1) / kB)),
             dim3(kB), 0, st, W.S.P, G, W.x, W.diag, u_out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cg_cuda_fail(W.who, e);
  g_jump_info = info;
  const bool converged = status == NBM_OK;
  return cg_report(W.who, converged, W.iters, W.rnorm, W.bnorm, rtol, iters_out, relres_out);
}

}  // namespace
}  // namespace nbm

extern "C" int nbm_grid_cg_solve(nbm_problem* p, int n, double rtol, int max_iter, double* u_out,
                                 int* iters_out, double* relres_out, nbm_stream_t stream) {
  return grid_solve(p, n, rtol, max_iter, u_out, iters_out, relres_out, stream, false);
}

extern "C" int nbm_grid_solve_refined(nbm_problem* p, int n, double rtol, int max_iter,
                                      double* u_out, int* iters_out, double* relres_out,
                                      nbm_stream_t stream) {
  return grid_solve(p, n, rtol, max_iter, u_out, iters_out, relres_out, stream, true);
}

extern "C" int nbm_grid_last_jump_info(int* passes_out, double* max_dj_out, int* fell_back_out) {
  if (passes_out) *passes_out = g_jump_info.passes;
  if (max_dj_out) *max_dj_out = g_jump_info.dj;
  if (fell_back_out) *fell_back_out = g_jump_info.fell_back;
  return NBM_OK;
}

extern "C" int nbm_grid_node_jump(nbm_problem* p, int n, int mode, const double* u,
                                  double* jump_out, nbm_stream_t stream) {
  if (!p || !jump_out || (mode == NBM_JUMP_EXTRAP && !u)) {
    set_error_message("NULL argument");
    return NBM_ERR_INVALID_ARG;
  }
  if (mode != NBM_JUMP_EXACT && mode != NBM_JUMP_EXTRAP && mode != NBM_JUMP_FIRST_ORDER) {
    set_error_message("unknown grid_jump mode");
    return NBM_ERR_INVALID_ARG;
  }
  if (int rc = check_aligned(u, 8, "u")) return rc;
  CgSetup S;
  if (int rc = cg_setup(p, n, 1.0, 0, jump_out, "node jump", S)) return rc;
  const int64_t blocks = (S.nodes + kB - 1) / kB, cap = 8 * (int64_t)problem_num_sms(p);
  launch_pdl(k_node_jump_all, dim3((int)(blocks < cap ? blocks : cap)), dim3(kB), 0,
             (cudaStream_t)stream, S.P, S.G, mode, u, jump_out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NBM_OK : cg_cuda_fail("node jump", e);
}
