// nbm_cg.cu -- the plain mesh-based method the NBM is bootstrapped from
// (arXiv 2210.14907, Sec. 1 and Sec. 3): the same finite-volume balance row on
// the nodes of a grid of spacing h = 2/n, one unknown per interior node, solved
// by Jacobi-preconditioned conjugate gradients in FP64.  HBM-bound: every
// iteration streams the operator (diagonal + three face weights per node) and
// five vectors.
//
// Row of interior node p (cell p + [-h/2, h/2]^3, fractions as in nbm_geom.cuh):
//   sum_f w_f (u_p - u_q) + h^2 sum_s V^s k^s u_p = -known_p,
//   w_f = sum_s A^s_f mu^s  (shared by the two cells of the face: A is SPD),
// where the value of network/side s at a node q of the other side is u_q plus
// the jump u+ - u- of the manufactured pair at q (the "exact jump" extension);
// all such terms, the source, the interface flux h S beta and the Dirichlet
// data move to the right-hand side.
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

__device__ inline void node_xyz(const Grid& G, int64_t r, int& i, int& j, int& k, double x[3]) {
  i = 1 + (int)(r % G.m1);
  j = 1 + (int)((r / G.m1) % G.m1);
  k = 1 + (int)(r / ((int64_t)G.m1 * G.m1));
  x[0] = -1.0 + i * G.h;
  x[1] = -1.0 + j * G.h;
  x[2] = -1.0 + k * G.h;
}

__device__ inline int phase_d(const ProbDev& P, const double x[3]) {
  return phi_d(P, x[0], x[1], x[2]) <= 0.0 ? 0 : 1;
}

// jump correction of side s at node x of side sx: U^s(x) = u_x + corr
__device__ inline void jump_corr(const ProbDev& P, const double x[3], int sx, double c[2]) {
  const double jmp = alpha_d(P, x);
  c[0] = sx == 1 ? -jmp : 0.0;
  c[1] = sx == 0 ? jmp : 0.0;
}

__global__ void __launch_bounds__(kB) k_grid_rows(ProbDev P, Grid G, double* diag, double* wx,
                                                  double* wy, double* wz, double* rhs,
                                                  double* inv_diag) {
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
  jump_corr(P, p, sp, cp);
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
    const double q[3] = {-1.0 + nb[0] * h, -1.0 + nb[1] * h, -1.0 + nb[2] * h};
    const bool bnd = nb[ax] == 0 || nb[ax] == G.n;
    double cq[2] = {0.0, 0.0};
    if (!bnd) jump_corr(P, q, phase_d(P, q), cq);
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
  inv_diag[r] = 1.0 / dg;  // the Jacobi preconditioner, applied by multiplication
  wx[r] = wplus[0];
  wy[r] = wplus[1];
  wz[r] = wplus[2];
  rhs[r] = -known;
}

// y = A v on the interior nodes; block partial of v . y.  Launched on a 3-D
// grid (x: runs of 256 nodes of one row, y: row j, z: plane k), so node
// indices need no integer division.
__global__ void __launch_bounds__(kB) k_spmv_dot(Grid G, const double* __restrict__ diag,
                                                 const double* __restrict__ wx,
                                                 const double* __restrict__ wy,
                                                 const double* __restrict__ wz,
                                                 const double* __restrict__ v, double* y,
                                                 double* part) {
  __shared__ double red[kB / 32];
  const int i = blockIdx.x * kB + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  const int64_t s1 = G.m1, s2 = (int64_t)G.m1 * G.m1;
  double d = 0.0;
  if (i < G.m1) {
    const int64_t r = i + s1 * j + s2 * k;
    const double vr = v[r];
    double acc = diag[r] * vr;
    if (i + 1 < G.m1) acc -= wx[r] * v[r + 1];
    if (i > 0) acc -= wx[r - 1] * v[r - 1];
    if (j + 1 < G.m1) acc -= wy[r] * v[r + s1];
    if (j > 0) acc -= wy[r - s1] * v[r - s1];
    if (k + 1 < G.m1) acc -= wz[r] * v[r + s2];
    if (k > 0) acc -= wz[r - s2] * v[r - s2];
    y[r] = acc;
    d = vr * acc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kB / 32; ++w) s += red[w];
    part[blockIdx.x + gridDim.x * ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z)] = s;
  }
}

// scalars[]: 0 rz, 1 pAp, 2 alpha, 3 rz_new, 4 rr, 5 beta
__global__ void k_reduce_parts(const double* __restrict__ part, int nparts, int nvec,
                               double* out) {
  __shared__ double red[2][256];
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nparts; b += 256) {
    s0 += part[b];
    if (nvec > 1) s1 += part[nparts + b];
  }
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = red[0][0];
    if (nvec > 1) out[1] = red[1][0];
  }
}

__global__ void k_alpha(double* sc) { sc[2] = sc[0] / sc[1]; }

__global__ void k_beta(double* sc) {
  sc[5] = sc[3] / sc[0];
  sc[0] = sc[3];
}

// x += alpha p; r -= alpha Ap; partials of r.z and r.r (z = r / diag)
__global__ void __launch_bounds__(kB) k_update(Grid G, const double* __restrict__ sc,
                                               const double* __restrict__ inv_diag,
                                               const double* __restrict__ p,
                                               const double* __restrict__ Ap, double* x, double* r,
                                               double* part, int nparts) {
  __shared__ double red[2][kB / 32];
  const int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (i < G.m) {
    const double a = sc[2];
    x[i] += a * p[i];
    const double ri = r[i] - a * Ap[i];
    r[i] = ri;
    rz = ri * ri * inv_diag[i];
    rr = ri * ri;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz += __shfl_xor_sync(0xffffffffu, rz, o);
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rz;
    red[1][threadIdx.x >> 5] = rr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kB / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[blockIdx.x] = s0;
    part[nparts + blockIdx.x] = s1;
  }
}

// p = r / diag + beta p   (beta = 0: p = z for the first direction)
__global__ void __launch_bounds__(kB) k_pupdate(Grid G, const double* __restrict__ sc, int first,
                                                const double* __restrict__ inv_diag,
                                                const double* __restrict__ r, double* p) {
  const int64_t i = (int64_t)blockIdx.x * kB + threadIdx.x;
  if (i >= G.m) return;
  const double z = r[i] * inv_diag[i];
  p[i] = first ? z : z + sc[5] * p[i];
}

__global__ void __launch_bounds__(kB) k_write_nodes(ProbDev P, Grid G, const double* __restrict__ x,
                                                    double* u) {
  const int64_t N1 = G.n + 1;
  const int64_t id = (int64_t)blockIdx.x * kB + threadIdx.x;
  if (id >= N1 * N1 * N1) return;
  const int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
  if (i == 0 || j == 0 || k == 0 || i == G.n || j == G.n || k == G.n) {
    u[id] = dirichlet_g<double>(P, -1.0 + i * G.h, -1.0 + j * G.h, -1.0 + k * G.h);
  } else {
    u[id] = x[(i - 1) + (int64_t)G.m1 * ((j - 1) + (int64_t)G.m1 * (k - 1))];
  }
}

}  // namespace
}  // namespace nbm

using namespace nbm;

extern "C" int nbm_grid_cg_solve(nbm_problem* p, int n, double rtol, int max_iter, double* u_out,
                                 int* iters_out, double* relres_out, nbm_stream_t stream) {
  char msg[256];
  if (!p || !u_out) {
    set_error_message("NULL argument");
    return NBM_ERR_INVALID_ARG;
  }
  if (int rc = check_aligned(u_out, 8, "u_out")) return rc;
  if (n < 2 || n > 2048 || !(rtol > 0.0) || max_iter < 0) {
    snprintf(msg, sizeof(msg), "grid CG needs 2 <= n <= 2048, rtol > 0, max_iter >= 0 (n=%d)", n);
    set_error_message(msg);
    return NBM_ERR_INVALID_ARG;
  }
  nbm_problem_desc d = problem_desc(p);
  d.h = 2.0 / n;
  ProbDev P;
  make_prob_dev(d, P);
  if (int rc = attach_level_set(p, P)) return rc;
  Grid G;
  G.n = n;
  G.m1 = n - 1;
  G.m = (int64_t)G.m1 * G.m1 * G.m1;
  G.h = 2.0 / n;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((G.m + kB - 1) / kB);
  const int64_t nodes = (int64_t)(n + 1) * (n + 1) * (n + 1);
  double *diag = nullptr, *wx = nullptr, *wy = nullptr, *wz = nullptr, *r = nullptr, *x = nullptr,
         *pv = nullptr, *Ap = nullptr, *idg = nullptr, *part = nullptr, *sc = nullptr;
  double** bufs[] = {&diag, &wx, &wy, &wz, &r, &x, &pv, &Ap, &idg};
  const dim3 sgrid((unsigned)((G.m1 + kB - 1) / kB), (unsigned)G.m1, (unsigned)G.m1);
  const int nsp = (int)(sgrid.x * sgrid.y * sgrid.z);  // SpMV partials
  cudaError_t e = cudaSuccess;
  for (double** b : bufs)
    if (e == cudaSuccess) e = cudaMalloc((void**)b, sizeof(double) * (size_t)(G.m > 0 ? G.m : 1));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&part, sizeof(double) * 2 * (size_t)(nb > nsp ? nb : nsp));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sc, sizeof(double) * 8);
  auto cleanup = [&]() {
    for (double** b : bufs)
      if (*b) cudaFree(*b);
    if (part) cudaFree(part);
    if (sc) cudaFree(sc);
  };
  auto cuda_fail = [&](cudaError_t err) {
    snprintf(msg, sizeof(msg), "grid CG: %s", cudaGetErrorString(err));
    set_error_message(msg);
    cleanup();
    return err == cudaErrorMemoryAllocation ? (int)NBM_ERR_OOM : (int)NBM_ERR_CUDA;
  };
  if (e != cudaSuccess) return cuda_fail(e);

  k_grid_rows<<<nb, kB, 0, st>>>(P, G, diag, wx, wy, wz, r, idg);
  cudaMemsetAsync(x, 0, sizeof(double) * G.m, st);
  cudaMemsetAsync(pv, 0, sizeof(double) * G.m, st);
  cudaMemsetAsync(Ap, 0, sizeof(double) * G.m, st);
  cudaMemsetAsync(sc, 0, sizeof(double) * 8, st);
  // r = b: rz = r.(r/diag), rr = r.r (an update with alpha = 0)
  k_update<<<nb, kB, 0, st>>>(G, sc, idg, pv, Ap, x, r, part, nb);
  k_reduce_parts<<<1, 256, 0, st>>>(part, nb, 2, sc + 3);
  k_beta<<<1, 1, 0, st>>>(sc);
  k_pupdate<<<nb, kB, 0, st>>>(G, sc, 1, idg, r, pv);
  double host_sc[8];
  e = cudaMemcpyAsync(host_sc, sc, sizeof(host_sc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  const double bnorm = sqrt(host_sc[4]);
  int it = 0;
  double rnorm = bnorm;
  bool converged = bnorm == 0.0;
  while (!converged && it < max_iter) {
    k_spmv_dot<<<sgrid, kB, 0, st>>>(G, diag, wx, wy, wz, pv, Ap, part);
    k_reduce_parts<<<1, 256, 0, st>>>(part, nsp, 1, sc + 1);
    k_alpha<<<1, 1, 0, st>>>(sc);
    k_update<<<nb, kB, 0, st>>>(G, sc, idg, pv, Ap, x, r, part, nb);
    k_reduce_parts<<<1, 256, 0, st>>>(part, nb, 2, sc + 3);
    k_beta<<<1, 1, 0, st>>>(sc);
    k_pupdate<<<nb, kB, 0, st>>>(G, sc, 0, idg, r, pv);
    ++it;
    if (it % 10 == 0 || it == max_iter) {
      e = cudaMemcpyAsync(host_sc, sc, sizeof(host_sc), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e);
      rnorm = sqrt(host_sc[4]);
      if (!(rnorm == rnorm)) break;  // NaN: stop, report below
      converged = rnorm <= rtol * bnorm;
    }
  }
  k_write_nodes<<<(int)((nodes + kB - 1) / kB), kB, 0, st>>>(P, G, x, u_out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  cleanup();
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  if (!(rnorm == rnorm)) {
    set_error_message("grid CG: residual is not finite");
    return NBM_ERR_NONFINITE;
  }
  if (!converged) {
    snprintf(msg, sizeof(msg), "grid CG: %d iterations, relative residual %.3e > %.3e", it,
             bnorm > 0 ? rnorm / bnorm : 0.0, rtol);
    set_error_message(msg);
    return NBM_ERR_NOT_CONVERGED;
  }
  return NBM_OK;
}
