/*
 * nbm_oracle.h -- plain FP64 CPU oracle of the Neural Bootstrapping Method
 * (NBM, arXiv 2210.14907) collocation-residual training step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library under
 * paper_2210_14907_gb300/, and neither includes the other.
 *
 * Everything here is written to be read against the paper:
 *   Sec. 2    interface problem  k u - div(mu grad u) = f,  [u]=alpha,
 *             [mu d_n u]=beta, Dirichlet data on the cube [-1,1]^3.
 *   Sec. 3    NBM: implicit compute cell at each collocation point, cell /
 *             interface crossings from a level set, two networks (one per
 *             side), point residual r_p = ||M^-1 A u - M^-1 b||, losses
 *             aggregated over points, Adam on the network parameters.
 *   Fig. 2    (caption) one point per kernel thread, local preconditioner.
 * The discretization equation is missing from the paper's text (Sec. 3 breaks
 * off where the loss would be written out); the finite-volume reading implemented
 * here is documented per function.
 *
 * Parity status: every function has a pin in tests/test_oracle_pins.py,
 * tests/test_oracle_conventions.py or tests/test_grid_identities.py.  No pin
 * compares the grid rows with the cited Bochkov-Gibou scheme (not available);
 * their order is pinned instead.  tests/oracle_mutants.py plants mistakes in
 * copies of this file and checks that the pins catch them.
 */
#ifndef NBM_ORACLE_H
#define NBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  NBO_GEOM_SPHERE = 1,    /* phi = |x| - r0                                     */
  NBO_GEOM_FLOWER = 2,    /* phi = r - r0 - amp sin(lt*theta) cos(lp*psi)       */
  NBO_GEOM_ALL_PLUS = 3,  /* phi = +1 everywhere: no interface, all of Omega+  */
  NBO_GEOM_ALL_MINUS = 4, /* phi = -1 everywhere: no interface, all of Omega-  */
  NBO_GEOM_GRID = 5       /* phi = trilinear interpolant of the node values
                             phi_grid on the (phi_n+1)^3 grid of [-1,1]^3
                             (Sec. 3: a coarse mesh holds the level set)      */
};

typedef struct {
  int32_t geometry;
  int32_t n_hidden;   /* tanh layers: 3->H, then (n_hidden-1) times H->H   */
  int32_t width;      /* H                                                   */
  int32_t pad0;
  double r0, amp, lobes_theta, lobes_psi;
  double mu_minus, mu_plus, k_minus, k_plus;
  double h;           /* stencil spacing of the implicit cell               */
  double lambda_jump; /* weight of the value-jump row in r_p^2               */
  int32_t solution;   /* manufactured pair: 0 the benchmark pair with constant
                         mu_minus/mu_plus; 1 the pair of Sec. 4.1 with the
                         variable coefficients mu- = y^2 ln(x+2) + 4,
                         mu+ = exp(-z) (mu_minus/mu_plus unused)            */
  int32_t activation; /* hidden-layer activation: 0 tanh, 1 sin            */
  int32_t phi_n;      /* NBO_GEOM_GRID: cells per axis of the level-set mesh */
  int32_t pad1;
  const double* phi_grid; /* NBO_GEOM_GRID: node values, node (i,j,k) at
                             i + (phi_n+1)(j + (phi_n+1)k), x_i = -1 + 2i/phi_n */
} nbo_problem;

/* Per-point terms of the residual (reading of Sec. 3). */
typedef struct {
  double B;          /* h^2-scaled finite-volume balance row               */
  double D;          /* Jacobi preconditioner diag(A)                       */
  double J;          /* value-jump row (0 when has_jump == 0)               */
  double r2;         /* (B/D)^2 + lambda J^2                                */
  int32_t has_jump;
  int32_t cut;
} nbo_point_terms;

typedef struct {
  int32_t cut;       /* 0: all 8 corners on one side; 1: Kuhn split used    */
  int32_t phase;     /* for uncut cells: 0 = Omega-, 1 = Omega+             */
  double V[2];       /* volume fractions [minus, plus]                      */
  double A[2][6];    /* face fractions, face f = 2*axis + (side>0)          */
  double S;          /* interface area / h^2                                */
  double centroid[3];/* area-weighted centroid of the linear interface      */
  double xg[3];      /* centroid projected onto phi = 0 (Newton)            */
} nbo_cell;

/* ---- counter-based generator (Salmon et al., SC'11, Philox4x32-10) ---- */
void nbo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* ---- geometry and manufactured problem (Sec. 2) ---- */
double nbo_phi(const nbo_problem* pr, const double x[3]);
void nbo_grad_phi(const nbo_problem* pr, const double x[3], double g[3]);
int nbo_phase(const nbo_problem* pr, const double x[3]); /* 0 = minus (phi<=0), 1 = plus */
double nbo_exact_u(const nbo_problem* pr, int s, const double x[3]);
double nbo_mu(const nbo_problem* pr, int s, const double x[3]); /* diffusion coefficient mu^s(x) */
void nbo_exact_grad_u(const nbo_problem* pr, int s, const double x[3], double g[3]);
double nbo_rhs_f(const nbo_problem* pr, int s, const double x[3]);
double nbo_alpha(const nbo_problem* pr, const double x[3]);
double nbo_beta(const nbo_problem* pr, const double x[3]);
double nbo_dirichlet_g(const nbo_problem* pr, const double x[3]);

/* ---- implicit compute cell (Fig. 2: cell/interface crossings) ---- */
void nbo_cell_geometry(const nbo_problem* pr, const double p[3], double h, nbo_cell* out);
double nbo_tri_fraction(double f0, double f1, double f2);
double nbo_tet_fraction(double f0, double f1, double f2, double f3);

/* ---- networks (Sec. 3: one network per side of the interface) ---- */
int64_t nbo_params_per_net(const nbo_problem* pr);
double nbo_mlp_eval(const nbo_problem* pr, const double* theta_net, const double x[3]);

/* ---- sampling of collocation points ---- */
void nbo_sample_points(const nbo_problem* pr, uint64_t seed, int64_t step, int64_t n,
                       int64_t n_band, double* pts /* n*3, AoS */);

/* ---- residual, loss, gradient ---- */
/* mode 0: U^s from the networks; mode 1: U^s from the exact manufactured u^s. */
void nbo_point_terms_eval(const nbo_problem* pr, const double* theta, const double p[3],
                          int mode, nbo_point_terms* out);
double nbo_loss(const nbo_problem* pr, const double* theta, const double* pts, int64_t n,
                double* r2_out /* n or NULL */, int n_threads);
double nbo_loss_grad(const nbo_problem* pr, const double* theta, const double* pts, int64_t n,
                     double* grad /* 2*P_net */, int n_threads);
void nbo_adam_step(double* theta, double* m, double* v, const double* grad, int64_t n,
                   int64_t t, double lr, double beta1, double beta2, double eps);
/* Full training loop with its own sampler; loss_hist[k] = loss before update k. */
void nbo_train(const nbo_problem* pr, double* theta, double* m, double* v, int64_t step0,
               int n_steps, int64_t batch, int64_t n_band, double lr, double beta1, double beta2,
               double eps, uint64_t seed, double* loss_hist, int n_threads);

/* Threads a call with n_threads = 0 uses (OpenMP's default team size). */
int nbo_default_threads(void);

/* ---- grid evaluation of the trained pair and the grid scheme (judge) ---- */
void nbo_eval_grid(const nbo_problem* pr, const double* theta, int n, double* u_out /*(n+1)^3*/,
                   int n_threads);
/* Dense assembly of the grid system on the (n-1)^3 interior nodes (small n only). */
int nbo_grid_assemble_dense(const nbo_problem* pr, int n, double* A /*m*m*/, double* b /*m*/);
int nbo_grid_cg_solve(const nbo_problem* pr, int n, double rtol, int max_iter,
                      double* u_out /*(n+1)^3*/, int* iters_out, double* relres_out, int n_threads);
void nbo_grid_error(const nbo_problem* pr, int n, const double* u /*(n+1)^3*/, double* linf,
                    double* rmse);
/* Extrapolated node jump J(x) = alpha(x_G) + d G (use_lag 0: G = beta/mu_big;
 * 1: G with the small-mu side's normal derivative dn_small).  Returns 1 and
 * J = 0 for nodes farther than 3h from Gamma. */
int nbo_jump_extrap(const nbo_problem* pr, const double x[3], double h, int use_lag,
                    double dn_small, double* J, double xg[3], double nrm[3], int* small_side);
/* d_n u_s at xg from node values u by a least-squares linear fit (1: no fit). */
int nbo_fit_dn(const nbo_problem* pr, int n, const double* u /*(n+1)^3*/, int s,
               const double xg[3], const double nrm[3], double* dn);
/* Grid solve with node jump mode 0 exact, 1 extrapolated + lagged fixed point,
 * 2 extrapolated first order.  Returns 0, 1 (CG not converged), 2 (passes out). */
int nbo_grid_solve_jump(const nbo_problem* pr, int n, int jump_mode, double rtol, int max_iter,
                        int max_passes, double jtol, double* u_out, int* iters_out,
                        double* relres_out, int* passes_out, double* dj_out, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
