/*
 * nbm.h -- C ABI of libnbm, a GB300 (sm_103a) implementation of the fused
 * collocation-residual training step of the Neural Bootstrapping Method
 * (NBM; Mistani, Pakravan, Ilango, Choudhry, Gibou, "Neuro-Symbolic Partial
 * Differential Equation Solver", arXiv 2210.14907).
 *
 * The method (Sec. 3 and Fig. 2 of the paper): two networks u^- and u^+,
 * one per side of a level-set interface Gamma, are evaluated at the vertices
 * of an implicit finite-volume cell placed at each random collocation point;
 * the cell's discretization of  k u - div(mu grad u) = f  with the jump
 * conditions [u] = alpha, [mu d_n u] = beta (Sec. 2) gives a locally
 * preconditioned residual r_p = ||M^-1 A u - M^-1 b||; the squared residuals
 * are averaged into the loss, differentiated through the kernels and fed to
 * Adam.
 *
 * Conventions shared by every entry point
 *  - Every call returns an nbm_status; on failure nbm_last_error() returns a
 *    thread-local, human-readable message.  No call aborts the process.
 *  - Array arguments are caller-owned DEVICE pointers unless marked "host".
 *    The library never frees them and never keeps them past the call.
 *    Float arrays must be 4-byte aligned; nothing else is assumed.
 *  - The library owns only the nbm_problem object and the device workspace
 *    it allocates (grown on demand to the largest batch seen); nbm_destroy
 *    frees both.
 *  - Work is enqueued on `stream` in order.  Calls that return a value
 *    through a HOST pointer synchronize `stream` before returning; the others
 *    are asynchronous.
 *  - Parameter vector: FP32, network minus then network plus.  Each network
 *    is W1[H][3], b1[H], then (W_l[H][H], b_l[H]) for l = 2..n_hidden, then
 *    w_out[H], b_out; P = 2 * (4H + (n_hidden-1)(H^2+H) + H + 1).
 *  - Collocation points: FP32, array-of-structs [n][3], inside the open cube
 *    (-1,1)^3.  Passing pts == NULL draws them on the device from the
 *    counter-based Philox4x32-10 stream (seed, step): uniform points on the
 *    lattice -1 + k 2^-22, plus round(band_fraction*n) points within 4h of
 *    Gamma (the last ones of the batch).  Point i of step t is drawn from the
 *    block at counter (i, t mod 2^32, t div 2^32, 0x4E424D31) under the key
 *    (seed mod 2^32, seed div 2^32); a uniform point takes coordinate j from
 *    word j as k = 1 + floor(w_j (2^23 - 1) / 2^32).  A band point takes an
 *    isotropic direction and an offset uniform on (-4h, 4h) from the
 *    interface along it, rounded to the lattice.
 *  - Batch sizes n of nbm_sample_points, nbm_residual, nbm_loss_grad and
 *    nbm_train_steps are 1..2^30; any other n, including an empty batch,
 *    returns NBM_ERR_INVALID_ARG.
 *  - One nbm_problem may be used by one host thread at a time.
 */
#ifndef NBM_H
#define NBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* nbm_stream_t; /* == cudaStream_t; NULL = legacy default stream */

typedef enum {
  NBM_OK = 0,
  NBM_ERR_INVALID_ARG = 1,   /* bad descriptor, size, pointer or unsupported shape     */
  NBM_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed            */
  NBM_ERR_NOT_CONVERGED = 3, /* grid CG hit max_iter before reaching rtol              */
  NBM_ERR_NONFINITE = 4,     /* the loss or the gradient of a step was NaN/Inf         */
  NBM_ERR_OOM = 5,           /* device workspace could not be allocated                */
  NBM_ERR_DEVICE_TIMEOUT = 6 /* a bounded device-side wait gave up (kernel returned)  */
} nbm_status;

typedef enum {
  NBM_GEOM_SPHERE = 1,    /* phi = |x| - r0                                           */
  NBM_GEOM_FLOWER = 2,    /* phi = r - r0 - amp sin(lobes_theta*theta) cos(lobes_psi*psi),
                             theta = polar angle from +z, psi = azimuth                */
  NBM_GEOM_ALL_PLUS = 3,  /* no interface; the whole cube is Omega+                   */
  NBM_GEOM_ALL_MINUS = 4, /* no interface; the whole cube is Omega-                   */
  NBM_GEOM_GRID = 5       /* phi stored on a separate coarse mesh (Sec. 3),
                             trilinearly interpolated; set with nbm_set_level_set before any
                             computation.  No band points (band_fraction must be 0). */
} nbm_geometry;

typedef enum {
  NBM_PREC_FP32 = 0,      /* hidden-layer GEMMs in FP32 FFMA (the plain path)         */
  NBM_PREC_BF16 = 1,      /* hidden-layer GEMMs on tcgen05, BF16 in / FP32 accumulate  */
  NBM_PREC_FP16 = 2       /* hidden-layer GEMMs on tcgen05, FP16 in / FP32 accumulate
                             (grid evaluation only)                                   */
} nbm_precision;

typedef enum {
  NBM_SOL_BENCH = 0,      /* u- = exp(x)cos(y)sin(z), u+ = x^2+y^2+z^2, constant
                             mu_minus/mu_plus and k_minus/k_plus                       */
  NBM_SOL_SEC41 = 1       /* the convergence study of Sec. 4.1: u- = exp(z),
                             u+ = cos(x)sin(y), mu- = y^2 ln(x+2) + 4, mu+ = exp(-z)
                             (mu_minus/mu_plus unused; k_minus/k_plus as given)        */
} nbm_solution;

typedef enum {
  NBM_JUMP_EXACT = 0,       /* the manufactured pair's own u+(x) - u-(x) at the node      */
  NBM_JUMP_EXTRAP = 1,      /* alpha(x_G) + d [d_n u], the small-mu side's d_n u lagged
                               from the previous solve (fixed-point passes, see below)   */
  NBM_JUMP_FIRST_ORDER = 2  /* alpha(x_G) + d beta(x_G) / mu_big: the lag term dropped    */
} nbm_grid_jump;

typedef enum {
  NBM_ACT_TANH = 0,       /* tanh hidden layers (every path)                            */
  NBM_ACT_SIN = 1         /* sine-activated hidden layers (Sec. 4.1 networks): FP32
                             precision and width <= 32 only                            */
} nbm_activation;

/* Problem descriptor (Sec. 2 problem + Sec. 3 NBM settings).  f, alpha, beta
 * and the Dirichlet data g = u+ follow analytically from the manufactured
 * pair; mu enters the rows at the face centres of the implicit cell. */
typedef struct {
  int32_t geometry;       /* nbm_geometry                                             */
  int32_t n_hidden;       /* number of activation layers: 2..4 (2..5 for width <= 32)  */
  int32_t width;          /* H: 64 or 128 (FP32 path), 128 (tcgen05 path), or 1..32
                             (narrow FP32 path, e.g. the 5 x 10 networks of Sec. 4.1)  */
  int32_t precision;      /* nbm_precision of the training/residual path              */
  double r0, amp, lobes_theta, lobes_psi;
  double mu_minus, mu_plus; /* constant diffusion coefficients, > 0                    */
  double k_minus, k_plus;   /* constant reaction coefficients, >= 0                    */
  double h;               /* stencil spacing of the implicit cell, 0 < h <= 0.25      */
  double lambda_jump;     /* weight of the value-jump row in r_p^2 (1 in the paper's reading) */
  double band_fraction;   /* share of sampled points drawn within 4h of Gamma         */
  int32_t fp64_stencil;   /* -1: automatic (on for h <= 2/512, per level), 0: off, 1: on */
  int32_t refine_levels;  /* implicit refinement (Sec. 3, Fig. 2: cells at several resolutions;
                             Sec. 4.2: a base resolution refined three times).  0..3: every
                             collocation point also gets the cells of spacing h/2, ...,
                             h/2^refine_levels; their rows are stacked into r_p, i.e.
                             r_p^2 = sum over the levels of (B/D)^2 + lambda J^2.  Band
                             points stay within 4h of the base spacing. */
  int32_t solution;       /* nbm_solution: manufactured pair and coefficients          */
  int32_t activation;     /* nbm_activation of the hidden layers                       */
  int32_t grid_jump;      /* nbm_grid_jump: value jump carried to the grid solvers' nodes */
  int32_t reserved0;      /* must be 0                                                 */
} nbm_problem_desc;

typedef struct nbm_problem nbm_problem;

/* Thread-local message describing the last failure of this thread. */
const char* nbm_last_error(void);

/* Validates `d` and creates a problem object on the current CUDA device.
 * Returns NBM_ERR_INVALID_ARG for an unsupported descriptor (e.g. a width
 * the chosen precision path does not implement).  *out is NULL on failure. */
int nbm_init_problem(const nbm_problem_desc* d, nbm_problem** out);

/* Frees the problem and its workspace.  Safe on NULL.  The caller must make
 * sure no work of this problem is still running on any stream. */
int nbm_destroy(nbm_problem* p);

/* Level set on a coarse mesh for an NBM_GEOM_GRID problem (Sec. 3): phi is a
 * caller-owned DEVICE array of (n+1)^3 FP64 node values, node (i,j,k) at
 * x = (-1 + 2i/n, -1 + 2j/n, -1 + 2k/n) stored at i + (n+1)(j + (n+1)k); phi is
 * the trilinear interpolant of those values in each mesh cell, Omega- = {phi <= 0}.
 * The values are copied into the problem (asynchronously on `stream`), so the
 * caller may free phi once the stream has passed the copy.  1 <= n <= 1024.
 * Returns NBM_ERR_INVALID_ARG for another geometry or a bad n.  Calling it again
 * replaces the level set; the caller makes sure no work of this problem is
 * still running. */
int nbm_set_level_set(nbm_problem* p, const double* phi, int n, nbm_stream_t stream);

/* Diagnostics for the failure handling of the device code: one warp waits,
 * with the bounded wait that every kernel of the library uses (mbarrier waits
 * that give up after a clock-cycle budget and set a status bit instead of
 * spinning), on a barrier that nothing completes.  Returns
 * NBM_ERR_DEVICE_TIMEOUT once the wait has given up after about budget_cycles
 * clock cycles (1e3..1e10) -- the error a computation reports when one of its
 * device waits runs out -- or NBM_OK if the barrier completed.  No fault, no
 * trap: the context stays usable.  Synchronizes the stream. */
int nbm_selftest_bounded_wait(int64_t budget_cycles, nbm_stream_t stream);

/* Number of FP32 parameters P of the network pair; -1 for a NULL problem. */
int64_t nbm_param_count(const nbm_problem* p);

/* Draws n collocation points (Sec. 3: random points in the domain) from the
 * Philox4x32-10 stream keyed by `seed` at counter `step`, as described under
 * "Collocation points" above; pts_out is a caller-owned DEVICE array [n][3].
 * Returns NBM_ERR_INVALID_ARG for a NULL argument, n outside 1..2^30 or a
 * misaligned pts_out.  Asynchronous. */
int nbm_sample_points(nbm_problem* p, uint64_t seed, int64_t step, int64_t n, float* pts_out,
                      nbm_stream_t stream);

/* Forward pass of the NBM residual (Sec. 3, Fig. 2): for every point, the two
 * networks at the 2d+1 cell vertices (and at the interface point of cut
 * cells), the balance and jump rows, r_p^2 = (B/D)^2 + lambda J^2 (summed
 * over the refinement levels when refine_levels > 0: one pass of the cells of
 * spacing h/2^l per level l, on the same points).
 *   params  [P]            network pair
 *   pts     [n][3] or NULL (NULL: sample with seed/step)
 *   r2_out  [n] or NULL    per-point squared residual
 *   loss_out (host) or NULL: mean of r_p^2 in FP64; synchronizes the stream. */
int nbm_residual(nbm_problem* p, const float* params, const float* pts, int64_t n, uint64_t seed,
                 int64_t step, float* r2_out, double* loss_out, nbm_stream_t stream);

/* Loss and its gradient with respect to all P parameters (Sec. 3: gradients
 * are taken through the NBM kernels themselves), by the
 * hand-written backward kernels.  grad_out [P] is overwritten.
 * loss_out (host) or NULL; a non-NULL loss_out synchronizes the stream. */
int nbm_loss_grad(nbm_problem* p, const float* params, const float* pts, int64_t n, uint64_t seed,
                  int64_t step, float* grad_out, double* loss_out, nbm_stream_t stream);

/* One data-parallel shard of a training step's loss and gradient (Sec. 3: the
 * collocation points of a step are distributed over processors and their
 * locally computed gradient updates are aggregated).  The step's batch has
 * n_total points; this call takes points first .. first+n-1 of it:
 *   pts [n][3] or NULL   the shard's points; NULL draws them on the device as
 *                        points first .. first+n-1 of nbm_sample_points(seed,
 *                        step, n_total) (same counters, same band points)
 *   grad_out [P]         overwritten with (1/n_total) sum over the shard of
 *                        the gradient of r_p^2
 *   loss_out [1]         DEVICE, FP64, 8-byte aligned: (1/n_total) sum over the
 *                        shard of r_p^2
 * Summed over shards that partition [0, n_total) (e.g. by an all-reduce),
 * grad_out and loss_out are the whole batch's gradient and loss, up to the
 * order of FP32 additions; nbm_adam_step then applies the update on every
 * rank.  Fully asynchronous: nothing is read back, so a bounded device wait
 * that gave up is reported by the next call of this problem that returns a
 * loss on the host.
 * Returns NBM_ERR_INVALID_ARG for a NULL or misaligned argument, n or n_total
 * outside 1..2^30, or a shard outside [0, n_total). */
int nbm_loss_grad_shard(nbm_problem* p, const float* params, const float* pts, int64_t n_total,
                        int64_t first, int64_t n, uint64_t seed, int64_t step, float* grad_out,
                        double* loss_out, nbm_stream_t stream);

/* One Adam update (Kingma & Ba: bias-corrected, constant lr, the optimizer of
 * Sec. 3) with a caller-supplied gradient grad [P], e.g. the all-reduced sum
 * of nbm_loss_grad_shard's outputs.  Update t = *step_io + 1; *step_io += 1 on
 * the host.  The arithmetic is that of the update inside nbm_train_steps, so a
 * single shard covering the whole batch followed by this call reproduces
 * nbm_train_steps bitwise.
 *   params, adam_m, adam_v [P]  updated in place
 *   loss  DEVICE FP64 scalar or NULL: when given and not finite, the update
 *         is skipped (parameters, m, v unchanged), as nbm_train_steps skips a
 *         step whose loss is not finite.
 * Asynchronous.  Returns NBM_ERR_INVALID_ARG for a NULL or misaligned argument,
 * *step_io < 0 or bad hyper-parameters (lr > 0, 0 <= beta < 1, eps > 0). */
int nbm_adam_step(nbm_problem* p, float* params, float* adam_m, float* adam_v, const float* grad,
                  int64_t* step_io, float lr, float beta1, float beta2, float eps,
                  const double* loss, nbm_stream_t stream);

/* n_steps fused training steps (sample -> cell geometry -> two-network stencil
 * forward -> residual -> backward -> Adam, Sec. 3).  Step t (1-based, t =
 * *step_io + 1, ...) samples `batch` points at Philox counter t and applies a
 * bias-corrected Adam update (Kingma & Ba) with constant lr.
 *   params, adam_m, adam_v  [P] updated in place (m, v zero for a fresh run)
 *   step_io (host)          in: steps already taken; out: += n_steps
 *   pts [n_steps][batch][3] or NULL: caller-supplied collocation points of
 *                           each step (e.g. points staged from the host);
 *                           NULL draws them on the device as described above
 *   loss_hist [n_steps] or NULL: loss of each step before its update.
 * Asynchronous: step_io is updated on the host immediately. */
int nbm_train_steps(nbm_problem* p, float* params, float* adam_m, float* adam_v, int64_t* step_io,
                    int n_steps, int64_t batch, float lr, float beta1, float beta2, float eps,
                    uint64_t seed, const float* pts, float* loss_hist, nbm_stream_t stream);

/* Evaluates the trained surrogate on the (n+1)^3 nodes -1 + i*2/n of the
 * cube, each node with the network of its side of Gamma (phi <= 0: minus):
 * the inference use of a trained NBM model (Fig. 1 caption: once trained,
 * the networks evaluate a 1024^3-resolution simulation in under a
 * millisecond; Sec. 4.1 measures the errors at grid nodes).
 * Node (i,j,k) is u_out[i + (n+1)(j + (n+1)k)], a caller-owned DEVICE array.
 * `precision` selects the hidden-GEMM type (nbm_precision): NBM_PREC_FP32
 * (CUDA cores; asynchronous), or NBM_PREC_BF16 / NBM_PREC_FP16 (tensor cores;
 * width 128 and 2..4 hidden layers only; these allocate their scratch,
 * synchronize the stream and free it).
 * Returns NBM_ERR_INVALID_ARG for a NULL or misaligned argument, n outside
 * 1..4096 or an unsupported precision, NBM_ERR_OOM if the scratch cannot be
 * allocated, NBM_ERR_DEVICE_TIMEOUT if a bounded device wait gave up. */
int nbm_eval_grid(nbm_problem* p, const float* params, int n, int precision, float* u_out,
                  nbm_stream_t stream);

/* The trained surrogate at n arbitrary points pts [n][3] (FP32, inside the
 * cube), each with the network of its side of the interface; u_out [n]: the
 * mesh-free solution the networks encode everywhere in the domain (Sec. 1
 * and the conclusion: NBM lifts a mesh-based discretization off its grid).
 * Same precision choices, kernels, synchronization and errors as
 * nbm_eval_grid, with 1 <= n <= 2^34 in place of the grid size. */
int nbm_eval_points(nbm_problem* p, const float* params, const float* pts, int64_t n,
                    int precision, float* u_out, nbm_stream_t stream);

/* The plain mesh-based method the NBM is bootstrapped from (Sec. 1 and Sec. 3:
 * the NBM evaluates a conventional finite-volume discretization of the
 * interface problem of Sec. 2 on implicit cells; here the same rows are
 * assembled on the grid of spacing 2/n and solved), one unknown per
 * interior node, solved in FP64 by Jacobi-preconditioned conjugate gradients
 * until ||r|| <= rtol ||b|| or max_iter.  u_out [(n+1)^3] FP64 (boundary
 * nodes = Dirichlet data).  iters_out (summed over the passes below),
 * relres_out (last solve) or NULL.  Synchronizes the stream.
 *   The other side's value at a node x across Gamma is u_x +- J(x), J chosen
 *   by the descriptor's grid_jump:
 *   NBM_JUMP_EXACT: J = u+(x) - u-(x) of the manufactured pair.
 *   NBM_JUMP_FIRST_ORDER / NBM_JUMP_EXTRAP: J = alpha(x_G) + d G, with x_G
 *     the node moved onto phi = 0 by three Newton steps, d = phi/|grad phi|
 *     at the node, n the normal at x_G, G = [d_n u] from the flux jump beta:
 *     G = beta/mu+ - (1 - mu-/mu+) d_n u- if mu- <= mu+, else
 *     G = beta/mu- + (1 - mu+/mu-) d_n u+ (coefficients at x_G).  The first-
 *     order mode drops the d_n term.  NBM_JUMP_EXTRAP takes d_n of the
 *     small-mu side from the previous solve (least-squares linear fit over
 *     that side's interior nodes in the 3x3x3 block around the node nearest
 *     one spacing into that side): pass 1 is the first-order solve, each
 *     later pass refits, rebuilds the right-hand side and re-solves from the
 *     previous solution, until max |J_new - J| <= 1e-6 max(1, max |J|).
 *     After 10 passes without that, it falls back to the first-order jump
 *     (re-solved; see nbm_grid_last_jump_info).  Nodes farther than 3h from
 *     Gamma carry J = 0 (no row weights them).
 * Returns NBM_ERR_NOT_CONVERGED (with u_out filled) if a solve reaches
 * max_iter. */
int nbm_grid_cg_solve(nbm_problem* p, int n, double rtol, int max_iter, double* u_out,
                      int* iters_out, double* relres_out, nbm_stream_t stream);

/* The same grid system as nbm_grid_cg_solve (Sec. 1, Sec. 3), solved to the
 * same FP64 stopping test ||b - A x|| <= rtol ||b|| by mixed-precision
 * iterative refinement: the rows, the solution x and every residual
 * b - A x are FP64; each correction e of A e = r is a Jacobi-preconditioned
 * CG solve in FP32 (operator rounded to FP32) of the normalised residual
 * r / ||r||, stopped at relative residual 1e-5 or where the outer target needs
 * no more, and x += ||r|| e in FP64.  The FP32 iterations move half the bytes
 * of FP64 ones and avoid GB300's narrow FP64 pipe.
 *   Arguments and u_out as nbm_grid_cg_solve; iters_out = FP32 inner
 *   iterations over all corrections (max_iter bounds that total); relres_out =
 *   the final FP64 ||b - A x|| / ||b||.
 *   Returns NBM_ERR_NOT_CONVERGED (u_out filled) at max_iter, or when three
 *   corrections in a row reduce ||b - A x|| by less than 10 % (an operator too
 *   ill-conditioned for FP32 corrections: use nbm_grid_cg_solve).
 * Synchronizes the stream. */
int nbm_grid_solve_refined(nbm_problem* p, int n, double rtol, int max_iter, double* u_out,
                           int* iters_out, double* relres_out, nbm_stream_t stream);

/* The value jump J(x) = u+(x) - u-(x) that the grid scheme above carries to each
 * node x of the (n+1)^3 grid (x fastest), for grid_jump mode `mode`
 * (nbm_grid_jump; not necessarily the descriptor's): with it the plain
 * method's node values u_x extend across Gamma (the other side's value at x is
 * u_x +- J(x)), e.g. to interpolate either side's solution between nodes.
 *   NBM_JUMP_EXACT         u+(x) - u-(x) of the manufactured pair (every node)
 *   NBM_JUMP_FIRST_ORDER   alpha(x_G) + d beta(x_G)/mu_big within 3h of Gamma
 *   NBM_JUMP_EXTRAP        alpha(x_G) + d G with the small-mu side's d_n u
 *                          fitted from the node values u [(n+1)^3] FP64 (e.g.
 *                          the solution of nbm_grid_cg_solve) as in a lagged pass
 * Nodes farther than 3h from Gamma get 0 in the two extrapolated modes (Sec. 3
 * bootstraps the NBM from this scheme; the jump conditions are those of Sec. 2).
 * u may be NULL except for NBM_JUMP_EXTRAP; jump_out [(n+1)^3] FP64 DEVICE.
 * Asynchronous.  Returns NBM_ERR_INVALID_ARG for a NULL or misaligned
 * argument, an unknown mode or n outside 2..2048. */
int nbm_grid_node_jump(nbm_problem* p, int n, int mode, const double* u, double* jump_out,
                       nbm_stream_t stream);

/* Outer-loop record of the calling thread's last nbm_grid_cg_solve or
 * nbm_grid_solve_refined: passes_out = solves with a lagged jump (1 for
 * NBM_JUMP_EXACT and NBM_JUMP_FIRST_ORDER), max_dj_out = max |J_new - J| of
 * the last pass (0 for one pass), fell_back_out = 1 if NBM_JUMP_EXTRAP used
 * its first-order fallback.  Any pointer may be NULL.  Host only. */
int nbm_grid_last_jump_info(int* passes_out, double* max_dj_out, int* fell_back_out);

/* Optional timing of the fused stencil-step kernel (the dominant kernel of a
 * training step).  enable = 1 clears the counters and brackets every later
 * launch of that kernel with CUDA events on its own stream; enable = 0 stops
 * recording, synchronizes, and returns the summed device time (ms) and the
 * number of timed launches through the host pointers (either may be NULL).
 * Up to 65536 launches are recorded; later ones are not timed. */
int nbm_profile(nbm_problem* p, int enable, double* fused_ms_out, int64_t* fused_launches_out);

/* nbm_loss_grad without any device allocation, for callers that cannot call
 * cudaMalloc while they run: a host that owns all device memory through its
 * own pool or arena (a plugin, an inference server), a real-time or embedded
 * host that forbids allocation after start-up, or code that must not
 * synchronize the device, which cudaMalloc and cudaFree may do.  (The paper
 * has no counterpart: this is a deployment variant of the loss-and-gradient
 * call.)
 *   Arguments, results and precision path are those of nbm_loss_grad; the
 *   caller still owns params, pts, grad_out.
 *   Scratch: one static device array of about 12 MB inside libnbm, held on
 *   every GPU that loads the library until the process exits.  Limits:
 *   n <= 16384 points, width <= 128, n_hidden <= 4, refine_levels == 0; the
 *   fused kernels run on at most 16 CTAs.  Other requests return
 *   NBM_ERR_INVALID_ARG.
 *   No cudaMalloc, cudaFree or other allocating call is made.  The first call
 *   on a device looks up the array's device address (cudaGetSymbolAddress,
 *   once per device, with that device current) and keeps it for the life of
 *   the process; after cudaDeviceReset of that device the kept address is
 *   stale, so do not call this entry point again in such a process.
 *   A non-NULL loss_out reads the loss back and synchronizes the stream, as
 *   in nbm_loss_grad; with loss_out == NULL the call only enqueues work.
 *   Every call shares the array and leaves its contents behind (the status
 *   word is cleared at the start of each call); calls whose work overlaps on
 *   the GPU (different streams, host threads or problems) race on it and
 *   must be serialized by the caller. */
int nbm_loss_grad_static(nbm_problem* p, const float* params, const float* pts, int64_t n,
                         uint64_t seed, int64_t step, float* grad_out, double* loss_out,
                         nbm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* NBM_H */
