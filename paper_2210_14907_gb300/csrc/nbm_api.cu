// nbm_api.cu -- the C ABI of libnbm (include/nbm.h): argument checking, the
// device workspace, and the order of the stage launches of one NBM step
// (arXiv 2210.14907, Sec. 3): sample -> classify/partition -> cut geometry ->
// cut-cell forward (both networks) -> cut rows -> fused stencil step ->
// loss / gradient reduction -> Adam.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "nbm_device.cuh"

namespace nbm {

// Named host-side ranges (NVTX v3, header only): a profiler attached to the
// process sees each stage of a call; without one they cost a function call.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


static thread_local char g_err[512] = "no error";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define NBM_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? NBM_ERR_OOM : NBM_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
  } while (0)

void make_prob_dev(const nbm_problem_desc& d, ProbDev& P, int level) {
  memset(&P, 0, sizeof(P));
  const double h = ldexp(d.h, -level);  // cell spacing of this refinement level
  P.geometry = d.geometry;
  P.H = d.width;
  P.L = d.n_hidden;
  P.fp64 = d.fp64_stencil < 0 ? (h <= 2.0 / 512 + 1e-15) : (d.fp64_stencil != 0);
  P.level = level;
  P.h_band = d.h;
  P.solution = d.solution;
  P.activation = d.activation;
  P.r0 = d.r0;
  P.amp = d.amp;
  P.lt = d.lobes_theta;
  P.lp = d.lobes_psi;
  // integer lobe counts: the level set's angular factors by Chebyshev recurrences
  auto as_int = [](double v) { return (v >= 0.0 && v <= 64.0 && v == floor(v)) ? (int)v : -1; };
  P.lt_i = as_int(d.lobes_theta);
  P.lp_i = as_int(d.lobes_psi);
  P.mu[0] = d.mu_minus;
  P.mu[1] = d.mu_plus;
  P.k[0] = d.k_minus;
  P.k[1] = d.k_plus;
  P.h = h;
  P.lambda = d.lambda_jump;
  P.hf = (float)h;
  P.inv_hf = (float)(1.0 / h);
  P.h2f = (float)(h * h);
  P.inv_h2f = (float)(1.0 / (h * h));
  P.r0f = (float)d.r0;
  P.ampf = (float)d.amp;
  P.ltf = (float)d.lobes_theta;
  P.lpf = (float)d.lobes_psi;
  P.muf[0] = (float)d.mu_minus;
  P.muf[1] = (float)d.mu_plus;
  P.kf[0] = (float)d.k_minus;
  P.kf[1] = (float)d.k_plus;
  P.inv_h = 1.0 / h;
  P.inv_h2 = 1.0 / (h * h);
  for (int s = 0; s < 2; ++s) {
    P.inv_D[s] = 1.0 / (6.0 * P.mu[s] + h * h * P.k[s]);
    P.inv_Df[s] = (float)P.inv_D[s];
  }
  const int64_t H = d.width;
  P.p_net = 4 * H + (int64_t)(d.n_hidden - 1) * (H * H + H) + H + 1;
  P.gstride = (P.p_net + 3) & ~(int64_t)3;  // 16-byte aligned slices
}

static void ws_free(Workspace& w) {
  void* ptrs[] = {w.x, w.y, w.z, w.cls, w.blockcnt, w.list_minus, w.list_plus, w.cut_pt, w.rec,
                  w.rec_cut, w.cut_rpos,
                  w.counters, w.cut, w.cut_out, w.cut_seed, w.loss_part, w.cut_loss_part, w.loss,
                  w.gpart, w.gpart_flag, w.wt, w.wtc, w.grad, w.step, w.status, w.loss_acc,
                  w.gacc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w = Workspace();
}

template <typename T>
static cudaError_t dalloc(T*& p, size_t count) {
  return cudaMalloc((void**)&p, count * sizeof(T) + 16);
}

static int ws_reserve(Problem& pb, int64_t n) {
  Workspace& w = pb.ws;
  if (w.cap_n >= n && w.grid > 0) return NBM_OK;
  ws_free(w);
  const int64_t cap = n < 1024 ? 1024 : n;
  const int nb = (int)((cap + 255) / 256);
  const int ncb = (int)((cap + 31) / 32);  // cut-row blocks (one warp each)
  const int grid = pb.num_sms;
  const int64_t H = pb.desc.width, L = pb.desc.n_hidden;
  NBM_CUDA(dalloc(w.x, cap));
  NBM_CUDA(dalloc(w.y, cap));
  NBM_CUDA(dalloc(w.z, cap));
  NBM_CUDA(dalloc(w.cls, cap));
  NBM_CUDA(dalloc(w.blockcnt, 3 * (size_t)nb));
  NBM_CUDA(dalloc(w.list_minus, cap));
  NBM_CUDA(dalloc(w.list_plus, cap));
  NBM_CUDA(dalloc(w.cut_pt, cap));
  NBM_CUDA(dalloc(w.counters, 4));
  NBM_CUDA(dalloc(w.cut, cap));
  NBM_CUDA(dalloc(w.rec, 2 * (size_t)cap + 64));
  NBM_CUDA(dalloc(w.rec_cut, (size_t)cap + 32));
  NBM_CUDA(dalloc(w.cut_out, 16 * (size_t)cap));
  NBM_CUDA(dalloc(w.cut_seed, 16 * (size_t)cap));
  NBM_CUDA(dalloc(w.loss_part, grid));
  NBM_CUDA(dalloc(w.cut_loss_part, ncb));
  NBM_CUDA(dalloc(w.loss, 1));
  NBM_CUDA(dalloc(w.loss_acc, 1));
  NBM_CUDA(dalloc(w.gacc, 2 * (size_t)pb.p_net));
  NBM_CUDA(dalloc(w.gpart, (size_t)grid * 2 * ((pb.p_net + 3) & ~(int64_t)3)));
  NBM_CUDA(dalloc(w.gpart_flag, 2 * (size_t)grid));
  NBM_CUDA(dalloc(w.wt, 2 * (size_t)(L - 1) * H * H));
  NBM_CUDA(dalloc((uint16_t*&)w.wtc, 2 * (size_t)(L - 1) * H * H));
  NBM_CUDA(dalloc(w.grad, 2 * (size_t)pb.p_net));
  NBM_CUDA(dalloc(w.step, 1));
  NBM_CUDA(dalloc(w.status, 1));
  // last, so that the buffers above keep the placement they had without it
  NBM_CUDA(dalloc(w.cut_rpos, cap));
  NBM_CUDA(cudaMemset(w.status, 0, sizeof(int)));
  NBM_CUDA(cudaMemset(w.step, 0, sizeof(int64_t)));
  w.cap_n = cap;
  w.grid = grid;
  return NBM_OK;
}

static int check_desc(const nbm_problem_desc* d) {
  if (!d) return fail(NBM_ERR_INVALID_ARG, "descriptor is NULL");
  if (d->geometry < NBM_GEOM_SPHERE || d->geometry > NBM_GEOM_GRID)
    return fail(NBM_ERR_INVALID_ARG, "unknown geometry %d", d->geometry);
  const bool narrow = d->width >= 1 && d->width <= 32;  // the narrow FP32 kernels
  if (d->n_hidden < 2 || d->n_hidden > (narrow ? 5 : 4))
    return fail(NBM_ERR_INVALID_ARG, "n_hidden must be 2..4 (2..5 for width <= 32; got %d)",
                d->n_hidden);
  if (d->width != 64 && d->width != 128 && !narrow)
    return fail(NBM_ERR_INVALID_ARG, "width must be 1..32, 64 or 128 (got %d)", d->width);
  if (narrow && d->precision != NBM_PREC_FP32)
    return fail(NBM_ERR_INVALID_ARG, "widths <= 32 run on the FP32 path");
  if (d->precision != NBM_PREC_FP32 && d->precision != NBM_PREC_BF16)
    return fail(NBM_ERR_INVALID_ARG, "training precision must be FP32 or BF16 (got %d)",
                d->precision);
  if (d->precision != NBM_PREC_FP32 && !tc_supported(d->width, d->n_hidden))
    return fail(NBM_ERR_INVALID_ARG, "the tensor-core path needs width 128 and 2..4 layers");
  if (!(d->h > 0.0 && d->h <= 0.25)) return fail(NBM_ERR_INVALID_ARG, "h must be in (0, 0.25]");
  if (!(d->mu_minus > 0.0 && d->mu_plus > 0.0)) return fail(NBM_ERR_INVALID_ARG, "mu must be > 0");
  if (!(d->k_minus >= 0.0 && d->k_plus >= 0.0)) return fail(NBM_ERR_INVALID_ARG, "k must be >= 0");
  if (!(d->band_fraction >= 0.0 && d->band_fraction <= 1.0))
    return fail(NBM_ERR_INVALID_ARG, "band_fraction must be in [0, 1]");
  if (!(d->lambda_jump >= 0.0)) return fail(NBM_ERR_INVALID_ARG, "lambda_jump must be >= 0");
  if (d->geometry == NBM_GEOM_GRID && d->band_fraction != 0.0)
    return fail(NBM_ERR_INVALID_ARG, "band points need an analytic level set (band_fraction 0)");
  if (d->solution != NBM_SOL_BENCH && d->solution != NBM_SOL_SEC41)
    return fail(NBM_ERR_INVALID_ARG, "unknown solution %d", d->solution);
  if (d->activation != NBM_ACT_TANH && d->activation != NBM_ACT_SIN)
    return fail(NBM_ERR_INVALID_ARG, "unknown activation %d", d->activation);
  if (d->activation == NBM_ACT_SIN && (d->precision != NBM_PREC_FP32 || d->width > 32))
    return fail(NBM_ERR_INVALID_ARG, "sine networks run on the FP32 path with width <= 32");
  if (d->grid_jump != NBM_JUMP_EXACT && d->grid_jump != NBM_JUMP_EXTRAP &&
      d->grid_jump != NBM_JUMP_FIRST_ORDER)
    return fail(NBM_ERR_INVALID_ARG, "unknown grid_jump %d", d->grid_jump);
  if (d->reserved0 != 0) return fail(NBM_ERR_INVALID_ARG, "reserved0 must be 0");
  if (d->refine_levels < 0 || d->refine_levels > 3)
    return fail(NBM_ERR_INVALID_ARG, "refine_levels must be 0..3 (got %d)", d->refine_levels);
  if (!(ldexp(d->h, -d->refine_levels) >= 0x1p-12))
    return fail(NBM_ERR_INVALID_ARG, "finest refined spacing h/2^levels must be >= 2^-12");
  if (d->geometry == NBM_GEOM_SPHERE || d->geometry == NBM_GEOM_FLOWER) {
    if (!(d->r0 > 0.0 && d->r0 + fabs(d->amp) < 0.9))
      return fail(NBM_ERR_INVALID_ARG, "interface must lie inside the cube (r0 + |amp| < 0.9)");
  }
  return NBM_OK;
}

static int check_n(int64_t n) {
  if (n <= 0) return fail(NBM_ERR_INVALID_ARG, "batch must be positive (got %lld)", (long long)n);
  if (n > (int64_t)1 << 30) return fail(NBM_ERR_INVALID_ARG, "batch too large (> 2^30)");
  return NBM_OK;
}

static int64_t band_count(const nbm_problem_desc& d, int64_t n) {
  if (d.geometry != NBM_GEOM_SPHERE && d.geometry != NBM_GEOM_FLOWER) return 0;
  return (int64_t)floor(d.band_fraction * (double)n + 0.5);
}

static StepArgs base_args(Problem& pb, const float* params, int mode, float scale) {
  Workspace& w = pb.ws;
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.x = w.x;
  a.y = w.y;
  a.z = w.z;
  a.list[0] = w.list_minus;
  a.list[1] = w.list_plus;
  a.counters = w.counters;
  a.cut = w.cut;
  a.rec = w.rec;
  a.rec_cut = w.rec_cut;
  a.params = params;
  a.wt = w.wt;
  a.wtc = w.wtc;
  a.cut_out = w.cut_out;
  a.cut_seed = w.cut_seed;
  a.loss_part = w.loss_part;
  a.gpart = w.gpart;
  a.gpart_flag = w.gpart_flag;
  a.status = w.status;
  a.mode = mode;
  a.scale = scale;
  return a;
}

static cudaError_t launch_step(Problem& pb, const ProbDev& P, const StepArgs& a, cudaStream_t st) {
  if (pb.desc.precision == NBM_PREC_FP32) return launch_step_fp32(P, a, pb.ws.grid, st);
  return launch_step_tc(P, a, pb.ws.grid, pb.desc.precision, st);
}

// the fused MODE_TRAIN launch, bracketed by events while profiling is on
static cudaError_t launch_timed(Problem& pb, const ProbDev& P, const StepArgs& a, cudaStream_t st) {
  NvtxRange r("nbm.fused (forward, rows, backward)");
  Profiler& pr = pb.prof;
  const bool rec = pr.on && pr.n < Profiler::kMax;
  if (rec) {
    if (!pr.ev[2 * pr.n]) {
      cudaEventCreate(&pr.ev[2 * pr.n]);
      cudaEventCreate(&pr.ev[2 * pr.n + 1]);
    }
    cudaEventRecord(pr.ev[2 * pr.n], st);
  }
  cudaError_t e = launch_step(pb, P, a, st);
  if (rec) {
    cudaEventRecord(pr.ev[2 * pr.n + 1], st);
    ++pr.n;
  }
  return e;
}

// sample/classify .. cut rows; leaves seeds of cut cells in the workspace.  The
// n points are points first .. first+n-1 of a batch of n_total (0: n) points:
// drawn points take their counters and band decisions from the whole batch, and
// the seeds carry the whole batch's 1/n_total.
static int front_stages(Problem& pb, const ProbDev& P, const float* params, const float* pts,
                        int64_t n, uint64_t seed, const int64_t* step_dev, int64_t step_host,
                        bool want_seeds, float* r2_out, cudaStream_t st, int64_t first = 0,
                        int64_t n_total = 0, bool prep_w = false) {
  Workspace& w = pb.ws;
  NvtxRange r("nbm.front (sample, cell geometry, cut rows)");
  const int64_t nt = n_total > 0 ? n_total : n;
  // prep_w: the same launch restages the hidden weights from params (the
  // first pass of a call; later steps get them from the Adam kernel).  The
  // tensor-core paths' tile records come from the scatter (uncut points) and
  // the cut geometry (cut cells), or for large batches from a gather after both.
  const bool tiles = pb.desc.precision != NBM_PREC_FP32;
  NBM_CUDA(launch_sample_classify(P, pts, seed, step_dev, step_host, n, band_count(pb.desc, nt), w,
                                  st, first, nt, prep_w ? params : nullptr, pb.desc.precision,
                                  tiles));
  NBM_CUDA(launch_cut_geometry(P, n, w, st, tiles));
  if (tiles && !tiles_in_scatter(n)) NBM_CUDA(launch_gather_tiles(P, n, w, st));
  StepArgs a = base_args(pb, params, MODE_CUT_FWD, 1.0f / (float)nt);
  // The fine-h mode (FP64 rows) evaluates the cut cells' networks on the FP32
  // path: their jump rows U+(x_G) - U-(x_G) - alpha difference two O(1) network
  // values, which 16-bit GEMM operands would carry with ~2^-9 relative error.
  // Cut cells are a small share of the points, so the cost is small.
  if (P.fp64 && pb.desc.precision != NBM_PREC_FP32) NBM_CUDA(launch_step_fp32(P, a, w.grid, st));
  else NBM_CUDA(launch_step(pb, P, a, st));
  NBM_CUDA(launch_cut_residual(P, n, (float)(1.0 / (double)nt), want_seeds, r2_out, w, st));
  return NBM_OK;
}

static int read_loss(Problem& pb, double* loss_out, cudaStream_t st) {
  NBM_CUDA(cudaMemcpyAsync(loss_out, pb.ws.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  int status = 0;
  NBM_CUDA(cudaMemcpyAsync(&status, pb.ws.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NBM_CUDA(cudaStreamSynchronize(st));
  if (status & 2) {
    cudaMemsetAsync(pb.ws.status, 0, sizeof(int), st);
    return fail(NBM_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up");
  }
  if (!std::isfinite(*loss_out)) {
    cudaMemsetAsync(pb.ws.status, 0, sizeof(int), st);
    return fail(NBM_ERR_NONFINITE, "loss is not finite");
  }
  return NBM_OK;
}

}  // namespace nbm

using namespace nbm;

struct nbm_problem {
  Problem pb;
};

namespace nbm {
void set_error_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
const nbm_problem_desc& problem_desc(const nbm_problem* p) { return p->pb.desc; }
int problem_num_sms(const nbm_problem* p) { return p->pb.num_sms; }
int check_aligned(const void* ptr, size_t align, const char* name) {
  if (ptr && ((uintptr_t)ptr & (align - 1)) != 0)
    return fail(NBM_ERR_INVALID_ARG, "%s is not %zu-byte aligned", name, align);
  return NBM_OK;
}

int attach_level_set(const nbm_problem* p, ProbDev& P) {
  P.phi_grid = p->pb.phi_grid;
  P.phi_n = p->pb.phi_n;
  if (P.geometry == NBM_GEOM_GRID && !P.phi_grid)
    return fail(NBM_ERR_INVALID_ARG, "the mesh level set is not set (nbm_set_level_set)");
  return NBM_OK;
}
}  // namespace nbm

extern "C" {

const char* nbm_last_error(void) { return g_err; }

int nbm_init_problem(const nbm_problem_desc* d, nbm_problem** out) {
  if (!out) return fail(NBM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = check_desc(d);
  if (rc) return rc;
  nbm_problem* p = new (std::nothrow) nbm_problem();
  if (!p) return fail(NBM_ERR_OOM, "host allocation failed");
  p->pb.desc = *d;
  cudaError_t e = cudaGetDevice(&p->pb.device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&p->pb.num_sms, cudaDevAttrMultiProcessorCount, p->pb.device);
  if (e != cudaSuccess) {
    delete p;
    return fail(NBM_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  ProbDev P;
  make_prob_dev(*d, P);
  p->pb.p_net = P.p_net;
  *out = p;
  return NBM_OK;
}

int nbm_destroy(nbm_problem* p) {
  if (!p) return NBM_OK;
  ws_free(p->pb.ws);
  if (p->pb.phi_grid) cudaFree(p->pb.phi_grid);
  for (cudaEvent_t& e : p->pb.prof.ev)
    if (e) cudaEventDestroy(e);
  delete p;
  return NBM_OK;
}

int64_t nbm_param_count(const nbm_problem* p) { return p ? 2 * p->pb.p_net : -1; }

int nbm_selftest_bounded_wait(int64_t budget_cycles, nbm_stream_t stream) {
  if (budget_cycles < 1000 || budget_cycles > 10000000000LL)
    return fail(NBM_ERR_INVALID_ARG, "budget_cycles must be in [1e3, 1e10]");
  cudaStream_t st = (cudaStream_t)stream;
  int* d_out = nullptr;
  NBM_CUDA(cudaMalloc((void**)&d_out, sizeof(int)));
  int h_out = -1;
  cudaError_t e = launch_selftest_wait((long long)budget_cycles, d_out, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_out, d_out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_out);
  if (e != cudaSuccess) return fail(NBM_ERR_CUDA, "self-test: %s", cudaGetErrorString(e));
  if (h_out & 2) return fail(NBM_ERR_DEVICE_TIMEOUT, "the bounded wait gave up (as intended)");
  return NBM_OK;
}

int nbm_set_level_set(nbm_problem* p, const double* phi, int n, nbm_stream_t stream) {
  if (!p || !phi) return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  if (int rc = check_aligned(phi, 8, "phi")) return rc;
  Problem& pb = p->pb;
  if (pb.desc.geometry != NBM_GEOM_GRID)
    return fail(NBM_ERR_INVALID_ARG, "the problem's geometry is not NBM_GEOM_GRID");
  if (n < 1 || n > 1024) return fail(NBM_ERR_INVALID_ARG, "mesh level set needs 1 <= n <= 1024");
  const size_t count = (size_t)(n + 1) * (n + 1) * (n + 1);
  if (pb.phi_grid && pb.phi_n != n) {
    NBM_CUDA(cudaFree(pb.phi_grid));
    pb.phi_grid = nullptr;
  }
  if (!pb.phi_grid) {
    cudaError_t e = cudaMalloc((void**)&pb.phi_grid, count * sizeof(double));
    if (e != cudaSuccess) {
      pb.phi_grid = nullptr;
      return fail(NBM_ERR_OOM, "level-set mesh allocation failed");
    }
  }
  pb.phi_n = n;
  NBM_CUDA(cudaMemcpyAsync(pb.phi_grid, phi, count * sizeof(double), cudaMemcpyDeviceToDevice,
                           (cudaStream_t)stream));
  return NBM_OK;
}

int nbm_profile(nbm_problem* p, int enable, double* fused_ms_out, int64_t* fused_launches_out) {
  if (!p) return fail(NBM_ERR_INVALID_ARG, "NULL problem");
  Profiler& pr = p->pb.prof;
  if (enable) {
    pr.on = true;
    pr.n = 0;
    return NBM_OK;
  }
  pr.on = false;
  double ms = 0.0;
  for (int i = 0; i < pr.n; ++i) {
    NBM_CUDA(cudaEventSynchronize(pr.ev[2 * i + 1]));
    float t = 0.f;
    NBM_CUDA(cudaEventElapsedTime(&t, pr.ev[2 * i], pr.ev[2 * i + 1]));
    ms += t;
  }
  if (fused_ms_out) *fused_ms_out = ms;
  if (fused_launches_out) *fused_launches_out = pr.n;
  return NBM_OK;
}

int nbm_sample_points(nbm_problem* p, uint64_t seed, int64_t step, int64_t n, float* pts_out,
                      nbm_stream_t stream) {
  if (!p || !pts_out) return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  int rc = check_n(n);
  if (!rc) rc = check_aligned(pts_out, 4, "pts_out");
  if (rc) return rc;
  Problem& pb = p->pb;
  rc = ws_reserve(pb, n);
  if (rc) return rc;
  ProbDev P;
  make_prob_dev(pb.desc, P);
  if ((rc = attach_level_set(p, P))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  NBM_CUDA(launch_sample_classify(P, nullptr, seed, nullptr, step, n, band_count(pb.desc, n),
                                  pb.ws, st));
  // interleave SoA -> [n][3] via three strided 2D copies
  NBM_CUDA(cudaMemcpy2DAsync(pts_out, 3 * sizeof(float), pb.ws.x, sizeof(float), sizeof(float), n,
                             cudaMemcpyDeviceToDevice, st));
  NBM_CUDA(cudaMemcpy2DAsync(pts_out + 1, 3 * sizeof(float), pb.ws.y, sizeof(float),
                             sizeof(float), n, cudaMemcpyDeviceToDevice, st));
  NBM_CUDA(cudaMemcpy2DAsync(pts_out + 2, 3 * sizeof(float), pb.ws.z, sizeof(float),
                             sizeof(float), n, cudaMemcpyDeviceToDevice, st));
  return NBM_OK;
}

int nbm_residual(nbm_problem* p, const float* params, const float* pts, int64_t n, uint64_t seed,
                 int64_t step, float* r2_out, double* loss_out, nbm_stream_t stream) {
  if (!p || !params) return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  int rc = check_n(n);
  if (!rc) rc = check_aligned(params, 4, "params");
  if (!rc) rc = check_aligned(pts, 4, "pts");
  if (!rc) rc = check_aligned(r2_out, 4, "r2_out");
  if (rc) return rc;
  Problem& pb = p->pb;
  rc = ws_reserve(pb, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = pb.desc.precision, nlev = 1 + pb.desc.refine_levels;
  for (int lv = 0; lv < nlev; ++lv) {  // refinement levels: the same points, spacing h/2^lv
    ProbDev P;
    make_prob_dev(pb.desc, P, lv);
    if ((rc = attach_level_set(p, P))) return rc;
    rc = front_stages(pb, P, params, pts, n, seed, nullptr, step, false, r2_out, st, 0, 0, lv == 0);
    if (rc) return rc;
    StepArgs a = base_args(pb, params, MODE_RESIDUAL, 1.0f / (float)n);
    a.r2_out = r2_out;
    NBM_CUDA(launch_step(pb, P, a, st));
    NBM_CUDA(launch_finish(P, n, pb.ws.grid, false, false, nullptr, nullptr, nullptr, nullptr, 0.f,
                           0.9f, 0.999f, 0.f, nullptr, 0, prec, pb.ws, st, lv, nlev));
  }
  if (loss_out) return read_loss(pb, loss_out, st);
  return NBM_OK;
}

int nbm_loss_grad(nbm_problem* p, const float* params, const float* pts, int64_t n, uint64_t seed,
                  int64_t step, float* grad_out, double* loss_out, nbm_stream_t stream) {
  if (!p || !params || !grad_out) return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  int rc = check_n(n);
  if (!rc) rc = check_aligned(params, 4, "params");
  if (!rc) rc = check_aligned(pts, 4, "pts");
  if (!rc) rc = check_aligned(grad_out, 4, "grad_out");
  if (rc) return rc;
  Problem& pb = p->pb;
  rc = ws_reserve(pb, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = pb.desc.precision, nlev = 1 + pb.desc.refine_levels;
  for (int lv = 0; lv < nlev; ++lv) {
    ProbDev P;
    make_prob_dev(pb.desc, P, lv);
    if ((rc = attach_level_set(p, P))) return rc;
    rc = front_stages(pb, P, params, pts, n, seed, nullptr, step, true, nullptr, st, 0, 0, lv == 0);
    if (rc) return rc;
    StepArgs a = base_args(pb, params, MODE_TRAIN, 1.0f / (float)n);
    NBM_CUDA(launch_timed(pb, P, a, st));
    NBM_CUDA(launch_finish(P, n, pb.ws.grid, false, true, nullptr, nullptr, nullptr, grad_out, 0.f,
                           0.9f, 0.999f, 0.f, nullptr, 0, prec, pb.ws, st, lv, nlev));
  }
  if (loss_out) return read_loss(pb, loss_out, st);
  return NBM_OK;
}

int nbm_loss_grad_shard(nbm_problem* p, const float* params, const float* pts, int64_t n_total,
                        int64_t first, int64_t n, uint64_t seed, int64_t step, float* grad_out,
                        double* loss_out, nbm_stream_t stream) {
  if (!p || !params || !grad_out || !loss_out) return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  int rc = check_n(n);
  if (!rc) rc = check_n(n_total);
  if (!rc && (first < 0 || first > n_total - n))
    rc = fail(NBM_ERR_INVALID_ARG, "shard [%lld, %lld) outside the batch of %lld points",
              (long long)first, (long long)(first + n), (long long)n_total);
  if (!rc) rc = check_aligned(params, 4, "params");
  if (!rc) rc = check_aligned(pts, 4, "pts");
  if (!rc) rc = check_aligned(grad_out, 4, "grad_out");
  if (!rc) rc = check_aligned(loss_out, 8, "loss_out");
  if (rc) return rc;
  Problem& pb = p->pb;
  rc = ws_reserve(pb, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = pb.desc.precision, nlev = 1 + pb.desc.refine_levels;
  const double inv_total = 1.0 / (double)n_total;
  for (int lv = 0; lv < nlev; ++lv) {
    ProbDev P;
    make_prob_dev(pb.desc, P, lv);
    if ((rc = attach_level_set(p, P))) return rc;
    rc = front_stages(pb, P, params, pts, n, seed, nullptr, step, true, nullptr, st, first,
                      n_total, lv == 0);
    if (rc) return rc;
    StepArgs a = base_args(pb, params, MODE_TRAIN, (float)inv_total);
    NBM_CUDA(launch_timed(pb, P, a, st));
    NBM_CUDA(launch_finish(P, n, pb.ws.grid, false, true, nullptr, nullptr, nullptr, grad_out, 0.f,
                           0.9f, 0.999f, 0.f, nullptr, 0, prec, pb.ws, st, lv, nlev, inv_total));
  }
  NBM_CUDA(cudaMemcpyAsync(loss_out, pb.ws.loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return NBM_OK;
}

int nbm_adam_step(nbm_problem* p, float* params, float* adam_m, float* adam_v, const float* grad,
                  int64_t* step_io, float lr, float beta1, float beta2, float eps,
                  const double* loss, nbm_stream_t stream) {
  if (!p || !params || !adam_m || !adam_v || !grad || !step_io)
    return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  if (*step_io < 0) return fail(NBM_ERR_INVALID_ARG, "*step_io < 0");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return fail(NBM_ERR_INVALID_ARG, "bad Adam hyper-parameters");
  int rc = check_aligned(params, 4, "params");
  if (!rc) rc = check_aligned(adam_m, 4, "adam_m");
  if (!rc) rc = check_aligned(adam_v, 4, "adam_v");
  if (!rc) rc = check_aligned(grad, 4, "grad");
  if (!rc) rc = check_aligned(loss, 8, "loss");
  if (rc) return rc;
  NBM_CUDA(launch_adam(2 * p->pb.p_net, params, adam_m, adam_v, grad, lr, beta1, beta2, eps,
                       *step_io + 1, loss, (cudaStream_t)stream));
  *step_io += 1;
  return NBM_OK;
}

int nbm_train_steps(nbm_problem* p, float* params, float* adam_m, float* adam_v, int64_t* step_io,
                    int n_steps, int64_t batch, float lr, float beta1, float beta2, float eps,
                    uint64_t seed, const float* pts, float* loss_hist, nbm_stream_t stream) {
  if (!p || !params || !adam_m || !adam_v || !step_io)
    return fail(NBM_ERR_INVALID_ARG, "NULL argument");
  if (n_steps < 0) return fail(NBM_ERR_INVALID_ARG, "n_steps < 0");
  if (*step_io < 0) return fail(NBM_ERR_INVALID_ARG, "*step_io < 0");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return fail(NBM_ERR_INVALID_ARG, "bad Adam hyper-parameters");
  int rc = check_n(batch);
  if (!rc) rc = check_aligned(params, 4, "params");
  if (!rc) rc = check_aligned(adam_m, 4, "adam_m");
  if (!rc) rc = check_aligned(adam_v, 4, "adam_v");
  if (!rc) rc = check_aligned(pts, 4, "pts");
  if (!rc) rc = check_aligned(loss_hist, 4, "loss_hist");
  if (rc) return rc;
  if (n_steps == 0) return NBM_OK;
  Problem& pb = p->pb;
  rc = ws_reserve(pb, batch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = pb.desc.precision, nlev = 1 + pb.desc.refine_levels;
  const int64_t base = *step_io;
  ProbDev PL[4];
  for (int lv = 0; lv < nlev; ++lv) {
    make_prob_dev(pb.desc, PL[lv], lv);
    if ((rc = attach_level_set(p, PL[lv]))) return rc;
  }
  NBM_CUDA(cudaMemcpyAsync(pb.ws.step, step_io, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  for (int k = 0; k < n_steps; ++k) {
    const float* pk = pts ? pts + (int64_t)k * batch * 3 : nullptr;
    NvtxRange step_range("nbm.train_step");
    // refinement levels: the same points (the device step counter advances
    // after the last level), spacing h/2^lv; one Adam update per step
    for (int lv = 0; lv < nlev; ++lv) {
      const ProbDev& P = PL[lv];
      rc = front_stages(pb, P, params, pk, batch, seed, pb.ws.step, 0, true, nullptr, st, 0, 0,
                        k == 0 && lv == 0);
      if (rc) return rc;
      StepArgs a = base_args(pb, params, MODE_TRAIN, 1.0f / (float)batch);
      NBM_CUDA(launch_timed(pb, P, a, st));
      NBM_CUDA(launch_finish(P, batch, pb.ws.grid, true, false, params, adam_m, adam_v, nullptr,
                             lr, beta1, beta2, eps, loss_hist, base, prec, pb.ws, st, lv, nlev,
                             0.0, base + k + 1));
    }
  }
  *step_io = base + n_steps;
  return NBM_OK;
}

}  // extern "C"
