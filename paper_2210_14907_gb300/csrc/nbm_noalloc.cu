// nbm_noalloc.cu -- nbm_loss_grad_static: the loss-and-gradient call with all
// of its device scratch in one file-scope static __device__ array, for callers
// that cannot allocate device memory while they run (see include/nbm.h).
//
// The array is sized for the stated maximum: 16,384 collocation points per
// call, networks of width <= 128 with <= 4 tanh layers, and at most 16 CTAs
// for the fused step kernels.  Every call on a device shares the array.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "nbm_device.cuh"

namespace nbm {
namespace {

constexpr int64_t kStaticMaxPoints = 16384;
constexpr int kStaticMaxGrid = 16;
constexpr int64_t kStaticMaxPNetStride = 50180;  // H = 128, 4 tanh layers, rounded to 4
constexpr int kStaticMaxHidden = 3;              // hidden H x H layers
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// byte budget of every workspace array at the stated maximum
constexpr size_t kScratchBytes =
    3 * align256(kStaticMaxPoints * 4)                     // x, y, z
    + align256(kStaticMaxPoints)                           // cls
    + align256(3 * ((kStaticMaxPoints + 255) / 256) * 4)   // per-block counts
    + 3 * align256(kStaticMaxPoints * 4)                   // two phase lists, cut list
    + align256(4 * 4)                                      // counters
    + align256(kStaticMaxPoints * sizeof(CutRec))          // cut cells
    + align256((2 * kStaticMaxPoints + 64) * sizeof(PRec))  // tile records, phase lists
    + align256((kStaticMaxPoints + 32) * sizeof(PRec))      // tile records, cut list
    + align256(kStaticMaxPoints * 8)                       // cut cells' record slots
    + 2 * align256(kStaticMaxPoints * 16 * 4)              // cut outputs and seeds
    + align256(kStaticMaxGrid * 8)                         // loss partials
    + align256(((kStaticMaxPoints + 127) / 128) * 8)       // cut loss partials
    + align256(8)                                          // loss
    + align256((size_t)kStaticMaxGrid * 2 * kStaticMaxPNetStride * 4)  // gradient partials
    + align256(2 * kStaticMaxGrid * 4)                     // partial flags
    + align256((size_t)2 * kStaticMaxHidden * 128 * 128 * 4)  // FP32 transposed weights
    + align256((size_t)2 * kStaticMaxHidden * 128 * 128 * 2)  // 16-bit weight images
    + align256(8) + align256(4);                           // step, status

// The scratch.  In host code `g_static_scratch` only names the symbol; its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

thread_local char g_msg[256];

int fail_static(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  set_error_message(g_msg);
  return code;
}

// device address of the scratch on the current device (set-up once per device)
int scratch_base(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_static(NBM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_static(NBM_ERR_INVALID_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
      return fail_static(NBM_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_base[dev] = (unsigned char*)ptr;
  }
  *out = g_base[dev];
  return NBM_OK;
}

template <typename T>
T* carve(unsigned char*& cur, size_t bytes) {
  T* p = (T*)cur;
  cur += align256(bytes);
  return p;
}

}  // namespace
}  // namespace nbm

using namespace nbm;

extern "C" int nbm_loss_grad_static(nbm_problem* p, const float* params, const float* pts,
                                    int64_t n, uint64_t seed, int64_t step, float* grad_out,
                                    double* loss_out, nbm_stream_t stream) {
  if (!p || !params || !grad_out) return fail_static(NBM_ERR_INVALID_ARG, "NULL argument");
  if (int rc = check_aligned(params, 4, "params")) return rc;
  if (int rc = check_aligned(pts, 4, "pts")) return rc;
  if (int rc = check_aligned(grad_out, 4, "grad_out")) return rc;
  if (n <= 0 || n > kStaticMaxPoints)
    return fail_static(NBM_ERR_INVALID_ARG,
                       "batch %lld outside the static-scratch limit [1, %lld]", (long long)n,
                       (long long)kStaticMaxPoints);
  const nbm_problem_desc& d = problem_desc(p);
  const int num_sms = problem_num_sms(p);
  ProbDev P;
  make_prob_dev(d, P);
  if (int rc = attach_level_set(p, P)) return rc;
  if (d.width > 128 || d.n_hidden - 1 > kStaticMaxHidden || P.gstride > kStaticMaxPNetStride)
    return fail_static(NBM_ERR_INVALID_ARG, "network larger than the static-scratch limit");
  if (d.refine_levels != 0)
    return fail_static(NBM_ERR_INVALID_ARG,
                       "refinement levels need the problem's own workspace (nbm_loss_grad)");
  unsigned char* base = nullptr;
  int rc = scratch_base(&base);
  if (rc) return rc;

  Workspace w;
  const int nb = (int)((kStaticMaxPoints + 255) / 256);
  const int ncb = (int)((kStaticMaxPoints + 127) / 128);
  const int grid = num_sms < kStaticMaxGrid ? num_sms : kStaticMaxGrid;
  unsigned char* cur = base;
  w.x = carve<float>(cur, kStaticMaxPoints * 4);
  w.y = carve<float>(cur, kStaticMaxPoints * 4);
  w.z = carve<float>(cur, kStaticMaxPoints * 4);
  w.cls = carve<uint8_t>(cur, kStaticMaxPoints);
  w.blockcnt = carve<int>(cur, 3 * (size_t)nb * 4);
  w.list_minus = carve<int>(cur, kStaticMaxPoints * 4);
  w.list_plus = carve<int>(cur, kStaticMaxPoints * 4);
  w.cut_pt = carve<int>(cur, kStaticMaxPoints * 4);
  w.counters = carve<int>(cur, 16);
  w.cut = carve<CutRec>(cur, kStaticMaxPoints * sizeof(CutRec));
  w.rec = carve<PRec>(cur, (2 * kStaticMaxPoints + 64) * sizeof(PRec));
  w.rec_cut = carve<PRec>(cur, (kStaticMaxPoints + 32) * sizeof(PRec));
  w.cut_rpos = carve<int2>(cur, kStaticMaxPoints * 8);
  w.cut_out = carve<float>(cur, kStaticMaxPoints * 16 * 4);
  w.cut_seed = carve<float>(cur, kStaticMaxPoints * 16 * 4);
  w.loss_part = carve<double>(cur, kStaticMaxGrid * 8);
  w.cut_loss_part = carve<double>(cur, (size_t)ncb * 8);
  w.loss = carve<double>(cur, 8);
  w.gpart = carve<float>(cur, (size_t)kStaticMaxGrid * 2 * kStaticMaxPNetStride * 4);
  w.gpart_flag = carve<int>(cur, 2 * kStaticMaxGrid * 4);
  w.wt = carve<float>(cur, (size_t)2 * kStaticMaxHidden * 128 * 128 * 4);
  w.wtc = carve<void>(cur, (size_t)2 * kStaticMaxHidden * 128 * 128 * 2);
  w.step = carve<int64_t>(cur, 8);
  w.status = carve<int>(cur, 4);
  w.cap_n = kStaticMaxPoints;
  w.grid = grid;
  if ((size_t)(cur - base) > kScratchBytes)
    return fail_static(NBM_ERR_INVALID_ARG, "static scratch layout overflow");

  cudaStream_t st = (cudaStream_t)stream;
  const int prec = d.precision;
  cudaError_t e = cudaMemsetAsync(w.status, 0, sizeof(int), st);  // must start at zero
  const int64_t n_band =
      (d.geometry == NBM_GEOM_SPHERE || d.geometry == NBM_GEOM_FLOWER)
          ? (int64_t)floor(d.band_fraction * (double)n + 0.5)
          : 0;
  // the sampling launch also restages the hidden weights from params; the
  // scatter and the cut geometry write the tensor-core tile records
  const bool tiles = prec != NBM_PREC_FP32;
  if (e == cudaSuccess)
    e = launch_sample_classify(P, pts, seed, nullptr, step, n, n_band, w, st, 0, 0, params, prec,
                               tiles);
  if (e == cudaSuccess) e = launch_cut_geometry(P, n, w, st, tiles);
  if (e == cudaSuccess && tiles && !tiles_in_scatter(n)) e = launch_gather_tiles(P, n, w, st);
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
  a.scale = 1.0f / (float)n;
  auto step_launch = [&](int mode) {
    a.mode = mode;
    return prec == NBM_PREC_FP32 ? launch_step_fp32(P, a, grid, st)
                                 : launch_step_tc(P, a, grid, prec, st);
  };
  if (e == cudaSuccess) {
    // fine-h mode: the cut cells' networks on the FP32 path (as nbm_loss_grad)
    a.mode = MODE_CUT_FWD;
    e = (P.fp64 && prec != NBM_PREC_FP32) ? launch_step_fp32(P, a, grid, st)
                                           : step_launch(MODE_CUT_FWD);
  }
  if (e == cudaSuccess)
    e = launch_cut_residual(P, n, (float)(1.0 / (double)n), true, nullptr, w, st);
  if (e == cudaSuccess) e = step_launch(MODE_TRAIN);
  if (e == cudaSuccess)
    e = launch_finish(P, n, grid, false, true, nullptr, nullptr, nullptr, grad_out, 0.f, 0.9f,
                      0.999f, 0.f, nullptr, 0, prec, w, st);
  if (e != cudaSuccess) return fail_static(NBM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  if (loss_out) {
    int status = 0;
    e = cudaMemcpyAsync(loss_out, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_static(NBM_ERR_CUDA, "%s", cudaGetErrorString(e));
    if (status & 2) return fail_static(NBM_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up");
    if (!(*loss_out == *loss_out) || *loss_out > 1.7e308 || *loss_out < -1.7e308)
      return fail_static(NBM_ERR_NONFINITE, "loss is not finite");
  }
  return NBM_OK;
}
