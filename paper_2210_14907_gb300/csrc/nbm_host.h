// nbm_host.h -- internal declarations shared by the libnbm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "nbm.h"

namespace nbm {

// Launches `kern` on `st` with programmatic stream serialization: the grid may
// be scheduled while its predecessor in the stream still runs, so the kernel
// must begin with pdl_enter() (nbm_device.cuh), which waits for that
// predecessor before any dependent memory access.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct ProbDev;

// Kernel modes of the fused step kernels.
enum StepMode : int {
  MODE_CUT_FWD = 0,   // forward of cut-cell points through both networks
  MODE_RESIDUAL = 1,  // forward + residual of uncut points
  MODE_TRAIN = 2      // forward + residual + backward + weight gradient
};

// Geometry of one cut cell (computed in FP64 by the classifier pipeline).
struct CutRec {
  double Vm;       // volume fraction of Omega- (Omega+ has 1 - Vm)
  double Am[6];    // face fractions of Omega-, face f = 2*axis + (side > 0)
  double S;        // interface area / h^2
  double xg[3];    // interface point (projected centroid)
  double beta;     // [mu d_n u] at xg
  double alpha;    // [u] at xg
  double f[2];     // f^-(p), f^+(p)
  int point;       // collocation point index
  int has_jump;    // S > 0
};

// One collocation point of a tensor-core tile, stored in list order (each list
// padded to a multiple of 16) so that a half-tile's 8 records are one
// contiguous 256-byte block.
struct PRec {
  float x, y, z;     // point
  float gx, gy, gz;  // cut cell: interface point.  Uncut point: gx = f^s(p) in
                     // FP32 (FP64 rows: gx + gy = f^s(p) as a two-float sum), gz = 0
  int pt;            // point index, -1 for padding
  int cutj;          // -1: uncut; else 2*cut_id + has_jump
};

// Everything the fused step kernels read or write.
struct StepArgs {
  const float* x;
  const float* y;
  const float* z;
  const int* list[2];     // phase lists; entry >= 0 point index, < 0 cut id -(e+1)
  const int* counters;    // [0] n-, [1] n+, [2] n_cut
  const CutRec* cut;
  const PRec* rec;        // tile records of the two phase lists (tensor-core path)
  const PRec* rec_cut;    // tile records of the cut list (tensor-core path)
  const float* params;    // FP32 parameter pair
  const float* wt;        // FP32 transposed hidden weights [net][layer][k][u]
  const void* wtc;        // 16-bit hidden weights in the tensor-core layout [net][layer]
  float* cut_out;         // [n_cut][2][8] network outputs of cut points
  const float* cut_seed;  // [n_cut][2][8] seeds of cut points
  float* r2_out;          // [n] or nullptr
  double* loss_part;      // [grid] partial sums of r^2 over uncut points
  float* gpart;           // [grid][2][p_net] partial gradients
  int* gpart_flag;        // [grid][2]
  int* status;            // device status word (bounded waits)
  int mode;
  float scale;            // 1/N
};

// Device workspace of a problem (grown on demand).
struct Workspace {
  int64_t cap_n = 0;       // points
  int grid = 0;            // CTAs of the fused kernels
  float *x = nullptr, *y = nullptr, *z = nullptr;
  uint8_t* cls = nullptr;
  int* blockcnt = nullptr;  // [3][nb]
  int* list_minus = nullptr;
  int* list_plus = nullptr;
  int* cut_pt = nullptr;
  int* counters = nullptr;  // [4]
  CutRec* cut = nullptr;
  PRec* rec = nullptr;      // [2 cap + 64]
  PRec* rec_cut = nullptr;  // [cap + 32]
  int2* cut_rpos = nullptr; // [cap] a cut cell's record slots in rec (minus, plus)
  float* cut_out = nullptr;
  float* cut_seed = nullptr;
  double* loss_part = nullptr;      // [grid]
  double* cut_loss_part = nullptr;  // [nb_cut]
  double* loss = nullptr;           // [1]
  double* loss_acc = nullptr;       // [1] loss of the refinement levels done so far
  float* gacc = nullptr;            // [2 p_net] gradient of the refinement levels done so far
  float* gpart = nullptr;
  int* gpart_flag = nullptr;
  float* wt = nullptr;              // FP32 transposed hidden weights
  void* wtc = nullptr;              // 16-bit hidden weights
  float* grad = nullptr;            // [P]
  int64_t* step = nullptr;          // [1] device step counter
  int* status = nullptr;            // [1]
};

struct Profiler {
  static constexpr int kMax = 65536;
  bool on = false;
  int n = 0;
  std::vector<cudaEvent_t> ev = std::vector<cudaEvent_t>(2 * kMax, nullptr);
};

struct Problem {
  Profiler prof;
  nbm_problem_desc desc;
  int device = 0;
  int num_sms = 0;
  int64_t p_net = 0;
  Workspace ws;
  double* phi_grid = nullptr;  // NBM_GEOM_GRID: node values of the mesh level set
  int phi_n = 0;
};

// Device constants of refinement level `level` (cell spacing h / 2^level).
void make_prob_dev(const nbm_problem_desc& d, ProbDev& P, int level = 0);
// accessors for translation units that do not see the problem object
void set_error_message(const char* msg);
const nbm_problem_desc& problem_desc(const nbm_problem* p);
int problem_num_sms(const nbm_problem* p);
// Gives P the problem's mesh level set; NBM_ERR_INVALID_ARG (with the message
// set) for an NBM_GEOM_GRID problem whose level set has not been set.
int attach_level_set(const nbm_problem* p, ProbDev& P);
// NBM_ERR_INVALID_ARG (with the message set) when a non-NULL pointer is not
// aligned to `align` bytes (its element size).
int check_aligned(const void* ptr, size_t align, const char* name);

// ---- launchers (return cudaError_t of the launch) ----
// Draws (pts_in == NULL) or reads n points and classifies their cells.  Drawn
// point i is point first + i of a batch of n_total points (0: n_total = n), so
// a shard of a batch gets the counters and band decisions the whole batch
// would give it; n_band counts the band points of that whole batch.
// Sampling and classification of a step's points, then the phase lists.
// prep_params non-NULL: extra blocks of the same launch restage the hidden
// weights from those parameters (prec: the tensor-core image's 16-bit type).
// tiles: the scatter also writes the tensor-core kernel's tile records of the
// uncut points and their padding, and each cut cell's record slots.
cudaError_t launch_sample_classify(const ProbDev& P, const float* pts_in, uint64_t seed,
                                   const int64_t* step_dev, int64_t step_host, int64_t n,
                                   int64_t n_band, Workspace& ws, cudaStream_t st,
                                   int64_t first = 0, int64_t n_total = 0,
                                   const float* prep_params = nullptr, int prec = 0,
                                   bool tiles = false);
// tiles: also the cut cells' tile records (slots from the scatter's tiles pass)
cudaError_t launch_cut_geometry(const ProbDev& P, int64_t n, Workspace& ws, cudaStream_t st,
                                bool tiles = false);
// Whether a batch of n points gets its tile records from the scatter and the
// cut geometry (true: up to 2048 point blocks) or from launch_gather_tiles,
// which runs after the cut geometry (larger batches).
bool tiles_in_scatter(int64_t n);
cudaError_t launch_gather_tiles(const ProbDev& P, int64_t n, Workspace& ws, cudaStream_t st);
cudaError_t launch_cut_residual(const ProbDev& P, int64_t n, float scale, bool want_seeds,
                                float* r2_out, Workspace& ws, cudaStream_t st);
cudaError_t launch_prep_weights(const ProbDev& P, const float* params, int prec, Workspace& ws,
                                cudaStream_t st);
cudaError_t launch_step_fp32(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st);
cudaError_t launch_step_small(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st);
size_t small_smem_bytes(int L);
cudaError_t launch_step_tc(const ProbDev& P, const StepArgs& a, int grid, int prec, cudaStream_t st);
cudaError_t launch_finish(const ProbDev& P, int64_t n, int grid, bool adam, bool want_grad,
                          float* params, float* m, float* v, float* grad_out, float lr, float b1,
                          float b2, float eps, float* loss_hist, int64_t hist_base, int prec,
                          Workspace& ws, cudaStream_t st, int level = 0, int n_levels = 1,
                          double loss_scale = 0.0,  // 0: the loss is the mean over the n points
                          int64_t adam_t = 0);      // the Adam step (1-based) of this update
// Adam's bias correction 1 - beta^t of step t, in FP64 rounded to FP32 (on the
// host, where t of every enqueued step is known; both update kernels take it)
float adam_correction(float beta, int64_t t);
// Adam update t (bias-corrected, 1-based) of n parameters with a caller-supplied
// gradient, by the arithmetic of the fused update.  Skipped when loss != NULL
// and *loss is not finite.
cudaError_t launch_adam(int64_t n, float* params, float* m, float* v, const float* grad, float lr,
                        float b1, float b2, float eps, int64_t t, const double* loss,
                        cudaStream_t st);
size_t tc_smem_bytes(int L);
cudaError_t launch_selftest_wait(long long budget, int* out, cudaStream_t st);
size_t fp32_smem_bytes(int H, int L);
int tc_supported(int H, int L);

}  // namespace nbm
