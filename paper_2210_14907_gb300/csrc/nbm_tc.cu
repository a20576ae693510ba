// nbm_tc.cu -- tcgen05 tensor-core fused NBM step (filled in below).
#include "nbm_device.cuh"

namespace nbm {

int tc_supported(int H, int L) { return H == 128 && L >= 2 && L <= 4; }
size_t tc_smem_bytes(int L) { return (size_t)(2 * L - 1) * 32768 + 4096; }

cudaError_t launch_step_tc(const ProbDev&, const StepArgs&, int, int, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t launch_eval_grid(const ProbDev&, const float*, int, int, float*, Workspace&, int,
                             cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace nbm
