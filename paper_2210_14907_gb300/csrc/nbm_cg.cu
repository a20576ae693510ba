// nbm_cg.cu -- grid scheme and Jacobi PCG (filled in below).
#include "nbm_device.cuh"

extern "C" int nbm_eval_grid(nbm_problem*, const float*, int, int, float*, nbm_stream_t) {
  return NBM_ERR_INVALID_ARG;
}
extern "C" int nbm_grid_cg_solve(nbm_problem*, int, double, int, double*, int*, double*,
                                 nbm_stream_t) {
  return NBM_ERR_INVALID_ARG;
}
