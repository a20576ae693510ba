// nbm_eval.cu -- evaluation of the trained surrogate on a dense grid (the
// "once trained, evaluate the simulation" use of arXiv 2210.14907, Fig. 1):
// u at the (n+1)^3 nodes -1 + i 2/n, each node with the network of its side
// of the interface (phi <= 0: minus).
//
// Tensor-core path: a persistent CTA per SM walks its tiles of 128 nodes once
// per network (the network's hidden weights are staged in shared memory once
// per pass; tiles without a node of that side are skipped).  Layer 1 (K = 3)
// and the output layer run in FP32; every hidden layer is one 128x128x128
// tcgen05 MMA with 16-bit operands (FP16 or BF16) and FP32 accumulation in
// TMEM.  The FP32 path is a plain SIMT evaluation (reference precision).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "nbm_device.cuh"
#include "nbm_tc_ptx.cuh"

namespace nbm {
namespace {

using namespace tc;

constexpr int kImgE = 32768;

// side of a grid node, decided as the FP64 level set would (FP32 first)
__device__ inline int node_phase(const ProbDev& P, float x, float y, float z) {
  const float f = phi_f(P, x, y, z);
  if (fabsf(f) < 2e-5f) return phi_d(P, (double)x, (double)y, (double)z) <= 0.0 ? 0 : 1;
  return f <= 0.f ? 0 : 1;
}

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (BF) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  } else {
    __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
}

__device__ __forceinline__ float fast_tanh(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void reduce32(float (&v)[32], int lane, float& s) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
#pragma unroll
    for (int i = 0; i < m; ++i) {
      const bool hi = lane & m;
      const float keep = hi ? v[m + i] : v[i], send = hi ? v[i] : v[m + i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  s = v[0];
}

// Points: the (n+1)^3 grid nodes, or (pts != nullptr) npts points pts[3i..3i+2].
template <int L, bool BF>
__global__ void __launch_bounds__(512, 1) k_eval_tc(ProbDev P, const float* __restrict__ params,
                                                    const unsigned char* __restrict__ wimg, int n,
                                                    const float* __restrict__ pts, int64_t npts,
                                                    float* __restrict__ u_out, int* status) {
  constexpr int H = 128, NG = L - 1;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Wimg = sm;                       // [NG]
  unsigned char* Aimg = sm + NG * kImgE;          // [2] ping-pong activations
  unsigned char* misc = sm + (NG + 2) * kImgE;
  uint64_t* bar_w = (uint64_t*)misc;
  uint64_t* bar_mma = (uint64_t*)(misc + 8);
  uint32_t* tslot = (uint32_t*)(misc + 16);
  float* red = (float*)(misc + 64);               // [4][128]
  float* xs = red + 512;                          // [3][128] node coordinates
  int* flag = (int*)(xs + 384);                   // [128]

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int q = w & 3, cg = w >> 2, u = 32 * q + lane, col0 = 32 * cg;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  const uint32_t idf = idesc_f16(BF, false, true);
  if (tid == 0) {
    mbar_init(smem_u32(bar_w), 1);
    mbar_init(smem_u32(bar_mma), 1);
    fence_mbar_init();
  }
  if (w == 0) tmem_alloc(smem_u32(tslot), 128);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  uint32_t ph_w = 0, ph_mma = 0;
  const int64_t N1 = n + 1, total = pts ? npts : N1 * N1 * N1;
  const int64_t T = (total + 127) / 128;
  const int64_t tb = (int64_t)blockIdx.x * T / gridDim.x, te = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  const float hg = 2.0f / (float)n;
  bool aborted = false;

  for (int s = 0; s < 2 && !aborted; ++s) {
    if (tid == 0) {
      mbar_expect_tx(smem_u32(bar_w), NG * kImgE);
      for (int g = 0; g < NG; ++g)
        bulk_g2s(smem_u32(Wimg + g * kImgE), wimg + ((int64_t)s * NG + g) * kImgE, kImgE,
                 smem_u32(bar_w));
    }
    const float* th = params + s * P.p_net;
    const float w10 = th[3 * u], w11 = th[3 * u + 1], w12 = th[3 * u + 2], b1 = th[3 * H + u];
    float bh[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) bh[g] = th[4 * H + (int64_t)g * (H * H + H) + (int64_t)H * H + u];
    const int64_t oo = 4 * H + (int64_t)NG * (H * H + H);
    const float wo = th[oo + u], bo = th[oo + H];
    {
      bool ok = mbar_wait_bounded(smem_u32(bar_w), ph_w);
      ph_w ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(status, 2);
        aborted = true;
        break;
      }
    }
    for (int64_t t = tb; t < te; ++t) {
      if (tid < 128) {
        const int64_t id = t * 128 + tid;
        int f = 0;
        float x = 0.f, y = 0.f, z = 0.f;
        if (id < total) {
          if (pts) {
            x = pts[3 * id];
            y = pts[3 * id + 1];
            z = pts[3 * id + 2];
          } else {
            const int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
            x = -1.f + hg * (float)i;
            y = -1.f + hg * (float)j;
            z = -1.f + hg * (float)k;
          }
          f = node_phase(P, x, y, z) == s;
        }
        xs[tid] = x;
        xs[128 + tid] = y;
        xs[256 + tid] = z;
        flag[tid] = f;
      }
      if (__syncthreads_count(tid < 128 && flag[tid]) == 0) continue;
      // layer 1 (FP32) -> 16-bit image
#pragma unroll
      for (int c8 = 0; c8 < 4; ++c8) {
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int c = col0 + 8 * c8 + e;
          o[e] = fast_tanh(fmaf(w10, xs[c], fmaf(w11, xs[128 + c], fmaf(w12, xs[256 + c], b1))));
        }
        uint4 pk = make_uint4(pack2<BF>(o[0], o[1]), pack2<BF>(o[2], o[3]), pack2<BF>(o[4], o[5]),
                              pack2<BF>(o[6], o[7]));
        *reinterpret_cast<uint4*>(Aimg + img_off(u, col0 + 8 * c8)) = pk;
      }
      fence_proxy_async();
      __syncthreads();
      float last[32];
#pragma unroll 1
      for (int g = 1; g <= NG; ++g) {
        if (tid == 0) {
          fence_after_sync();
          const uint32_t wa = smem_u32(Wimg + (g - 1) * kImgE);
          const uint32_t ab = smem_u32(Aimg + ((g - 1) & 1) * kImgE);
#pragma unroll
          for (int k = 0; k < 8; ++k) mma_f16(tmem, desc_kmajor(wa, k), desc_mnmajor(ab, k), idf, k > 0);
          mma_commit(smem_u32(bar_mma));
        }
        bool ok = mbar_wait_bounded(smem_u32(bar_mma), ph_mma);
        ph_mma ^= 1u;
        fence_after_sync();
        if (__syncthreads_or(!ok)) {
          if (tid == 0) atomicOr(status, 2);
          aborted = true;
          break;
        }
        float bb = bh[0];
#pragma unroll
        for (int i = 1; i < NG; ++i) bb = (g - 1 == i) ? bh[i] : bb;
        float acc[32];
        tmem_ld32(tmem + lane_base + col0, acc);
        if (g < NG) {
          unsigned char* dst = Aimg + (g & 1) * kImgE;
#pragma unroll
          for (int c8 = 0; c8 < 4; ++c8) {
            float o[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) o[e] = fast_tanh(acc[8 * c8 + e] + bb);
            uint4 pk = make_uint4(pack2<BF>(o[0], o[1]), pack2<BF>(o[2], o[3]),
                                  pack2<BF>(o[4], o[5]), pack2<BF>(o[6], o[7]));
            *reinterpret_cast<uint4*>(dst + img_off(u, col0 + 8 * c8)) = pk;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) last[i] = fast_tanh(acc[i] + bb);
        }
        fence_before_sync();
        fence_proxy_async();
        __syncthreads();
      }
      if (aborted) break;
      // output layer (FP32): sum over units
      {
        float v[32], sres;
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = wo * last[i];
        reduce32(v, lane, sres);
        red[q * 128 + col0 + lane] = sres;
      }
      __syncthreads();
      if (tid < 128 && flag[tid]) {
        const int64_t id = t * 128 + tid;
        u_out[id] = red[tid] + red[128 + tid] + red[256 + tid] + red[384 + tid] + bo;
      }
      __syncthreads();
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, 128);
}

// Plain FP32 evaluation: one thread per node, activations in shared memory
// ([unit][thread]), weights read through the read-only cache.
template <int H, int L>
__global__ void __launch_bounds__(128) k_eval_fp32(ProbDev P, const float* __restrict__ params,
                                                   int n, const float* __restrict__ pts,
                                                   int64_t npts, float* __restrict__ u_out) {
  extern __shared__ float act[];  // [2][H][128]
  const int tid = threadIdx.x;
  const int64_t N1 = n + 1, total = pts ? npts : N1 * N1 * N1;
  const int64_t id = (int64_t)blockIdx.x * 128 + tid;
  const float hg = 2.0f / (float)n;
  float x = 0.f, y = 0.f, z = 0.f;
  int s = 0;
  if (id < total) {
    if (pts) {
      x = pts[3 * id];
      y = pts[3 * id + 1];
      z = pts[3 * id + 2];
    } else {
      const int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
      x = -1.f + hg * (float)i;
      y = -1.f + hg * (float)j;
      z = -1.f + hg * (float)k;
    }
    s = node_phase(P, x, y, z);
  }
  float result = 0.f;
  for (int net = 0; net < 2; ++net) {
    const float* th = params + net * P.p_net;
    float* a0 = act;
    float* a1 = act + H * 128;
    for (int j = 0; j < H; ++j)
      a0[j * 128 + tid] = tanhf(fmaf(__ldg(th + 3 * j), x,
                                     fmaf(__ldg(th + 3 * j + 1), y,
                                          fmaf(__ldg(th + 3 * j + 2), z, __ldg(th + 3 * H + j)))));
    const float* Wl = th + 4 * H;
    for (int g = 1; g < L; ++g) {
      for (int j = 0; j < H; ++j) {
        float acc = __ldg(Wl + (int64_t)H * H + j);
        for (int k = 0; k < H; ++k) acc = fmaf(__ldg(Wl + (int64_t)j * H + k), a0[k * 128 + tid], acc);
        a1[j * 128 + tid] = tanhf(acc);
      }
      float* tmp = a0;
      a0 = a1;
      a1 = tmp;
      Wl += (int64_t)H * H + H;
    }
    float o = __ldg(Wl + H);
    for (int k = 0; k < H; ++k) o = fmaf(__ldg(Wl + k), a0[k * 128 + tid], o);
    if (net == s) result = o;
  }
  if (id < total) u_out[id] = result;
}

// Narrow networks (width <= 32, up to five layers; tanh or the sine layers of
// Sec. 4.1): the same per-node evaluation with the width and depth at run time.
template <int ACT>
__global__ void __launch_bounds__(128) k_eval_small(ProbDev P, const float* __restrict__ params,
                                                    int n, const float* __restrict__ pts,
                                                    int64_t npts, float* __restrict__ u_out) {
  __shared__ float act[2][32 * 128];
  const int tid = threadIdx.x, H = P.H, L = P.L;
  const int64_t N1 = n + 1, total = pts ? npts : N1 * N1 * N1;
  const int64_t id = (int64_t)blockIdx.x * 128 + tid;
  const float hg = 2.0f / (float)n;
  float x = 0.f, y = 0.f, z = 0.f;
  int s = 0;
  if (id < total) {
    if (pts) {
      x = pts[3 * id];
      y = pts[3 * id + 1];
      z = pts[3 * id + 2];
    } else {
      const int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
      x = -1.f + hg * (float)i;
      y = -1.f + hg * (float)j;
      z = -1.f + hg * (float)k;
    }
    s = node_phase(P, x, y, z);
  }
  auto actf = [](float v) { return ACT == NBM_ACT_SIN ? sinf(v) : tanhf(v); };
  float result = 0.f;
  for (int net = 0; net < 2; ++net) {
    const float* th = params + net * P.p_net;
    float* a0 = act[0];
    float* a1 = act[1];
    for (int j = 0; j < H; ++j)
      a0[j * 128 + tid] = actf(fmaf(__ldg(th + 3 * j), x,
                                    fmaf(__ldg(th + 3 * j + 1), y,
                                         fmaf(__ldg(th + 3 * j + 2), z, __ldg(th + 3 * H + j)))));
    const float* Wl = th + 4 * H;
    for (int g = 1; g < L; ++g) {
      for (int j = 0; j < H; ++j) {
        float acc = __ldg(Wl + (int64_t)H * H + j);
        for (int k = 0; k < H; ++k) acc = fmaf(__ldg(Wl + (int64_t)j * H + k), a0[k * 128 + tid], acc);
        a1[j * 128 + tid] = actf(acc);
      }
      float* tmp = a0;
      a0 = a1;
      a1 = tmp;
      Wl += (int64_t)H * H + H;
    }
    float o = __ldg(Wl + H);
    for (int k = 0; k < H; ++k) o = fmaf(__ldg(Wl + k), a0[k * 128 + tid], o);
    if (net == s) result = o;
  }
  if (id < total) u_out[id] = result;
}

cudaError_t launch_eval_small(const ProbDev& P, const float* params, int n, const float* pts,
                              int64_t npts, float* u, cudaStream_t st) {
  if (P.H < 1 || P.H > 32 || P.L < 2 || P.L > 5) return cudaErrorInvalidValue;
  const int64_t total = pts ? npts : (int64_t)(n + 1) * (n + 1) * (n + 1);
  const int nb = (int)((total + 127) / 128);
  if (P.activation == NBM_ACT_SIN)
    k_eval_small<NBM_ACT_SIN><<<nb, 128, 0, st>>>(P, params, n, pts, npts, u);
  else
    k_eval_small<NBM_ACT_TANH><<<nb, 128, 0, st>>>(P, params, n, pts, npts, u);
  return cudaGetLastError();
}

template <int L, bool BF>
cudaError_t launch_eval_tc_t(const ProbDev& P, const float* params, const unsigned char* wimg,
                             int n, const float* pts, int64_t npts, float* u, int grid, int* status,
                             cudaStream_t st) {
  const size_t smem = (size_t)(L + 1) * kImgE + 1024 + 8192;
  cudaError_t e = cudaFuncSetAttribute(k_eval_tc<L, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_eval_tc<L, BF><<<grid, 512, smem, st>>>(P, params, wimg, n, pts, npts, u, status);
  return cudaGetLastError();
}

template <int H, int L>
cudaError_t launch_eval_fp32_t(const ProbDev& P, const float* params, int n, const float* pts,
                               int64_t npts, float* u, cudaStream_t st) {
  const size_t smem = 2 * (size_t)H * 128 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_eval_fp32<H, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t total = pts ? npts : (int64_t)(n + 1) * (n + 1) * (n + 1);
  k_eval_fp32<H, L><<<(int)((total + 127) / 128), 128, smem, st>>>(P, params, n, pts, npts, u);
  return cudaGetLastError();
}

}  // namespace
}  // namespace nbm

using namespace nbm;

static int eval_common(nbm_problem* p, const float* params, int n, const float* pts, int64_t npts,
                       int precision, float* u_out, nbm_stream_t stream) {
  char msg[256];
  if (!p || !params || !u_out) {
    set_error_message("NULL argument");
    return NBM_ERR_INVALID_ARG;
  }
  if (int rc = check_aligned(params, 4, "params")) return rc;
  if (int rc = check_aligned(pts, 4, "pts")) return rc;
  if (int rc = check_aligned(u_out, 4, "u_out")) return rc;
  const nbm_problem_desc& d = problem_desc(p);
  if (!pts && (n < 1 || n > 4096)) {
    snprintf(msg, sizeof(msg), "grid evaluation needs 1 <= n <= 4096 (n=%d)", n);
    set_error_message(msg);
    return NBM_ERR_INVALID_ARG;
  }
  if (precision != NBM_PREC_FP32 && precision != NBM_PREC_BF16 && precision != NBM_PREC_FP16) {
    set_error_message("unknown precision");
    return NBM_ERR_INVALID_ARG;
  }
  if (precision != NBM_PREC_FP32 && !tc_supported(d.width, d.n_hidden)) {
    set_error_message("the tensor-core grid evaluation needs width 128 and 2..4 layers");
    return NBM_ERR_INVALID_ARG;
  }
  ProbDev P;
  make_prob_dev(d, P);
  if (int rc = attach_level_set(p, P)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (precision == NBM_PREC_FP32) {
#define NBM_EVAL32(HH, LL) \
  else if (d.width == HH && d.n_hidden == LL) e = launch_eval_fp32_t<HH, LL>(P, params, n, pts, npts, u_out, st);
    if (d.width <= 32) {
      e = launch_eval_small(P, params, n, pts, npts, u_out, st);
    }
    NBM_EVAL32(64, 2) NBM_EVAL32(64, 3) NBM_EVAL32(64, 4) NBM_EVAL32(128, 2) NBM_EVAL32(128, 3)
    NBM_EVAL32(128, 4)
#undef NBM_EVAL32
    else e = cudaErrorInvalidValue;
  } else {
    // the 16-bit weight images of both networks, in the shared-memory layout
    const size_t bytes = (size_t)2 * (d.n_hidden - 1) * kImgE;
    unsigned char* wimg = nullptr;
    int* status = nullptr;
    e = cudaMalloc((void**)&wimg, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    Workspace tmp;
    tmp.wtc = wimg;
    if (e == cudaSuccess) e = launch_prep_weights(P, params, precision, tmp, st);
    const int grid = problem_num_sms(p);
    const bool bf = precision == NBM_PREC_BF16;
    if (e == cudaSuccess) {
      if (d.n_hidden == 2) e = bf ? launch_eval_tc_t<2, true>(P, params, wimg, n, pts, npts, u_out, grid, status, st)
                                  : launch_eval_tc_t<2, false>(P, params, wimg, n, pts, npts, u_out, grid, status, st);
      else if (d.n_hidden == 3) e = bf ? launch_eval_tc_t<3, true>(P, params, wimg, n, pts, npts, u_out, grid, status, st)
                                       : launch_eval_tc_t<3, false>(P, params, wimg, n, pts, npts, u_out, grid, status, st);
      else e = bf ? launch_eval_tc_t<4, true>(P, params, wimg, n, pts, npts, u_out, grid, status, st)
                  : launch_eval_tc_t<4, false>(P, params, wimg, n, pts, npts, u_out, grid, status, st);
    }
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (wimg) cudaFree(wimg);
    if (status) cudaFree(status);
    if (e == cudaSuccess && (hs & 2)) {
      set_error_message("grid evaluation: a bounded device wait gave up");
      return NBM_ERR_DEVICE_TIMEOUT;
    }
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "grid evaluation: %s", cudaGetErrorString(e));
    set_error_message(msg);
    return NBM_ERR_CUDA;
  }
  return NBM_OK;
}

extern "C" int nbm_eval_grid(nbm_problem* p, const float* params, int n, int precision,
                             float* u_out, nbm_stream_t stream) {
  return eval_common(p, params, n, nullptr, 0, precision, u_out, stream);
}

extern "C" int nbm_eval_points(nbm_problem* p, const float* params, const float* pts, int64_t n,
                               int precision, float* u_out, nbm_stream_t stream) {
  if (!pts || n <= 0 || n > ((int64_t)1 << 34)) {
    set_error_message("nbm_eval_points: need pts != NULL and 0 < n <= 2^34");
    return NBM_ERR_INVALID_ARG;
  }
  return eval_common(p, params, 0, pts, n, precision, u_out, stream);
}
