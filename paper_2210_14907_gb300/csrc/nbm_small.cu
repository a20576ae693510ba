// nbm_small.cu -- the FP32 fused NBM step for narrow networks (width <= 32, up
// to five tanh or sine layers): the sine-activated 5 x 10 networks of the
// convergence study (arXiv 2210.14907, Sec. 4.1).
//
// Same organisation as the wide FP32 kernel: 8-point tiles, one warp per
// point, every point carrying 8 difference-form stencil columns (centre
// value, symmetric and antisymmetric increments of the three axes, value at
// the interface point of a cut cell); lane u < H owns unit u.  Each layer
// keeps its pre-activation columns (the sine adjoint needs z, mu, del) and its
// output columns (the next layer's input and the weight-gradient operand) in
// shared memory.  The weight gradient of a hidden layer is accumulated per
// tile into this CTA's partial slice in a fixed order (deterministic); the
// small parameters are accumulated per lane and written once per network.
#include "nbm_device.cuh"
#include "nbm_host.h"

namespace nbm {

namespace {

constexpr int kSPT = 8;   // points per tile (one per warp)
constexpr int kHM = 32;   // unit slots per point (lanes)
constexpr int kLM = 5;    // maximum number of activation layers

template <int ACT>
__device__ __forceinline__ float act_f(float z) {
  if constexpr (ACT == NBM_ACT_SIN) return sinf(z);
  else return act_tanh<false>(z);
}

// outputs of one unit's activation layer from its pre-activation columns
// zc[8] (scaled convention); o[8] receives the output columns
template <int ACT>
__device__ __forceinline__ void layer_fwd(const float zc[8], bool jump, float h, float h2,
                                          float ih, float ih2, float o[8]) {
  if constexpr (ACT == NBM_ACT_SIN) {
    float sz, cz;
    sincosf(zc[0], &sz, &cz);
    o[0] = sz;
#pragma unroll
    for (int i = 0; i < 3; ++i) sin_stencil_fwd(sz, cz, zc[1 + i], zc[4 + i], h, h2, ih, ih2, o[1 + i], o[4 + i]);
  } else {
    const float t = act_tanh<false>(zc[0]);
    o[0] = t;
#pragma unroll
    for (int i = 0; i < 3; ++i)
      tanh_stencil_fwd<false>(t, zc[1 + i], zc[4 + i], h, h2, ih, ih2, o[1 + i], o[4 + i]);
  }
  o[7] = jump ? act_f<ACT>(zc[7]) : 0.f;
}

// adjoint of one unit's activation layer: upstream gradients G[8] with respect
// to the output columns, gz[8] receives the gradients with respect to the
// pre-activation columns
template <int ACT>
__device__ __forceinline__ void layer_bwd(const float zc[8], const float oc[8], const float G[8],
                                          float h, float h2, float ih, float ih2, float gz[8]) {
  if constexpr (ACT == NBM_ACT_SIN) {
    float sz, cz;
    sincosf(zc[0], &sz, &cz);
    float gzc = cz * G[0];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      gzc += sin_stencil_bwd(sz, cz, zc[1 + i], zc[4 + i], G[1 + i], G[4 + i], h, h2, ih, ih2,
                             gz[1 + i], gz[4 + i]);
    gz[0] = gzc;
    gz[7] = cosf(zc[7]) * G[7];
  } else {
    const float t = oc[0], s0 = fmaf(-t, t, 1.f);
    float gzc = s0 * G[0];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      gzc += tanh_stencil_bwd(t, s0, oc[1 + i], oc[4 + i], G[1 + i], G[4 + i], h, h2, ih, ih2,
                              gz[1 + i], gz[4 + i]);
    gz[0] = gzc;
    gz[7] = fmaf(-oc[7], oc[7], 1.f) * G[7];
  }
}

__device__ __forceinline__ void ld8(const float* p, float v[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void st8(float* p, const float v[8]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

}  // namespace

size_t small_smem_bytes(int L) { return (size_t)2 * L * kSPT * kHM * 8 * sizeof(float); }

template <int ACT>
__global__ void __launch_bounds__(256, 1) k_step_small(ProbDev P, StepArgs a) {
  pdl_enter();
  extern __shared__ __align__(16) float sbuf[];
  __shared__ double loss_red[8];
  const int H = P.H, L = P.L;
  float* Zb = sbuf;                                   // [L][kSPT][kHM][8] pre-activations
  float* Ab = sbuf + (size_t)L * kSPT * kHM * 8;      // [L][kSPT][kHM][8] outputs
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
  const bool own = lane < H;  // lane u owns unit u
  auto Z = [&](int l, int pw, int u) -> float* { return Zb + (((size_t)l * kSPT + pw) * kHM + u) * 8; };
  auto A = [&](int l, int pw, int u) -> float* { return Ab + (((size_t)l * kSPT + pw) * kHM + u) * 8; };

  const int nm = a.counters[0], np = a.counters[1], nc = a.counters[2];
  int64_t T0, T;
  if (a.mode == MODE_CUT_FWD) {
    T0 = (nc + kSPT - 1) / kSPT;
    T = 2 * T0;
  } else {
    T0 = (nm + kSPT - 1) / kSPT;
    T = T0 + (np + kSPT - 1) / kSPT;
  }
  const int64_t tb = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t te = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  const float hf = P.hf, h2f = P.h2f, ihf = P.inv_hf, ih2f = P.inv_h2f;
  const bool train = a.mode == MODE_TRAIN;

  // small-parameter gradient accumulators of the current net (per lane)
  float gW1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gwo = 0.f, gbo = 0.f;
  float gbh[kLM - 1];
#pragma unroll
  for (int i = 0; i < kLM - 1; ++i) gbh[i] = 0.f;
  double loss_acc = 0.0;
  int cur_net = -1;
  bool first_tile = true;
  int wrote0 = 0, wrote1 = 0;

  auto flush = [&](int net) {
    __syncthreads();
    float* stage = Ab;  // [8 warps][nsmall]; activations are dead here
    const int nsmall = 4 * H + (L - 1) * H + H + 1;
    if (own) {
      float* st = stage + (size_t)w * nsmall;
      const int u = lane;
      st[3 * u] = gW1[0];
      st[3 * u + 1] = gW1[1];
      st[3 * u + 2] = gW1[2];
      st[3 * H + u] = gb1;
#pragma unroll
      for (int g = 0; g < kLM - 1; ++g)
        if (g < L - 1) st[4 * H + g * H + u] = gbh[g];
      st[4 * H + (L - 1) * H + u] = gwo;
    }
    if (lane == 0) stage[(size_t)w * nsmall + nsmall - 1] = gbo;
    __syncthreads();
    float* gp = a.gpart + ((int64_t)blockIdx.x * 2 + net) * P.gstride;
    for (int idx = tid; idx < nsmall; idx += blockDim.x) {
      float s = 0.f;
      for (int ww = 0; ww < 8; ++ww) s += stage[(size_t)ww * nsmall + idx];
      int64_t dst;
      if (idx < 4 * H) {
        dst = idx;  // W1, b1
      } else if (idx < 4 * H + (L - 1) * H) {
        const int g = (idx - 4 * H) / H, u = (idx - 4 * H) % H;  // bias of hidden layer g+1
        dst = 4 * H + (int64_t)g * (H * H + H) + (int64_t)H * H + u;
      } else {
        dst = 4 * H + (int64_t)(L - 1) * (H * H + H) + (idx - 4 * H - (L - 1) * H);
      }
      gp[dst] = s;
    }
    if (net) wrote1 = 1; else wrote0 = 1;
    gW1[0] = gW1[1] = gW1[2] = gb1 = gwo = gbo = 0.f;
#pragma unroll
    for (int i = 0; i < kLM - 1; ++i) gbh[i] = 0.f;
    __syncthreads();
  };

  for (int64_t tau = tb; tau < te; ++tau) {
    const int net = tau < T0 ? 0 : 1;
    const int64_t local = tau - (net ? T0 : 0);
    if (train && net != cur_net) {
      if (cur_net >= 0) flush(cur_net);
      cur_net = net;
      first_tile = true;
    }
    // ---- this warp's point (list entry >= 0: point index; < 0: cut id)
    const int64_t slot = local * kSPT + w;
    bool valid;
    int cut_id = -1, pt = 0;
    if (a.mode == MODE_CUT_FWD) {
      valid = slot < nc;
      if (valid) {
        cut_id = (int)slot;
        pt = a.cut[cut_id].point;
      }
    } else {
      valid = slot < (net ? np : nm);
      if (valid) {
        const int e = a.list[net][slot];
        if (e < 0) {
          cut_id = -e - 1;
          pt = a.cut[cut_id].point;
        } else {
          pt = e;
        }
      }
    }
    float px = 0.f, py = 0.f, pz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    bool jump = false;
    if (valid) {
      px = a.x[pt];
      py = a.y[pt];
      pz = a.z[pt];
      if (cut_id >= 0) {
        const CutRec& cr = a.cut[cut_id];
        jump = cr.has_jump;
        gx = (float)cr.xg[0];
        gy = (float)cr.xg[1];
        gz = (float)cr.xg[2];
      }
    }
    const float* th = a.params + net * P.p_net;
    const float* wo = th + 4 * H + (int64_t)(L - 1) * (H * H + H);

    // ---- layer 1 (3 -> H): exact increments mu = 0, del_i = h W1[u][i]
    if (own) {
      const int u = lane;
      const float w0 = th[3 * u], w1 = th[3 * u + 1], w2 = th[3 * u + 2], bb = th[3 * H + u];
      float zc[8] = {fmaf(w0, px, fmaf(w1, py, fmaf(w2, pz, bb))), 0.f, 0.f, 0.f, w0, w1, w2,
                     jump ? fmaf(w0, gx, fmaf(w1, gy, fmaf(w2, gz, bb))) : 0.f};
      float o[8];
      layer_fwd<ACT>(zc, jump, hf, h2f, ihf, ih2f, o);
      st8(Z(0, w, u), zc);
      st8(A(0, w, u), o);
    }
    __syncwarp();

    // ---- hidden layers (H -> H), FP32 FFMA
#pragma unroll 1
    for (int g = 1; g < L; ++g) {
      const float* WT = a.wt + ((int64_t)net * (L - 1) + (g - 1)) * H * H;  // [k][u]
      const float* bg = th + 4 * H + (int64_t)(g - 1) * (H * H + H) + (int64_t)H * H;
      if (own) {
        const int u = lane;
        const float bb = bg[u];
        float acc[8] = {bb, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, bb};
        for (int k = 0; k < H; ++k) {
          float av[8];
          ld8(A(g - 1, w, k), av);
          const float wv = WT[(int64_t)k * H + u];
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[c] = fmaf(wv, av[c], acc[c]);
        }
        float o[8];
        layer_fwd<ACT>(acc, jump, hf, h2f, ihf, ih2f, o);
        st8(Z(g, w, u), acc);
        st8(A(g, w, u), o);
      }
      __syncwarp();
    }

    // ---- output layer (H -> 1): warp reduction over units
    float out[8];
    {
      float oc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (own) ld8(A(L - 1, w, lane), oc);
      const float wv = own ? wo[lane] : 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float v = wv * oc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        out[c] = v;
      }
      out[0] += wo[H];
      out[7] += wo[H];
    }

    if (a.mode == MODE_CUT_FWD) {
      if (valid && lane == 0) {
        float* co = a.cut_out + (int64_t)cut_id * 16 + net * 8;
        st8(co, out);
      }
      continue;
    }

    // ---- residual row and seeds (every lane computes the same row)
    float seeds[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid && cut_id < 0) {
      double r2;
      if (P.fp64) r2 = uncut_residual<double>(P, net, px, py, pz, out, (double)a.scale, seeds);
      else r2 = (double)uncut_residual<float>(P, net, px, py, pz, out, a.scale, seeds);
      if (lane == 0) {
        loss_acc += r2;
        if (a.r2_out) a.r2_out[pt] = (P.level ? a.r2_out[pt] : 0.f) + (float)r2;
      }
    } else if (valid && train) {
      ld8(a.cut_seed + (int64_t)cut_id * 16 + net * 8, seeds);
    }
    if (!train) continue;

    // ---- backward: output layer
    float G[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (own) {
      float oc[8];
      ld8(A(L - 1, w, lane), oc);
      const float wv = wo[lane];
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        s = fmaf(seeds[c], oc[c], s);
        G[c] = wv * seeds[c];
      }
      gwo += s;
    }
    if (lane == 0) gbo += seeds[0] + seeds[7];

    // ---- backward through the hidden layers g = L-1 .. 1
#pragma unroll 1
    for (int g = L - 1; g >= 1; --g) {
      // adjoint of the activation layer that produced act[g]; the gradient with
      // respect to its pre-activation columns replaces them in Z
      if (own) {
        float zc[8], oc[8], gzv[8];
        ld8(Z(g, w, lane), zc);
        ld8(A(g, w, lane), oc);
        layer_bwd<ACT>(zc, oc, G, hf, h2f, ihf, ih2f, gzv);
        const float gsum = gzv[0] + gzv[7];
#pragma unroll
        for (int i = 0; i < kLM - 1; ++i) gbh[i] += (g - 1 == i) ? gsum : 0.f;
        st8(Z(g, w, lane), gzv);
      }
      __syncthreads();
      // weight gradient of hidden layer g: dW[u][k] += sum_{pw,c} gz[pw][u][c] act[g-1][pw][k][c]
      {
        float* gp = a.gpart + ((int64_t)blockIdx.x * 2 + net) * P.gstride + 4 * H +
                    (int64_t)(g - 1) * (H * H + H);
        for (int idx = tid; idx < H * H; idx += blockDim.x) {
          const int u = idx / H, k = idx % H;
          float acc = 0.f;
#pragma unroll 1
          for (int pw = 0; pw < kSPT; ++pw) {
            float gv[8], av[8];
            ld8(Z(g, pw, u), gv);
            ld8(A(g - 1, pw, k), av);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc = fmaf(gv[c], av[c], acc);
          }
          gp[idx] = first_tile ? acc : gp[idx] + acc;
        }
      }
      // input gradient: G[k][c] = sum_u W_g[u][k] gz[u][c]
      if (own) {
        const float* Wg = th + 4 * H + (int64_t)(g - 1) * (H * H + H);
#pragma unroll
        for (int c = 0; c < 8; ++c) G[c] = 0.f;
        for (int u = 0; u < H; ++u) {
          float gv[8];
          ld8(Z(g, w, u), gv);
          const float wv = Wg[(int64_t)u * H + lane];
#pragma unroll
          for (int c = 0; c < 8; ++c) G[c] = fmaf(wv, gv[c], G[c]);
        }
      }
      __syncthreads();
    }

    // ---- adjoint of layer 1 and its (3 -> H) parameter gradient; the
    // increments del_i = h W1[u][i] give d(dt_i)/dW1[u][i] = 1 (scaled columns)
    if (own) {
      float zc[8], oc[8], gzv[8];
      ld8(Z(0, w, lane), zc);
      ld8(A(0, w, lane), oc);
      layer_bwd<ACT>(zc, oc, G, hf, h2f, ihf, ih2f, gzv);
      gW1[0] += fmaf(gzv[0], px, fmaf(gzv[7], gx, gzv[4]));
      gW1[1] += fmaf(gzv[0], py, fmaf(gzv[7], gy, gzv[5]));
      gW1[2] += fmaf(gzv[0], pz, fmaf(gzv[7], gz, gzv[6]));
      gb1 += gzv[0] + gzv[7];
    }
    first_tile = false;
  }
  if (train && cur_net >= 0) flush(cur_net);
  // loss partial of this CTA (fixed order)
  if (lane == 0) loss_red[w] = loss_acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int ww = 0; ww < 8; ++ww) s += loss_red[ww];
    if (a.mode != MODE_CUT_FWD) a.loss_part[blockIdx.x] = s;
    if (train) {
      a.gpart_flag[2 * blockIdx.x] = wrote0;
      a.gpart_flag[2 * blockIdx.x + 1] = wrote1;
    }
  }
}

template <int ACT>
static cudaError_t launch_small_t(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st) {
  const size_t smem = small_smem_bytes(P.L);
  cudaError_t e = cudaFuncSetAttribute(k_step_small<ACT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_step_small<ACT>, dim3(grid), dim3(256), smem, st, P, a);
}

cudaError_t launch_step_small(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st) {
  if (P.H < 1 || P.H > kHM || P.L < 2 || P.L > kLM) return cudaErrorInvalidValue;
  if (P.activation == NBM_ACT_SIN) return launch_small_t<NBM_ACT_SIN>(P, a, grid, st);
  return launch_small_t<NBM_ACT_TANH>(P, a, grid, st);
}

}  // namespace nbm
