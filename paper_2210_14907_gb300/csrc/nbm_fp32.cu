// nbm_fp32.cu -- the plain FP32 fused NBM step (arXiv 2210.14907, Sec. 3,
// Fig. 2): hidden-layer GEMMs in FP32 FFMA on the SIMT pipes.
//
// Tile = 8 collocation points, one warp per point.  Each point carries 8
// columns through the network: the centre value, the symmetric and
// antisymmetric stencil increments of the three axes (difference form, see
// nbm_device.cuh) and the value at the interface point of a cut cell.
// Lane l owns units l, l+32, ... of every layer.  Activations of all layers
// stay in shared memory for the backward; the weight gradient of a hidden
// layer is one CTA-wide [H x 64] x [64 x H] product per tile, accumulated into
// this CTA's slice of the partial-gradient buffer (no atomics: the final
// reduction over CTAs runs in a fixed order).
#include "nbm_device.cuh"
#include "nbm_host.h"

namespace nbm {

constexpr int kPT = 8;  // points per tile (one per warp)

template <int H, int L>
struct Fp32Cfg {
  static constexpr int NJ = H / 32;
  static constexpr int UB = H / 16;  // wgrad register block per thread
  static constexpr size_t act_floats = (size_t)L * kPT * H * 8;
};

template <int H, int L>
__global__ void __launch_bounds__(256, 1) k_step_fp32(ProbDev P, StepArgs a) {
  pdl_enter();
  using C = Fp32Cfg<H, L>;
  constexpr int NJ = C::NJ;
  extern __shared__ __align__(16) float act[];  // [L][kPT][H][8]
  __shared__ double loss_red[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tid = threadIdx.x;

  const int nm = a.counters[0], np = a.counters[1], nc = a.counters[2];
  int64_t T0, T;
  if (a.mode == MODE_CUT_FWD) {
    T0 = (nc + kPT - 1) / kPT;
    T = 2 * T0;
  } else {
    T0 = (nm + kPT - 1) / kPT;
    T = T0 + (np + kPT - 1) / kPT;
  }
  const int64_t tb = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t te = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  const float hf = P.hf, h2f = P.h2f, ihf = P.inv_hf, ih2f = P.inv_h2f;
  const bool train = a.mode == MODE_TRAIN;

  auto A = [&](int l, int pw, int u) -> float* {
    return act + (((size_t)l * kPT + pw) * H + u) * 8;
  };

  // small-parameter gradient accumulators of the current net (per lane)
  float gW1[NJ][3], gb1[NJ], gbh[L - 1][NJ], gwo[NJ], gbo = 0.f;
  auto zero_small = [&]() {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      gW1[j][0] = gW1[j][1] = gW1[j][2] = 0.f;
      gb1[j] = 0.f;
      gwo[j] = 0.f;
#pragma unroll
      for (int g = 0; g < L - 1; ++g) gbh[g][j] = 0.f;
    }
    gbo = 0.f;
  };
  zero_small();
  double loss_acc = 0.0;
  int cur_net = -1;
  bool first_tile = true;
  int wrote[2] = {0, 0};

  // flush the per-lane accumulators of net `net` into this CTA's partial
  auto flush = [&](int net) {
    __syncthreads();
    float* stage = act;  // [8 warps][nsmall]
    const int nsmall = 4 * H + (L - 1) * H + H + 1;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int u = lane + 32 * j;
      float* st = stage + (size_t)w * nsmall;
      st[3 * u] = gW1[j][0];
      st[3 * u + 1] = gW1[j][1];
      st[3 * u + 2] = gW1[j][2];
      st[3 * H + u] = gb1[j];
#pragma unroll
      for (int g = 0; g < L - 1; ++g) st[4 * H + g * H + u] = gbh[g][j];
      st[4 * H + (L - 1) * H + u] = gwo[j];
    }
    if (lane == 0) stage[(size_t)w * nsmall + nsmall - 1] = gbo;
    __syncthreads();
    float* gp = a.gpart + ((int64_t)blockIdx.x * 2 + net) * P.gstride;
    for (int idx = tid; idx < nsmall; idx += blockDim.x) {
      float s = 0.f;
      for (int ww = 0; ww < 8; ++ww) s += stage[(size_t)ww * nsmall + idx];
      int64_t dst;
      if (idx < 4 * H) dst = idx;  // W1, b1
      else if (idx < 4 * H + (L - 1) * H) {
        int g = (idx - 4 * H) / H, u = (idx - 4 * H) % H;  // bias of hidden layer g+1
        dst = 4 * H + (int64_t)g * (H * H + H) + (int64_t)H * H + u;
      } else {
        dst = 4 * H + (int64_t)(L - 1) * (H * H + H) + (idx - 4 * H - (L - 1) * H);
      }
      gp[dst] = s;
    }
    wrote[net] = 1;
    zero_small();
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
    // ---- this warp's point ----
    const int64_t slot = local * kPT + w;
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
        int e = a.list[net][slot];
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
    const float* W1 = th;
    const float* b1 = th + 3 * H;
    const float* wo = th + 4 * H + (int64_t)(L - 1) * (H * H + H);

    // ---- layer 1 (3 -> H), FP32, stencil increments exact: mt = 0, dt_i = W1[u][i]
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int u = lane + 32 * j;
      const float w0 = W1[3 * u], w1 = W1[3 * u + 1], w2 = W1[3 * u + 2], bb = b1[u];
      const float z = fmaf(w0, px, fmaf(w1, py, fmaf(w2, pz, bb)));
      const float t = act_tanh<false>(z);
      float o[8];
      o[0] = t;
      const float wi[3] = {w0, w1, w2};
#pragma unroll
      for (int i = 0; i < 3; ++i)
        tanh_stencil_fwd<false>(t, 0.f, wi[i], hf, h2f, ihf, ih2f, o[1 + i], o[4 + i]);
      o[7] = jump ? act_tanh<false>(fmaf(w0, gx, fmaf(w1, gy, fmaf(w2, gz, bb)))) : 0.f;
      float4* dst = reinterpret_cast<float4*>(A(0, w, u));
      dst[0] = make_float4(o[0], o[1], o[2], o[3]);
      dst[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    __syncwarp();

    // ---- hidden layers (H -> H), FP32 FFMA
    float last[NJ][8];
#pragma unroll 1
    for (int g = 1; g < L; ++g) {
      const float* WT = a.wt + ((int64_t)net * (L - 1) + (g - 1)) * H * H;
      const float* bg = th + 4 * H + (int64_t)(g - 1) * (H * H + H) + (int64_t)H * H;
      float acc[NJ][8];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float bb = bg[lane + 32 * j];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[j][c] = 0.f;
        acc[j][0] = bb;
        acc[j][7] = bb;
      }
      const float* ain = A(g - 1, w, 0);
#pragma unroll 4
      for (int k = 0; k < H; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(ain + 8 * k);
        const float4 a1 = *reinterpret_cast<const float4*>(ain + 8 * k + 4);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const float wv = WT[(int64_t)k * H + lane + 32 * j];
          acc[j][0] = fmaf(wv, a0.x, acc[j][0]);
          acc[j][1] = fmaf(wv, a0.y, acc[j][1]);
          acc[j][2] = fmaf(wv, a0.z, acc[j][2]);
          acc[j][3] = fmaf(wv, a0.w, acc[j][3]);
          acc[j][4] = fmaf(wv, a1.x, acc[j][4]);
          acc[j][5] = fmaf(wv, a1.y, acc[j][5]);
          acc[j][6] = fmaf(wv, a1.z, acc[j][6]);
          acc[j][7] = fmaf(wv, a1.w, acc[j][7]);
        }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int u = lane + 32 * j;
        float o[8];
        const float t = act_tanh<false>(acc[j][0]);
        o[0] = t;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          tanh_stencil_fwd<false>(t, acc[j][1 + i], acc[j][4 + i], hf, h2f, ihf, ih2f, o[1 + i],
                                  o[4 + i]);
        o[7] = act_tanh<false>(acc[j][7]);
        float4* dst = reinterpret_cast<float4*>(A(g, w, u));
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
#pragma unroll
        for (int c = 0; c < 8; ++c) last[j][c] = o[c];
      }
      __syncwarp();
    }

    // ---- output layer (H -> 1), FP32: warp reduction over units
    float out[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) out[c] = 0.f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float wv = wo[lane + 32 * j];
#pragma unroll
      for (int c = 0; c < 8; ++c) out[c] = fmaf(wv, last[j][c], out[c]);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) out[c] += __shfl_xor_sync(0xffffffffu, out[c], o);
    }
    out[0] += wo[H];
    out[7] += wo[H];

    if (a.mode == MODE_CUT_FWD) {
      if (valid && lane < 8) a.cut_out[(int64_t)cut_id * 16 + net * 8 + lane] = out[lane];
      continue;
    }

    // ---- residual and seeds
    float seeds[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) seeds[c] = 0.f;
    if (valid && cut_id < 0) {
      float sd[8];
      double r2;
      if (P.fp64) r2 = uncut_residual<double>(P, net, px, py, pz, out, (double)a.scale, sd);
      else r2 = (double)uncut_residual<float>(P, net, px, py, pz, out, a.scale, sd);
      if (lane == 0) {
        loss_acc += r2;
        if (a.r2_out) a.r2_out[pt] = (P.level ? a.r2_out[pt] : 0.f) + (float)r2;
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) seeds[c] = sd[c];
    } else if (valid && train) {
#pragma unroll
      for (int c = 0; c < 8; ++c) seeds[c] = a.cut_seed[(int64_t)cut_id * 16 + net * 8 + c];
    }
    if (!train) continue;

    // ---- backward: output layer
    float G[NJ][8];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float wv = wo[lane + 32 * j];
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        s = fmaf(seeds[c], last[j][c], s);
        G[j][c] = wv * seeds[c];
      }
      gwo[j] += s;
    }
    if (lane == 0) gbo += seeds[0] + seeds[7];

    // ---- backward through hidden layers g = L-1 .. 1
#pragma unroll 1
    for (int g = L - 1; g >= 1; --g) {
      // adjoint of the tanh layer that produced act[g]; gradient written in place
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int u = lane + 32 * j;
        float4* sp = reinterpret_cast<float4*>(A(g, w, u));
        const float4 s0v = sp[0], s1v = sp[1];
        const float st[8] = {s0v.x, s0v.y, s0v.z, s0v.w, s1v.x, s1v.y, s1v.z, s1v.w};
        const float t = st[0];
        const float s0 = fmaf(-t, t, 1.f);
        float gzv[8];
        float gzc = s0 * G[j][0];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          gzc += tanh_stencil_bwd(t, s0, st[1 + i], st[4 + i], G[j][1 + i], G[j][4 + i], hf, h2f,
                                  ihf, ih2f, gzv[1 + i], gzv[4 + i]);
        gzv[0] = gzc;
        gzv[7] = fmaf(-st[7], st[7], 1.f) * G[j][7];
        gbh[g - 1][j] += gzv[0] + gzv[7];
        sp[0] = make_float4(gzv[0], gzv[1], gzv[2], gzv[3]);
        sp[1] = make_float4(gzv[4], gzv[5], gzv[6], gzv[7]);
      }
      __syncthreads();
      // weight gradient of hidden layer g: dW[u][k] += sum_{pw,c} gz[pw][u][c] a[g-1][pw][k][c]
      {
        constexpr int UB = C::UB;
        const int ub = tid >> 4, kb = tid & 15;
        float acc[UB][UB];
#pragma unroll
        for (int i = 0; i < UB; ++i)
#pragma unroll
          for (int k = 0; k < UB; ++k) acc[i][k] = 0.f;
#pragma unroll 1
        for (int pw = 0; pw < kPT; ++pw) {
#pragma unroll
          for (int c4 = 0; c4 < 8; c4 += 4) {
            float4 gv[UB], av[UB];
#pragma unroll
            for (int i = 0; i < UB; ++i)
              gv[i] = *reinterpret_cast<const float4*>(A(g, pw, ub + 16 * i) + c4);
#pragma unroll
            for (int k = 0; k < UB; ++k)
              av[k] = *reinterpret_cast<const float4*>(A(g - 1, pw, kb + 16 * k) + c4);
#pragma unroll
            for (int i = 0; i < UB; ++i)
#pragma unroll
              for (int k = 0; k < UB; ++k) {
                acc[i][k] = fmaf(gv[i].x, av[k].x, acc[i][k]);
                acc[i][k] = fmaf(gv[i].y, av[k].y, acc[i][k]);
                acc[i][k] = fmaf(gv[i].z, av[k].z, acc[i][k]);
                acc[i][k] = fmaf(gv[i].w, av[k].w, acc[i][k]);
              }
          }
        }
        float* gp = a.gpart + ((int64_t)blockIdx.x * 2 + net) * P.gstride + 4 * H +
                    (int64_t)(g - 1) * (H * H + H);
#pragma unroll
        for (int i = 0; i < UB; ++i)
#pragma unroll
          for (int k = 0; k < UB; ++k) {
            const int64_t idx = (int64_t)(ub + 16 * i) * H + kb + 16 * k;
            gp[idx] = first_tile ? acc[i][k] : gp[idx] + acc[i][k];
          }
      }
      // input gradient: G[k][c] = sum_u W_g[u][k] gz[u][c]
      {
        const float* Wg = th + 4 * H + (int64_t)(g - 1) * (H * H + H);
        const float* gzp = A(g, w, 0);
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
          for (int c = 0; c < 8; ++c) G[j][c] = 0.f;
#pragma unroll 4
        for (int u = 0; u < H; ++u) {
          const float4 g0 = *reinterpret_cast<const float4*>(gzp + 8 * u);
          const float4 g1 = *reinterpret_cast<const float4*>(gzp + 8 * u + 4);
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const float wv = Wg[(int64_t)u * H + lane + 32 * j];
            G[j][0] = fmaf(wv, g0.x, G[j][0]);
            G[j][1] = fmaf(wv, g0.y, G[j][1]);
            G[j][2] = fmaf(wv, g0.z, G[j][2]);
            G[j][3] = fmaf(wv, g0.w, G[j][3]);
            G[j][4] = fmaf(wv, g1.x, G[j][4]);
            G[j][5] = fmaf(wv, g1.y, G[j][5]);
            G[j][6] = fmaf(wv, g1.z, G[j][6]);
            G[j][7] = fmaf(wv, g1.w, G[j][7]);
          }
        }
      }
      __syncthreads();
    }

    // ---- adjoint of layer 1 and its (3 -> H) parameter gradient
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int u = lane + 32 * j;
      const float4* sp = reinterpret_cast<const float4*>(A(0, w, u));
      const float4 s0v = sp[0], s1v = sp[1];
      const float st[8] = {s0v.x, s0v.y, s0v.z, s0v.w, s1v.x, s1v.y, s1v.z, s1v.w};
      const float t = st[0];
      const float s0 = fmaf(-t, t, 1.f);
      float gmu[3], gdl[3];
      float gzc = s0 * G[j][0];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        gzc += tanh_stencil_bwd(t, s0, st[1 + i], st[4 + i], G[j][1 + i], G[j][4 + i], hf, h2f,
                                ihf, ih2f, gmu[i], gdl[i]);
      const float gzg = fmaf(-st[7], st[7], 1.f) * G[j][7];
      gW1[j][0] += fmaf(gzc, px, fmaf(gzg, gx, gdl[0]));
      gW1[j][1] += fmaf(gzc, py, fmaf(gzg, gy, gdl[1]));
      gW1[j][2] += fmaf(gzc, pz, fmaf(gzg, gz, gdl[2]));
      gb1[j] += gzc + gzg;
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
      a.gpart_flag[2 * blockIdx.x] = wrote[0];
      a.gpart_flag[2 * blockIdx.x + 1] = wrote[1];
    }
  }
}

size_t fp32_smem_bytes(int H, int L) { return (size_t)L * kPT * H * 8 * sizeof(float); }

template <int H, int L>
static cudaError_t launch_fp32_t(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st) {
  size_t smem = fp32_smem_bytes(H, L);
  cudaError_t e = cudaFuncSetAttribute(k_step_fp32<H, L>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_step_fp32<H, L>, dim3(grid), dim3(256), smem, st, P, a);
}

cudaError_t launch_step_fp32(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st) {
  if (P.H <= 32) return launch_step_small(P, a, grid, st);  // narrow networks (nbm_small.cu)
#define NBM_FP32_CASE(HH, LL) \
  if (P.H == HH && P.L == LL) return launch_fp32_t<HH, LL>(P, a, grid, st);
  NBM_FP32_CASE(64, 2)
  NBM_FP32_CASE(64, 3)
  NBM_FP32_CASE(64, 4)
  NBM_FP32_CASE(128, 2)
  NBM_FP32_CASE(128, 3)
  NBM_FP32_CASE(128, 4)
#undef NBM_FP32_CASE
  return cudaErrorInvalidValue;
}

}  // namespace nbm
