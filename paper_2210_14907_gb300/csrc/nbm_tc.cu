// nbm_tc.cu -- the mixed-precision fused NBM step on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators), arXiv 2210.14907 Sec. 3 / Fig. 2.
//
// One persistent CTA per SM, 16 warps.  A tile is 16 collocation points x 8
// columns (centre value, symmetric and antisymmetric stencil increments of the
// three axes in difference form, and the interface-point value of cut cells),
// i.e. 128 GEMM columns.  Every hidden layer is one 128 x 128 x 128 product
// D[unit][col] = W[unit][k] A[k][col] on tcgen05 with 16-bit operands and FP32
// accumulation in TMEM; warp w reads TMEM lanes 32(w%4).. (one unit per
// thread) for columns 32(w/4).. (4 points).  The epilogue applies the tanh
// stencil layer in FP32 and writes the next 16-bit operand image to shared
// memory.  The first layer (K = 3), the output layer (H -> 1, a warp
// transpose-reduction), the residual rows and the seeds stay FP32 (FP64 rows
// on request).  The backward reuses the stored images: per hidden layer one
// input-gradient MMA (W^T gz, into the same TMEM columns) and one
// weight-gradient MMA (gz A^T) accumulated across all tiles of the CTA in
// dedicated TMEM columns, so the weight gradient never leaves the SM until
// the CTA's partial is written once per network.
//
// Shared memory: (L-1) weight images + L activation images of 32 KB each.
// TMEM: 128 columns for D + 128 per hidden layer for the weight gradient.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nbm_device.cuh"
#include "nbm_tc_ptx.cuh"

namespace nbm {

using namespace tc;

namespace {

constexpr int kTPts = 16;  // points per tile
constexpr int kImg = 32768;
constexpr int kMisc = 2048;

template <bool BF>
struct F16T;
template <>
struct F16T<true> {
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(v);
  }
};
template <>
struct F16T<false> {
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    __half2 v = *reinterpret_cast<__half2*>(&u);
    return __half22float2(v);
  }
};

template <bool BF>
__device__ __forceinline__ void store8o(unsigned char* img, uint32_t off, const float* o) {
  uint4 pk;
  pk.x = F16T<BF>::pack(o[0], o[1]);
  pk.y = F16T<BF>::pack(o[2], o[3]);
  pk.z = F16T<BF>::pack(o[4], o[5]);
  pk.w = F16T<BF>::pack(o[6], o[7]);
  *reinterpret_cast<uint4*>(img + off) = pk;
}
template <bool BF>
__device__ __forceinline__ void load8o(const unsigned char* img, uint32_t off, float* o) {
  const uint4 pk = *reinterpret_cast<const uint4*>(img + off);
  float2 a = F16T<BF>::unpack(pk.x), b = F16T<BF>::unpack(pk.y), c = F16T<BF>::unpack(pk.z),
         d = F16T<BF>::unpack(pk.w);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
}
template <bool BF>
__device__ __forceinline__ void store8(unsigned char* img, int row, int col0, const float* o) {
  uint4 pk;
  pk.x = F16T<BF>::pack(o[0], o[1]);
  pk.y = F16T<BF>::pack(o[2], o[3]);
  pk.z = F16T<BF>::pack(o[4], o[5]);
  pk.w = F16T<BF>::pack(o[6], o[7]);
  *reinterpret_cast<uint4*>(img + img_off(row, col0)) = pk;
}
template <bool BF>
__device__ __forceinline__ void load8(const unsigned char* img, int row, int col0, float* o) {
  const uint4 pk = *reinterpret_cast<const uint4*>(img + img_off(row, col0));
  float2 a = F16T<BF>::unpack(pk.x), b = F16T<BF>::unpack(pk.y), c = F16T<BF>::unpack(pk.z),
         d = F16T<BF>::unpack(pk.w);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
}

// Sum of v[0..31] over the 32 lanes of the warp: on return lane l holds the
// sum of column l (recursive halving, one exchange per value).
__device__ __forceinline__ void warp_transpose_reduce32(float (&v)[32], int lane, float& s) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const bool hi = lane & 16;
    const float keep = hi ? v[16 + i] : v[i], send = hi ? v[i] : v[16 + i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 8;
    const float keep = hi ? v[8 + i] : v[i], send = hi ? v[i] : v[8 + i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 4;
    const float keep = hi ? v[4 + i] : v[i], send = hi ? v[i] : v[4 + i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 2;
    const float keep = hi ? v[2 + i] : v[i], send = hi ? v[i] : v[2 + i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  {
    const bool hi = lane & 1;
    const float keep = hi ? v[1] : v[0], send = hi ? v[0] : v[1];
    s = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
}

}  // namespace

size_t tc_smem_bytes(int L) { return (size_t)(2 * L - 1) * kImg + 1024 + kMisc; }
int tc_supported(int H, int L) { return H == 128 && L >= 2 && L <= 4; }

// Column convention.  SCALED: the difference columns hold mt = mu/h^2 and
// dt = del/h (keeps FP16 operands out of the subnormal range).  Unscaled (BF16,
// whose exponent range is that of FP32): they hold mu and del themselves,
// which saves the rescaling in every epilogue; the output stage converts to
// the scaled convention of the residual rows.
template <int L, bool BF, bool FAST, bool SCALED>
__global__ void __launch_bounds__(512, 1) k_step_tc(ProbDev P, StepArgs a) {
  constexpr int H = 128;
  constexpr int NG = L - 1;  // hidden GEMM layers
  constexpr int kPPT = 4;    // points per thread (16 warps = 4 lane quadrants x 4 column groups)
  constexpr uint32_t NCOLS = (NG + 1) * 128 <= 256 ? 256 : 512;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Wimg = sm;                   // [NG][32 KB]
  unsigned char* Aimg = sm + NG * kImg;       // [L][32 KB]
  unsigned char* misc = sm + (2 * L - 1) * kImg;
  uint64_t* bar_w = (uint64_t*)misc;
  uint64_t* bar_mma = (uint64_t*)(misc + 8);
  uint64_t* bar_p = (uint64_t*)(misc + 16);
  uint32_t* tslot = (uint32_t*)(misc + 24);
  PRec* pbuf = (PRec*)(misc + 64);                 // [2][16] tile records (double buffer)
  float* seeds = (float*)(misc + 64 + 1024);       // 128 floats
  double* loss_red = (double*)(misc + 64 + 1024 + 512);  // 16 doubles
  float* red = (float*)(Aimg + (L - 1) * kImg);    // [4][128] scratch (forward end only)

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int q = w & 3, cg = w >> 2;
  const int u = 32 * q + lane;   // unit (TMEM lane) of this thread
  const int col0 = 32 * cg;      // first of this thread's 32 columns (points 4cg .. 4cg+3)
  // image byte offset of (unit u, point 4cg + j): the row part is fixed per
  // thread, the 16-byte chunk is ((4cg + j) mod 8) xor (u mod 8)
  const uint32_t row_off = (uint32_t)(((cg >> 1) * 16 + (u >> 3)) * 1024 + (u & 7) * 128);
  const uint32_t pbase = (uint32_t)((cg & 1) << 2), uxor = (uint32_t)(u & 7);
  auto poff = [&](int j) -> uint32_t { return row_off + ((((pbase + j) ^ uxor) & 7u) << 4); };
  const bool train = a.mode == MODE_TRAIN;
  const float hs = SCALED ? P.hf : 1.f, h2s = SCALED ? P.h2f : 1.f;
  const float ihs = SCALED ? P.inv_hf : 1.f, ih2s = SCALED ? P.inv_h2f : 1.f;
  const uint32_t id_fwd = idesc_f16(BF, false, true);
  const uint32_t id_dgr = idesc_f16(BF, true, true);
  const uint32_t id_wgr = idesc_f16(BF, false, false);

  if (tid == 0) {
    mbar_init(smem_u32(bar_w), 1);
    mbar_init(smem_u32(bar_mma), 1);
    mbar_init(smem_u32(bar_p), 1);
    fence_mbar_init();
  }
  if (w == 0) tmem_alloc(smem_u32(tslot), NCOLS);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t d_tm = tmem;                      // D: columns [0, 128)
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  uint32_t ph_w = 0, ph_mma = 0, ph_p = 0;
  bool aborted = false;

  const int nm = a.counters[0], np = a.counters[1], nc = a.counters[2];
  int64_t T0, T;
  if (a.mode == MODE_CUT_FWD) {
    T0 = (nc + kTPts - 1) / kTPts;
    T = 2 * T0;
  } else {
    T0 = (nm + kTPts - 1) / kTPts;
    T = T0 + (np + kTPts - 1) / kTPts;
  }
  const int64_t tb = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t te = (int64_t)(blockIdx.x + 1) * T / gridDim.x;

  // tile records: one 512-byte bulk copy per tile, fetched a tile ahead
  const PRec* recs = a.mode == MODE_CUT_FWD ? a.rec_cut : a.rec;
  auto prefetch = [&](int64_t tau) {
    const int64_t r = a.mode == MODE_CUT_FWD ? (tau < T0 ? tau : tau - T0) : tau;
    fence_proxy_async();
    mbar_expect_tx(smem_u32(bar_p), 16 * sizeof(PRec));
    bulk_g2s(smem_u32(pbuf + 16 * (tau & 1)), recs + 16 * r, 16 * sizeof(PRec), smem_u32(bar_p));
  };
  if (tid == 0 && tb < te) prefetch(tb);

  // per-net constants of this thread's unit
  float w1[3] = {0.f, 0.f, 0.f}, b1 = 0.f, bh[NG], wo = 0.f, bo = 0.f;
#pragma unroll
  for (int g = 0; g < NG; ++g) bh[g] = 0.f;
  // gradient accumulators of the small parameters
  float gW1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gbh[NG], gwo = 0.f, gbo = 0.f;
#pragma unroll
  for (int g = 0; g < NG; ++g) gbh[g] = 0.f;
  float loss_acc = 0.f;     // per-thread FP32 sum of r^2 (FP32 rows)
  double loss_acc_d = 0.0;  // per-thread FP64 sum of r^2 (FP64 rows)
  int cur_net = -1;
  bool first_tile = true;
  int wrote0 = 0, wrote1 = 0;

  auto wait_mma = [&]() -> bool {
    bool ok = mbar_wait_bounded(smem_u32(bar_mma), ph_mma);
    ph_mma ^= 1u;
    fence_after_sync();
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(a.status, 2);
      return false;
    }
    return true;
  };

  auto flush = [&](int net) {
    // weight gradients of the hidden layers straight from TMEM
    float* gp = a.gpart + ((int64_t)blockIdx.x * 2 + net) * P.gstride;
#pragma unroll 1
    for (int g = 1; g <= NG; ++g) {
      float* dst = gp + 4 * H + (int64_t)(g - 1) * (H * H + H) + (int64_t)u * H + col0;
      float v[32];
      tmem_ld32(tmem + 128u * g + lane_base + col0, v);
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
    // small parameters: the four column groups of a unit are combined in smem
    float* stage = (float*)Aimg;  // [4 groups][128 units][8]
    fence_before_sync();
    __syncthreads();
    {
      float* s = stage + (cg * 128 + u) * 8;
      s[0] = gW1[0]; s[1] = gW1[1]; s[2] = gW1[2]; s[3] = gb1; s[4] = gwo;
#pragma unroll
      for (int g = 0; g < NG; ++g) s[5 + g] = gbh[g];
    }
    __syncthreads();
    if (cg == 0) {
      float t[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) t[k] = stage[u * 8 + k];
#pragma unroll
      for (int c2 = 1; c2 < 4; ++c2)
#pragma unroll
        for (int k = 0; k < 8; ++k) t[k] += stage[(c2 * 128 + u) * 8 + k];
      gp[3 * u] = t[0];
      gp[3 * u + 1] = t[1];
      gp[3 * u + 2] = t[2];
      gp[3 * H + u] = t[3];
#pragma unroll
      for (int g = 0; g < NG; ++g) gp[4 * H + (int64_t)g * (H * H + H) + (int64_t)H * H + u] = t[5 + g];
      const int64_t oo = 4 * H + (int64_t)NG * (H * H + H);
      gp[oo + u] = t[4];
      if (tid == 0) gp[oo + H] = gbo;
    }
    gW1[0] = gW1[1] = gW1[2] = gb1 = gwo = gbo = 0.f;
#pragma unroll
    for (int g = 0; g < NG; ++g) gbh[g] = 0.f;
    if (net) wrote1 = 1; else wrote0 = 1;
    __syncthreads();
  };

  for (int64_t tau = tb; tau < te && !aborted; ++tau) {
    const int net = tau < T0 ? 0 : 1;
    const int64_t local = tau - (net ? T0 : 0);
    if (net != cur_net) {
      if (train && cur_net >= 0) flush(cur_net);
      cur_net = net;
      first_tile = true;
      // stage this network's hidden weights (bulk copy engine)
      if (tid == 0) {
        const unsigned char* src = (const unsigned char*)a.wtc + (int64_t)net * NG * kImg;
        mbar_expect_tx(smem_u32(bar_w), NG * kImg);
        for (int g = 0; g < NG; ++g)
          bulk_g2s(smem_u32(Wimg + g * kImg), src + (int64_t)g * kImg, kImg, smem_u32(bar_w));
      }
      const float* th = a.params + net * P.p_net;
      w1[0] = th[3 * u];
      w1[1] = th[3 * u + 1];
      w1[2] = th[3 * u + 2];
      b1 = th[3 * H + u];
#pragma unroll
      for (int g = 0; g < NG; ++g) bh[g] = th[4 * H + (int64_t)g * (H * H + H) + (int64_t)H * H + u];
      const int64_t oo = 4 * H + (int64_t)NG * (H * H + H);
      wo = th[oo + u];
      bo = th[oo + H];
      bool ok = mbar_wait_bounded(smem_u32(bar_w), ph_w);
      ph_w ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.status, 2);
        aborted = true;
        break;
      }
    }
    // ---- tile records (prefetched during the previous tile)
    {
      bool ok = mbar_wait_bounded(smem_u32(bar_p), ph_p);
      ph_p ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.status, 2);
        aborted = true;
        break;
      }
      if (tid == 0 && tau + 1 < te) prefetch(tau + 1);
    }
    const PRec* pr = pbuf + 16 * (tau & 1);
    // seed of a cut point (from the cut-row kernel): load it now, use it after
    // the forward, so that the global-memory latency is hidden
    float cut_sd = 0.f;
    if (train && tid < 128) {
      const PRec& pc = pr[tid >> 3];
      if (pc.pt >= 0 && pc.cutj >= 0)
        cut_sd = __ldg(a.cut_seed + (int64_t)(pc.cutj >> 1) * 16 + net * 8 + (tid & 7));
    }

    // ---- layer 1 (3 -> H) in FP32; exact increments mu = 0, del_i = h W1[u][i]
    {
      const float dl1[3] = {SCALED ? w1[0] : w1[0] * P.hf, SCALED ? w1[1] : w1[1] * P.hf,
                            SCALED ? w1[2] : w1[2] * P.hf};
#pragma unroll
      for (int pp = 0; pp < kPPT; ++pp) {
        const int p = 4 * cg + pp;
        const PRec pi = pr[p];
        const float z = fmaf(w1[0], pi.x, fmaf(w1[1], pi.y, fmaf(w1[2], pi.z, b1)));
        const float t = act_tanh<FAST>(z);
        float o[8];
        o[0] = t;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          tanh_stencil_fwd<FAST>(t, 0.f, dl1[i], hs, h2s, ihs, ih2s, o[1 + i], o[4 + i]);
        const bool jump = pi.cutj >= 0 && (pi.cutj & 1);
        o[7] = jump ? act_tanh<FAST>(fmaf(w1[0], pi.gx, fmaf(w1[1], pi.gy, fmaf(w1[2], pi.gz, b1))))
                    : 0.f;
        store8o<BF>(Aimg, poff(pp), o);
      }
    }
    fence_proxy_async();
    __syncthreads();

    // ---- hidden layers on the tensor cores
    float last[32];
#pragma unroll 1
    for (int g = 1; g <= NG; ++g) {
      if (tid == 0) {
        fence_after_sync();
        const uint32_t wa = smem_u32(Wimg + (g - 1) * kImg), ab = smem_u32(Aimg + (g - 1) * kImg);
#pragma unroll
        for (int k = 0; k < 8; ++k) mma_f16(d_tm, desc_kmajor(wa, k), desc_mnmajor(ab, k), id_fwd, k > 0);
        mma_commit(smem_u32(bar_mma));
      }
      if (!wait_mma()) {
        aborted = true;
        break;
      }
      float bb = bh[0];
#pragma unroll
      for (int i = 1; i < NG; ++i) bb = (g - 1 == i) ? bh[i] : bb;
      float acc[32];
      tmem_ld32(d_tm + lane_base + col0, acc);
#pragma unroll
      for (int j = 0; j < kPPT; ++j) {
        const float* c = acc + 8 * j;
        float o[8];
        const float t = act_tanh<FAST>(c[0] + bb);
        o[0] = t;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          tanh_stencil_fwd<FAST>(t, c[1 + i], c[4 + i], hs, h2s, ihs, ih2s, o[1 + i], o[4 + i]);
        o[7] = act_tanh<FAST>(c[7] + bb);
        if (g < NG) {
          store8o<BF>(Aimg + g * kImg, poff(j), o);
        } else {
#pragma unroll
          for (int c2 = 0; c2 < 8; ++c2) last[8 * j + c2] = o[c2];
        }
      }
      fence_before_sync();
      fence_proxy_async();
      __syncthreads();
    }
    if (aborted) break;

    // ---- output layer (H -> 1) in FP32: sum over the 32 units of the warp,
    // then over the four lane quadrants
    {
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = wo * last[i];
      float s;
      warp_transpose_reduce32(v, lane, s);  // lane l: column col0 + l
      red[q * 128 + col0 + lane] = s;
    }
    __syncthreads();
    // ---- output columns and residual rows: thread (p, k) owns column 8p + k
    // of point p; the centre term (k = 0) and the six cell faces (k = 1..6)
    // are combined across the 8 lanes of the point
    if (tid < 128) {
      const int c = tid, p = c >> 3, k = c & 7;
      float o = red[c] + red[128 + c] + red[256 + c] + red[384 + c];
      if (k == 0 || k == 7) o += bo;
      // scaled convention of the rows: U, Mt_i = M_i/h^2, Dt_i = D_i/h, U(x_G)
      if (!SCALED) o *= (k >= 1 && k <= 3) ? P.inv_h2f : ((k >= 4 && k <= 6) ? P.inv_hf : 1.f);
      const PRec pi = pr[p];
      const bool valid = pi.pt >= 0, is_cut = pi.cutj >= 0;
      float sd = 0.f;
      if (a.mode == MODE_CUT_FWD) {
        if (valid) a.cut_out[(int64_t)(pi.cutj >> 1) * 16 + net * 8 + k] = o;
      } else {
        float sr, r2;
        double r2d = 0.0;
        if (P.fp64) {
          r2d = uncut_residual8<double>(P, net, pi.x, pi.y, pi.z, o, k, lane, (double)a.scale, sr);
          r2 = (float)r2d;
        } else {
          r2 = uncut_residual8<float>(P, net, pi.x, pi.y, pi.z, o, k, lane, a.scale, sr);
        }
        if (valid && !is_cut) {
          sd = sr;
          if (k == 0) {
            if (P.fp64) loss_acc_d += r2d;
            else loss_acc += r2;
            if (a.r2_out) a.r2_out[pi.pt] = r2;
          }
        } else if (valid && train) {
          sd = cut_sd;
        }
      }
      // seeds in this kernel's column convention
      if (!SCALED) sd *= (k >= 1 && k <= 3) ? P.inv_h2f : ((k >= 4 && k <= 6) ? P.inv_hf : 1.f);
      seeds[c] = sd;
    }
    __syncthreads();
    if (!train) continue;

    // ---- backward: adjoint of the last tanh layer (FP32 state in registers)
#pragma unroll
    for (int pp = 0; pp < kPPT; ++pp) {
      const int p = 4 * cg + pp;
      float sd[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) sd[c] = seeds[8 * p + c];
      const float* st = last + 8 * pp;
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) s = fmaf(sd[c], st[c], s);
      gwo += s;
      const float t = st[0], s0 = fmaf(-t, t, 1.f);
      float gz[8];
      float gzc = s0 * (wo * sd[0]);
#pragma unroll
      for (int i = 0; i < 3; ++i)
        gzc += tanh_stencil_bwd(t, s0, st[1 + i], st[4 + i], wo * sd[1 + i], wo * sd[4 + i], hs,
                                h2s, ihs, ih2s, gz[1 + i], gz[4 + i]);
      gz[0] = gzc;
      gz[7] = fmaf(-st[7], st[7], 1.f) * (wo * sd[7]);
      gbh[NG - 1] += gz[0] + gz[7];
      store8o<BF>(Aimg + (L - 1) * kImg, poff(pp), gz);
    }
    if (tid == 0) {
      float s = 0.f;
      for (int p = 0; p < kTPts; ++p) s += seeds[8 * p] + seeds[8 * p + 7];
      gbo += s;
    }
    fence_proxy_async();
    __syncthreads();

    // ---- backward through the hidden GEMMs g = NG .. 1
#pragma unroll 1
    for (int g = NG; g >= 1; --g) {
      if (tid == 0) {
        fence_after_sync();
        const uint32_t wa = smem_u32(Wimg + (g - 1) * kImg);
        const uint32_t gzb = smem_u32(Aimg + g * kImg);        // gz of act[g]
        const uint32_t ain = smem_u32(Aimg + (g - 1) * kImg);  // act[g-1]
#pragma unroll
        for (int k = 0; k < 8; ++k)  // input gradient: D = W^T gz
          mma_f16(d_tm, desc_mnmajor(wa, k), desc_mnmajor(gzb, k), id_dgr, k > 0);
#pragma unroll
        for (int k = 0; k < 8; ++k)  // weight gradient: Wacc += gz act^T
          mma_f16(tmem + 128u * g, desc_kmajor(gzb, k), desc_kmajor(ain, k), id_wgr,
                  (k > 0 || !first_tile) ? 1u : 0u);
        mma_commit(smem_u32(bar_mma));
      }
      if (!wait_mma()) {
        aborted = true;
        break;
      }
      unsigned char* img = Aimg + (g - 1) * kImg;  // state of act[g-1]
      float G[32];
      tmem_ld32(d_tm + lane_base + col0, G);
#pragma unroll
      for (int j = 0; j < kPPT; ++j) {
        const int p = 4 * cg + j;
        float st[8];
        load8o<BF>(img, poff(j), st);
        const float* Gp = G + 8 * j;
        const float t = st[0], s0 = fmaf(-t, t, 1.f);
        float gz[8];
        float gzc = s0 * Gp[0];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          gzc += tanh_stencil_bwd(t, s0, st[1 + i], st[4 + i], Gp[1 + i], Gp[4 + i], hs, h2s,
                                  ihs, ih2s, gz[1 + i], gz[4 + i]);
        gz[0] = gzc;
        gz[7] = fmaf(-st[7], st[7], 1.f) * Gp[7];
        if (g > 1) {
          const float gsum = gz[0] + gz[7];
#pragma unroll
          for (int i = 0; i < NG; ++i) gbh[i] += (g - 2 == i) ? gsum : 0.f;
          store8o<BF>(img, poff(j), gz);
        } else {
          // d del_i / d W1[u][i] = h (unscaled columns) or 1 (scaled)
          const PRec pi = pr[p];
          const float dd = SCALED ? 1.f : P.hf;
          gW1[0] += fmaf(gz[0], pi.x, fmaf(gz[7], pi.gx, gz[4] * dd));
          gW1[1] += fmaf(gz[0], pi.y, fmaf(gz[7], pi.gy, gz[5] * dd));
          gW1[2] += fmaf(gz[0], pi.z, fmaf(gz[7], pi.gz, gz[6] * dd));
          gb1 += gz[0] + gz[7];
        }
      }
      fence_before_sync();
      fence_proxy_async();
      __syncthreads();
    }
    first_tile = false;
  }

  if (!aborted && train && cur_net >= 0) flush(cur_net);
  double lsum = (double)loss_acc + loss_acc_d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) loss_red[w] = lsum;
  fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int ww = 0; ww < 16; ++ww) s += loss_red[ww];
    if (a.mode != MODE_CUT_FWD) a.loss_part[blockIdx.x] = s;
    if (train) {
      a.gpart_flag[2 * blockIdx.x] = aborted ? 0 : wrote0;
      a.gpart_flag[2 * blockIdx.x + 1] = aborted ? 0 : wrote1;
    }
  }
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, NCOLS);
}

template <int L, bool BF, bool FAST>
static cudaError_t launch_tc_t(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st) {
  constexpr bool SCALED = !BF;  // FP16 operands need the 1/h^2, 1/h column scaling
  const size_t smem = tc_smem_bytes(L);
  cudaError_t e = cudaFuncSetAttribute(k_step_tc<L, BF, FAST, SCALED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_step_tc<L, BF, FAST, SCALED><<<grid, 512, smem, st>>>(P, a);
  return cudaGetLastError();
}

cudaError_t launch_step_tc(const ProbDev& P, const StepArgs& a, int grid, int prec, cudaStream_t st) {
  if (P.H != 128) return cudaErrorInvalidValue;
  // The tanh/reciprocal of the epilogue run on the SFU (tanh.approx, rcp.approx,
  // relative error ~2^-11): every value they produce is rounded to BF16
  // (2^-9) before the next GEMM, so they do not add an error class.  The
  // fine-h mode (FP64 rows) keeps the accurate functions: there the BF16
  // rounding alone already uses most of the gradient tolerance.
  if (prec == NBM_PREC_BF16 && !P.fp64) {
    if (P.L == 2) return launch_tc_t<2, true, true>(P, a, grid, st);
    if (P.L == 3) return launch_tc_t<3, true, true>(P, a, grid, st);
    if (P.L == 4) return launch_tc_t<4, true, true>(P, a, grid, st);
  }
  if (prec == NBM_PREC_BF16) {
    if (P.L == 2) return launch_tc_t<2, true, false>(P, a, grid, st);
    if (P.L == 3) return launch_tc_t<3, true, false>(P, a, grid, st);
    if (P.L == 4) return launch_tc_t<4, true, false>(P, a, grid, st);
  }
  return cudaErrorInvalidValue;
}


}  // namespace nbm
