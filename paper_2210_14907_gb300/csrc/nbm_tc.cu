// nbm_tc.cu -- the mixed-precision fused NBM step on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators), arXiv 2210.14907 Sec. 3 / Fig. 2.
//
// One persistent CTA per SM, 16 warps in two groups of 8.  Each group owns a
// half-tile: 8 collocation points x 8 columns (centre value, symmetric and
// antisymmetric stencil increments of the three axes in difference form, and
// the interface-point value of cut cells), i.e. 64 GEMM columns, with its own
// operand images and its own 64 TMEM accumulator columns.  The groups run
// independently, so that one group's epilogue (CUDA cores) overlaps the other
// group's GEMMs (tensor pipe).  Every hidden layer is one 128 x 64 x 128
// product D[unit][col] = W[unit][k] A[k][col] with 16-bit operands and FP32
// accumulation in TMEM; warp w reads TMEM lanes 32(w%4).. (one unit per
// thread) for 32 columns (4 points).  The epilogue applies the tanh stencil
// layer in FP32 and writes the next 16-bit operand image to shared memory.
// The first layer (K = 3), the output layer (H -> 1, a warp
// transpose-reduction), the residual rows and the seeds stay FP32 (FP64 rows
// on request).  In the BF16 training path the epilogues' FP32 arithmetic runs
// on packed pairs (add/mul/fma .f32x2: two points per instruction, each
// rounded as its scalar form).  The backward reuses the stored images: per hidden layer one
// input-gradient MMA (W^T gz, into the group's D columns) and one
// weight-gradient MMA (gz A^T, K = 64) accumulated across all half-tiles of
// the CTA in shared TMEM columns, in a fixed order of the half-tiles, so the
// weight gradient never leaves the SM until the CTA's partial is written once
// per network and is bitwise reproducible.
//
// Shared memory: (L-1) weight images of 32 KB + 2 x L operand images of 16 KB.
// TMEM: 2 x 64 columns for D + 128 per hidden layer for the weight gradient.
// Every wait is bounded.  The group barrier that ends each phase agrees on an
// abort; an aborted CTA gives its MMAs and copies in flight a short bounded
// wait before it frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nbm_device.cuh"
#include "nbm_tc_ptx.cuh"
#include "nbm_f32x2.cuh"

namespace nbm {

using namespace tc;

namespace {

constexpr int kHP = 8;        // points per half-tile (one warp group)
constexpr int kImg = 32768;   // 128 x 128 16-bit weight image
constexpr int kImgH = 16384;  // 128 x 64 16-bit operand image of a half-tile
constexpr int kMisc = 2048;
constexpr int kPrefetchT = 224;  // rank in the group of the thread that fetches tile records

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

// Sum of wo * x[0..31] over the 32 lanes of the warp: on return lane l holds
// the sum of column l (recursive halving, one exchange per value; the scaling
// is folded into the first halving so that x stays intact for the backward).
__device__ __forceinline__ void warp_transpose_reduce32(const float (&x)[32], float wo, int lane,
                                                        float& s) {
  float v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const bool hi = lane & 16;
    const float keep = wo * (hi ? x[16 + i] : x[i]), send = wo * (hi ? x[i] : x[16 + i]);
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

// Two points' tanh stencil layer on packed FP32 pairs (unscaled columns, every
// lane's symmetric increments small): the arithmetic of tanh_stencil_fwd's
// series path, operation for operation.
template <bool FAST>
__device__ __forceinline__ void tanh_stencil_fwd_pair(F2 T, F2 NT, F2 S0, F2 MU, F2 DE, F2& M,
                                                      F2& D, bool small_de = false) {
  const bool sde = !FAST && small_de;  // the series of tanh d and 1/(1-x) (accurate path)
  F2 TD;
  if (sde) {
    const F2 d2 = mul2(DE, DE);
    TD = mul2(DE, fma2(d2, fma2(d2, f2s(2.0f / 15.0f), f2s(-1.0f / 3.0f)), f2s(1.0f)));
  } else {
    float dA, dB;
    f2get(DE, dA, dB);
    TD = f2(act_tanh<FAST>(dA), act_tanh<FAST>(dB));
  }
  const F2 poly = fma2(fma2(T, T, f2s(-1.0f / 3.0f)), mul2(MU, MU), fma2(NT, MU, f2s(1.0f)));
  const F2 dm = mul2(mul2(S0, MU), poly);
  const F2 tw = add2(T, dm);
  const F2 ntw = mul2(tw, f2s(-1.0f));
  const F2 sw = fma2(ntw, tw, f2s(1.0f));
  const F2 td2 = mul2(TD, TD);
  F2 r2;
  if (sde) {
    const F2 x = mul2(mul2(tw, tw), td2);  // 1/(1-x) = 1 + x (1 + x (1 + x))
    r2 = fma2(x, fma2(x, add2(x, f2s(1.0f)), f2s(1.0f)), f2s(1.0f));
  } else {
    float eA, eB;
    f2get(fma2(add2(sw, f2s(-1.0f)), td2, f2s(1.0f)), eA, eB);
    r2 = f2(rcp<FAST>(eA), rcp<FAST>(eB));
  }
  const F2 k = mul2(sw, r2);
  M = fma2(mul2(ntw, td2), k, dm);
  D = mul2(k, TD);
}

// Two points' adjoint of one stencil axis (unscaled columns): the arithmetic of
// tanh_stencil_bwd on packed pairs.
__device__ __forceinline__ F2 tanh_stencil_bwd_pair(F2 T, F2 S0, F2 MO, F2 DO, F2 GM, F2 GD,
                                                    F2& gmu, F2& gdel) {
  const F2 P = mul2(fma2(mul2(T, f2s(2.0f)), MO, fma2(MO, MO, mul2(DO, DO))), f2s(-1.0f));
  const F2 Q = mul2(mul2(DO, f2s(-2.0f)), add2(T, MO));
  const F2 S = add2(S0, P);
  const F2 qgd = mul2(Q, GD);
  gmu = fma2(S, GM, qgd);
  gdel = fma2(Q, GM, mul2(S, GD));
  return fma2(P, GM, qgd);
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
  pdl_enter();
  constexpr int H = 128;
  constexpr int NG = L - 1;  // hidden GEMM layers
  constexpr int kPPT = 4;    // points per thread (8 warps = 4 lane quadrants x 2 column groups)
  constexpr uint32_t NCOLS = (NG + 1) * 128 <= 256 ? 256 : 512;
  // Two hidden GEMMs use 384 of the 512 columns: the forward GEMMs then take
  // their weights (the A operand) from the last 128, which spares each of them
  // the 32 KB weight read from shared memory.
  constexpr bool kWTmem = NG == 2;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int grp = tid >> 8, gtid = tid & 255;  // warp group and rank in it
  const int q = w & 3, cgl = (w >> 2) & 1;     // TMEM lane quadrant, column group
  const int u = 32 * q + lane;                 // unit (TMEM lane) of this thread
  const int col0 = 32 * cgl;                   // first of its 32 columns (points 4cgl .. 4cgl+3)
  const uint32_t gbar = 1u + (uint32_t)grp;    // named barrier of the group
  unsigned char* Wimg = sm;                                   // [NG][32 KB]
  unsigned char* Aimg = sm + NG * kImg + grp * L * kImgH;     // this group's [L][16 KB]
  unsigned char* misc = sm + NG * kImg + 2 * L * kImgH;
  uint64_t* bar_w = (uint64_t*)misc;
  uint64_t* bar_mma = (uint64_t*)(misc + 8 + 8 * grp);
  uint64_t* bar_p = (uint64_t*)(misc + 24 + 8 * grp);
  uint32_t* tslot = (uint32_t*)(misc + 40);
  int* done_cnt = (int*)(misc + 44);               // [2] backward MMA phases completed
  volatile int* abort_f = (volatile int*)(misc + 52);
  float* gbo_red = (float*)(misc + 56);            // [2]
  PRec* pbuf = (PRec*)(misc + 64 + grp * 512);     // this group's [2][8] tile records
  float* seeds = (float*)(misc + 1088 + grp * 256);  // this group's 64 seeds
  double* loss_red = (double*)(misc + 1600);         // 16 doubles
  float* red = (float*)(Aimg + (L - 1) * kImgH);     // [4][64] scratch (forward end only)

  // image byte offset of (unit u, point 4cgl + j): the row part is fixed per
  // thread, the 16-byte chunk is ((4cgl + j) mod 8) xor (u mod 8)
  const uint32_t row_off = (uint32_t)((u >> 3) * 1024 + (u & 7) * 128);
  const uint32_t pbase = (uint32_t)(cgl << 2), uxor = (uint32_t)(u & 7);
  auto poff = [&](int j) -> uint32_t { return row_off + ((((pbase + j) ^ uxor) & 7u) << 4); };
  const bool train = a.mode == MODE_TRAIN;
  const float hs = SCALED ? P.hf : 1.f, h2s = SCALED ? P.h2f : 1.f;
  const float ihs = SCALED ? P.inv_hf : 1.f, ih2s = SCALED ? P.inv_h2f : 1.f;
  const uint32_t id_fwd = idesc_f16_n(BF, false, true, kHP * 8);
  const uint32_t id_dgr = idesc_f16_n(BF, true, true, kHP * 8);
  const uint32_t id_wgr = idesc_f16_n(BF, false, false, 128);

  if (tid == 0) {
    mbar_init(smem_u32(bar_w), 1);
    mbar_init(smem_u32((uint64_t*)(misc + 8)), 1);
    mbar_init(smem_u32((uint64_t*)(misc + 16)), 1);
    mbar_init(smem_u32((uint64_t*)(misc + 24)), 1);
    mbar_init(smem_u32((uint64_t*)(misc + 32)), 1);
    *abort_f = 0;
    fence_mbar_init();
  }
  if (w == 0) tmem_alloc(smem_u32(tslot), NCOLS);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t d_tm = tmem + 64u * (uint32_t)grp;  // this group's D: 64 columns
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  uint32_t ph_w = 0, ph_mma = 0, ph_p = 0;
  bool aborted = false;

  // half-tiles of 8 points: net 0 (or the cut list for net 0), then net 1
  const int nm = a.counters[0], np = a.counters[1], nc = a.counters[2];
  const bool cutfwd = a.mode == MODE_CUT_FWD;
  const int T0 = cutfwd ? (nc + kHP - 1) / kHP : (nm + kHP - 1) / kHP;
  const int T = cutfwd ? 2 * T0 : T0 + (np + kHP - 1) / kHP;
  const int tb = (int)((int64_t)blockIdx.x * T / gridDim.x);
  const int te = (int)((int64_t)(blockIdx.x + 1) * T / gridDim.x);

  // tile records: one 256-byte bulk copy per half-tile, fetched a tile ahead
  auto prefetch = [&](int tau, int buf) {
    // the record lists are padded to 16 per list; net 1 starts after net 0's padding
    const PRec* src = cutfwd ? a.rec_cut + (int64_t)kHP * (tau < T0 ? tau : tau - T0)
                    : tau < T0 ? a.rec + (int64_t)kHP * tau
                               : a.rec + 16 * (int64_t)((nm + 15) / 16) + (int64_t)kHP * (tau - T0);
    fence_proxy_async();
    mbar_expect_tx(smem_u32(bar_p), kHP * sizeof(PRec));
    bulk_g2s(smem_u32(pbuf + kHP * buf), src, kHP * sizeof(PRec), smem_u32(bar_p));
  };

  // per-net constants of this thread's unit
  // (first-layer weights and hidden biases are read where they are used, from
  // the L1-resident parameter vector: registers are short at the output stage)
  float wo = 0.f, bo = 0.f;
  const float* th = a.params;
  // gradient accumulators of the small parameters
  float gW1[3] = {0.f, 0.f, 0.f}, gb1 = 0.f, gbh[NG], gwo = 0.f, gbo = 0.f;
#pragma unroll
  for (int g = 0; g < NG; ++g) gbh[g] = 0.f;
  float loss_acc = 0.f;     // per-thread FP32 sum of r^2 (FP32 rows)
  double loss_acc_d = 0.0;  // per-thread FP64 sum of r^2 (FP64 rows)
  int wrote0 = 0, wrote1 = 0;

  // Completion of this group's MMA phase; false (and the CTA-wide abort flag
  // set) if the wait ran out or either group gave up.
  // Bounded wait for the group's MMA phase (no group barrier: the one that ends
  // the phase's epilogue agrees on an abort; until then a thread whose wait
  // gave up only computes on undefined accumulator values).
  auto wait_mma = [&]() -> bool {
    const bool ok = mbar_wait_bounded(smem_u32(bar_mma), ph_mma);
    if (ok) ph_mma ^= 1u;  // a wait that gave up leaves the phase for the exit drain
    fence_after_sync();
    return ok;
  };
  // The group barrier that ends an MMA phase's epilogue.  It orders the
  // epilogue's shared-memory images before the next MMA, keeps every thread
  // within one phase of bar_mma, and agrees on an abort (a wait that gave up,
  // or the abort flag).  False: abort.
  auto end_phase = [&](bool ok) -> bool {
    fence_before_sync();
    fence_proxy_async();
    const bool bad = named_sync_or(gbar, 256, !ok || *abort_f != 0);
    if (bad && gtid == 0) {
      if (!ok) atomicOr(a.status, 2);
      *abort_f = 1;
    }
    return !bad;
  };
  // Gate of one MMA phase, run by the group's first thread before it issues.
  // `order` > 0: wait until the other group has completed that many backward
  // phases first (the weight-gradient accumulators are shared, and a fixed
  // accumulation order keeps the result bitwise reproducible).  Returns false
  // when it gives up; the thread then arrives on the barrier itself, so that
  // its group wakes up and sees the abort flag.
  auto gate = [&](int order) -> bool {
    bool ok = true;
    if (order > 0) {
      const int* other = done_cnt + (grp ^ 1);
      if (ld_acquire_s32(other) < order) {
        const long long t0 = clock64();
        while (ld_acquire_s32(other) < order) {
          if (*abort_f) { ok = false; break; }
          if (clock64() - t0 > 4000000000LL) {
            atomicOr(a.status, 2);
            ok = false;
            break;
          }
          __nanosleep(20);
        }
      }
    }
    if (!ok || *abort_f) {
      *abort_f = 1;
      mbar_arrive(smem_u32(bar_mma));
      return false;
    }
    fence_after_sync();
    return true;
  };

  auto flush = [&](int net) {
    // weight gradients of the hidden layers straight from TMEM: warp w reads
    // lanes 32(w%4).. and columns 32(w/4)..
    const int cgf = w >> 2;
    float* gp = a.gpart + ((int64_t)blockIdx.x * 2 + net) * P.gstride;
#pragma unroll 1
    for (int g = 1; g <= NG; ++g) {
      float* dst = gp + 4 * H + (int64_t)(g - 1) * (H * H + H) + (int64_t)u * H + 32 * cgf;
      float v[32];
      tmem_ld32(tmem + 128u * g + lane_base + 32u * cgf, v);
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    }
    // small parameters: the four column groups of a unit are combined in smem
    float* stage = (float*)(sm + NG * kImg);  // [4 column groups][128 units][8]
    if (gtid == 0) gbo_red[grp] = gbo;
    fence_before_sync();
    __syncthreads();
    {
      float* s = stage + (cgf * 128 + u) * 8;
      s[0] = gW1[0]; s[1] = gW1[1]; s[2] = gW1[2]; s[3] = gb1; s[4] = gwo;
#pragma unroll
      for (int g = 0; g < NG; ++g) s[5 + g] = gbh[g];
    }
    __syncthreads();
    if (cgf == 0) {
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
      if (tid == 0) gp[oo + H] = gbo_red[0] + gbo_red[1];
    }
    gW1[0] = gW1[1] = gW1[2] = gb1 = gwo = gbo = 0.f;
#pragma unroll
    for (int g = 0; g < NG; ++g) gbh[g] = 0.f;
    if (net) wrote1 = 1; else wrote0 = 1;
    __syncthreads();
  };

  int kk = 0;  // half-tiles of this group so far (record buffer parity)
#pragma unroll 1
  for (int net = 0; net < 2; ++net) {
    const int s0 = net == 0 ? tb : (tb > T0 ? tb : T0);
    const int s1 = net == 0 ? (te < T0 ? te : T0) : te;
    if (s0 >= s1) continue;  // the same in every thread of the CTA
    // stage this network's hidden weights (bulk copy engine); the two groups
    // take the segment's half-tiles alternately, group 0 the first
    if (tid == 0) {
      done_cnt[0] = 0;
      done_cnt[1] = 0;
      const unsigned char* src = (const unsigned char*)a.wtc + (int64_t)net * NG * kImg;
      mbar_expect_tx(smem_u32(bar_w), NG * kImg);
      for (int g = 0; g < NG; ++g)
        bulk_g2s(smem_u32(Wimg + g * kImg), src + (int64_t)g * kImg, kImg, smem_u32(bar_w));
    }
    if (gtid == kPrefetchT && s0 + grp < s1) prefetch(s0 + grp, kk & 1);
    {
      th = a.params + net * P.p_net;
      const int64_t oo = 4 * H + (int64_t)NG * (H * H + H);
      wo = th[oo + u];
      bo = th[oo + H];
    }
    {
      const bool ok = mbar_wait_bounded(smem_u32(bar_w), ph_w);
      if (ok) ph_w ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.status, 2);
        aborted = true;
        break;
      }
    }
    if constexpr (kWTmem) {
      // this network's forward weights into TMEM: layer g in columns 384 +
      // 64 (g-1) .., unit u (row of W) in lane u, W[u][2c] and W[u][2c+1] in
      // column c; the previous segment's GEMMs have all completed
      if (w < 4) stage_weights_tmem(Wimg, kImg, tmem + ((uint32_t)(32 * w) << 16) + 384u, u, NG);
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
    }

    int tile_i = 0;  // index of the half-tile among this group's tiles of the segment
#pragma unroll 1
    for (int tau = s0 + grp; tau < s1; tau += 2, ++tile_i, ++kk) {
      // layer-1 weights of this thread's unit, loaded while the records arrive
      const float w1[3] = {th[3 * u], th[3 * u + 1], th[3 * u + 2]};
      const float b1 = th[3 * H + u];
      // ---- tile records (prefetched during the previous tile)
      {
        const bool ok = mbar_wait_bounded(smem_u32(bar_p), ph_p);
        if (ok) ph_p ^= 1u;
        if (named_sync_or(gbar, 256, !ok || *abort_f != 0)) {
          if (gtid == 0) {
            if (!ok) atomicOr(a.status, 2);
            *abort_f = 1;
          }
          aborted = true;
          break;
        }
        if (gtid == kPrefetchT && tau + 2 < s1) prefetch(tau + 2, (kk + 1) & 1);
      }
      const PRec* pr = pbuf + kHP * (kk & 1);
      // seeds of cut points (from the cut-row kernel): copied into the seed
      // buffer now (asynchronously), used after the forward
      if (train && gtid < 8 * kHP) {
        const PRec& pc = pr[gtid >> 3];
        if (pc.pt >= 0 && pc.cutj >= 0)
          cp_async4(smem_u32(seeds + gtid),
                    a.cut_seed + (int64_t)(pc.cutj >> 1) * 16 + net * 8 + (gtid & 7));
      }

      // ---- layer 1 (3 -> H) in FP32; exact increments mu = 0, del_i = h W1[u][i]
      {
        const float dl1[3] = {SCALED ? w1[0] : w1[0] * P.hf, SCALED ? w1[1] : w1[1] * P.hf,
                              SCALED ? w1[2] : w1[2] * P.hf};
        if constexpr (!SCALED) {
          // two points per packed FP32 instruction; tanh(h W1[u][i]) depends on the
          // unit only
          float Td[3];
          // accurate path with small increments h W1[u][i] in every lane: the series
          bool sd1 = false;
          if constexpr (!FAST)
            sd1 = __all_sync(0xffffffffu, fmaxf(fabsf(dl1[0]), fmaxf(fabsf(dl1[1]), fabsf(dl1[2]))) <=
                                              kSmallDelAccurate);
#pragma unroll
          for (int i = 0; i < 3; ++i) Td[i] = sd1 ? tanh_small(dl1[i]) : act_tanh<FAST>(dl1[i]);
#pragma unroll
          for (int pp = 0; pp < kPPT; pp += 2) {
            const PRec pa = pr[4 * cgl + pp], pb = pr[4 * cgl + pp + 1];
            const F2 W0 = f2s(w1[0]), W1 = f2s(w1[1]), W2 = f2s(w1[2]), B1 = f2s(b1);
            float zA, zB;
            f2get(fma2(W0, f2(pa.x, pb.x), fma2(W1, f2(pa.y, pb.y), fma2(W2, f2(pa.z, pb.z), B1))),
                  zA, zB);
            const F2 T = f2(act_tanh<FAST>(zA), act_tanh<FAST>(zB));
            const F2 NT = mul2(T, f2s(-1.0f));
            const F2 SW = fma2(NT, T, f2s(1.0f));
            const F2 NTT = mul2(NT, T);
            const F2 NTS = mul2(NT, SW);
            float oA[8], oB[8];
            f2get(T, oA[0], oB[0]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const F2 TD = f2s(Td[i]), TD2 = mul2(TD, TD);
              F2 R2;
              if (sd1) {  // 1 / (1 - t^2 Td^2) by its series
                const F2 x = mul2(mul2(T, T), TD2);
                R2 = fma2(x, fma2(x, add2(x, f2s(1.0f)), f2s(1.0f)), f2s(1.0f));
              } else {
                float eA, eB;
                f2get(fma2(NTT, TD2, f2s(1.0f)), eA, eB);
                R2 = f2(rcp<FAST>(eA), rcp<FAST>(eB));
              }
              f2get(mul2(mul2(NTS, TD2), R2), oA[1 + i], oB[1 + i]);
              f2get(mul2(mul2(SW, TD), R2), oA[4 + i], oB[4 + i]);
            }
            const bool ja = pa.cutj >= 0 && (pa.cutj & 1), jb = pb.cutj >= 0 && (pb.cutj & 1);
            oA[7] = ja ? act_tanh<FAST>(fmaf(w1[0], pa.gx, fmaf(w1[1], pa.gy, fmaf(w1[2], pa.gz, b1))))
                       : 0.f;
            oB[7] = jb ? act_tanh<FAST>(fmaf(w1[0], pb.gx, fmaf(w1[1], pb.gy, fmaf(w1[2], pb.gz, b1))))
                       : 0.f;
            store8o<BF>(Aimg, poff(pp), oA);
            store8o<BF>(Aimg, poff(pp + 1), oB);
          }
        } else {
#pragma unroll
        for (int pp = 0; pp < kPPT; ++pp) {
          const int p = 4 * cgl + pp;
          const PRec pi = pr[p];
          const float z = fmaf(w1[0], pi.x, fmaf(w1[1], pi.y, fmaf(w1[2], pi.z, b1)));
          const float t = act_tanh<FAST>(z);
          float o[8];
          o[0] = t;
#pragma unroll
          for (int i = 0; i < 3; ++i) tanh_stencil_fwd0<FAST>(t, dl1[i], hs, ihs, ih2s, o[1 + i], o[4 + i]);
          const bool jump = pi.cutj >= 0 && (pi.cutj & 1);
          o[7] = jump ? act_tanh<FAST>(fmaf(w1[0], pi.gx, fmaf(w1[1], pi.gy, fmaf(w1[2], pi.gz, b1))))
                      : 0.f;
          store8o<BF>(Aimg, poff(pp), o);
        }
        }
      }
      fence_proxy_async();
      named_sync(gbar, 256);

      // ---- hidden layers on the tensor cores: D[unit][col] = W[unit][k] A[k][col]
      float last[32];
#pragma unroll 1
      for (int g = 1; g <= NG; ++g) {
        // the layer's bias, loaded while the GEMM runs
        const float bb = th[4 * H + (g - 1) * (H * H + H) + H * H + u];
        if (gtid == 0 && gate(0)) {
          const uint32_t ab = smem_u32(Aimg + (g - 1) * kImgH);
          if constexpr (kWTmem) {
            const uint32_t wt = tmem + 384u + 64u * (uint32_t)(g - 1);
#pragma unroll
            for (int k = 0; k < 8; ++k)
              mma_f16_ta(d_tm, wt + 8u * (uint32_t)k, desc_mnmajor(ab, k), id_fwd, k > 0);
          } else {
            const uint32_t wa = smem_u32(Wimg + (g - 1) * kImg);
#pragma unroll
            for (int k = 0; k < 8; ++k)
              mma_f16(d_tm, desc_kmajor(wa, k), desc_mnmajor(ab, k), id_fwd, k > 0);
          }
          mma_commit(smem_u32(bar_mma));
        }
        const bool ok_w = wait_mma();
        float acc[32];
        tmem_ld32(d_tm + lane_base + col0, acc);
        if constexpr (!SCALED) {
          // two points per packed FP32 instruction
          constexpr float kSmall = FAST ? kSmallMu : kSmallMuAccurate;
#pragma unroll
          for (int jp = 0; jp < kPPT; jp += 2) {
            const float* cA = acc + 8 * jp;
            const float* cB = cA + 8;
            float oA[8], oB[8];
            const float tA = act_tanh<FAST>(cA[0] + bb), tB = act_tanh<FAST>(cB[0] + bb);
            oA[0] = tA;
            oB[0] = tB;
            const bool smA = __all_sync(
                0xffffffffu, fmaxf(fabsf(cA[1]), fmaxf(fabsf(cA[2]), fabsf(cA[3]))) <= kSmall);
            const bool smB = __all_sync(
                0xffffffffu, fmaxf(fabsf(cB[1]), fmaxf(fabsf(cB[2]), fabsf(cB[3]))) <= kSmall);
            // accurate path: antisymmetric increments small in every lane (their series)
            bool sdA = false, sdB = false;
            if constexpr (!FAST) {
              sdA = __all_sync(0xffffffffu, fmaxf(fabsf(cA[4]), fmaxf(fabsf(cA[5]), fabsf(cA[6]))) <=
                                                kSmallDelAccurate);
              sdB = __all_sync(0xffffffffu, fmaxf(fabsf(cB[4]), fmaxf(fabsf(cB[5]), fabsf(cB[6]))) <=
                                                kSmallDelAccurate);
            }
            if (smA && smB) {
              const F2 T = f2(tA, tB), NT = mul2(T, f2s(-1.0f));
              const F2 S0 = fma2(NT, T, f2s(1.0f));
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                F2 M, D;
                tanh_stencil_fwd_pair<FAST>(T, NT, S0, f2(cA[1 + i], cB[1 + i]),
                                            f2(cA[4 + i], cB[4 + i]), M, D, sdA && sdB);
                f2get(M, oA[1 + i], oB[1 + i]);
                f2get(D, oA[4 + i], oB[4 + i]);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                tanh_stencil_fwd<FAST>(tA, cA[1 + i], cA[4 + i], 1.f, 1.f, 1.f, 1.f, oA[1 + i],
                                       oA[4 + i], smA, sdA);
                tanh_stencil_fwd<FAST>(tB, cB[1 + i], cB[4 + i], 1.f, 1.f, 1.f, 1.f, oB[1 + i],
                                       oB[4 + i], smB, sdB);
              }
            }
            // column 7 (the interface point) only matters for cut cells with a jump
            // row; elsewhere its seeds are 0.  The accurate path skips its tanh there
            // (0, as layer 1 leaves it); in the SFU path the test cost more than it
            // saved (C2 6 % slower), so that path keeps computing it.
            if constexpr (FAST) {
              oA[7] = act_tanh<FAST>(cA[7] + bb);
              oB[7] = act_tanh<FAST>(cB[7] + bb);
            } else {
              const PRec& qa = pr[4 * cgl + jp];
              const PRec& qb = pr[4 * cgl + jp + 1];
              oA[7] = (qa.cutj >= 0 && (qa.cutj & 1)) ? act_tanh<FAST>(cA[7] + bb) : 0.f;
              oB[7] = (qb.cutj >= 0 && (qb.cutj & 1)) ? act_tanh<FAST>(cB[7] + bb) : 0.f;
            }
            if (g < NG) {
              store8o<BF>(Aimg + g * kImgH, poff(jp), oA);
              store8o<BF>(Aimg + g * kImgH, poff(jp + 1), oB);
            } else {
#pragma unroll
              for (int c2 = 0; c2 < 8; ++c2) {
                last[8 * jp + c2] = oA[c2];
                last[8 * jp + 8 + c2] = oB[c2];
              }
            }
          }
        } else {
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
          const float* c = acc + 8 * j;
          float o[8];
          const float t = act_tanh<FAST>(c[0] + bb);
          o[0] = t;
          // symmetric increments small in every lane: their series (see tanh_stencil_fwd)
          const bool small_mu =
              FAST && __all_sync(0xffffffffu,
                                 fmaxf(fabsf(c[1]), fmaxf(fabsf(c[2]), fabsf(c[3]))) * h2s <= kSmallMu);
#pragma unroll
          for (int i = 0; i < 3; ++i)
            tanh_stencil_fwd<FAST>(t, c[1 + i], c[4 + i], hs, h2s, ihs, ih2s, o[1 + i], o[4 + i],
                                   small_mu);
          o[7] = act_tanh<FAST>(c[7] + bb);
          if (g < NG) {
            store8o<BF>(Aimg + g * kImgH, poff(j), o);
          } else {
#pragma unroll
            for (int c2 = 0; c2 < 8; ++c2) last[8 * j + c2] = o[c2];
          }
        }
        }
        if (!end_phase(ok_w)) {
          aborted = true;
          break;
        }
      }
      if (aborted) break;

      // ---- output layer (H -> 1) in FP32: sum over the 32 units of the warp,
      // then over the four lane quadrants
      {
        float s;
        warp_transpose_reduce32(last, wo, lane, s);  // lane l: column col0 + l
        red[q * 64 + col0 + lane] = s;
      }
      if (train && gtid < 8 * kHP) cp_async_wait_all();
      named_sync(gbar, 256);
      // ---- output columns and residual rows: lane c of the 8 lanes
      // gtid = 8 p + c of the group's first two warps takes column c of point
      // p, and the point's row is spread over its 8 lanes
      // (uncut_residual_lanes: one face per lane, sums by shuffles), so the
      // row's dependency chain runs on 8 lanes instead of 1.  FP64 rows only
      // occur in the accurate (!FAST) instances.  The fast four-layer
      // instance keeps one thread per point (uncut_residual_pt): there the
      // lane rows cost registers elsewhere and made the kernel 4 % slower.
      constexpr bool kLaneRows = !FAST || L <= 3;
      if (kLaneRows && gtid < 8 * kHP) {
        const int p = gtid >> 3, c = gtid & 7;
        const unsigned gmask = 0xFFu << (gtid & 24);
        float oc = red[8 * p + c];
#pragma unroll
        for (int qq = 1; qq < 4; ++qq) oc += red[64 * qq + 8 * p + c];
        if (c == 0 || c == 7) oc += bo;
        const float csc = SCALED ? 1.f : (c >= 1 && c <= 3) ? P.inv_h2f
                                       : (c >= 4 && c <= 6) ? P.inv_hf : 1.f;
        oc *= csc;  // the scaled convention of the rows: U, Mt_i = M_i/h^2, Dt_i = D_i/h
        // U and the Mt, Dt columns of this lane's face axis (c / 2)
        const float Uc = __shfl_sync(gmask, oc, 0, 8);
        const float Mtc = __shfl_sync(gmask, oc, 1 + (c >> 1), 8);
        const float Dtc = __shfl_sync(gmask, oc, 4 + (c >> 1), 8);
        const PRec pi = pr[p];
        const bool valid = pi.pt >= 0, is_cut = pi.cutj >= 0;
        float* sdp = seeds + 8 * p;
        if (cutfwd) {
          if (valid) a.cut_out[(int64_t)(pi.cutj >> 1) * 16 + net * 8 + c] = oc;
        } else if (valid && !is_cut) {
          float sdc, r2;
          bool rows64 = false;
          if constexpr (!FAST) rows64 = P.fp64;
          if (rows64) {
            const double r2d = uncut_residual_lanes<double>(P, net, pi.x, pi.y, pi.z,
                                                            (double)pi.gx + (double)pi.gy, Uc, Mtc,
                                                            Dtc, (double)a.scale, c, gmask, sdc);
            if (c == 0) loss_acc_d += r2d;
            r2 = (float)r2d;
          } else {
            r2 = uncut_residual_lanes<float>(P, net, pi.x, pi.y, pi.z, pi.gx, Uc, Mtc, Dtc,
                                             a.scale, c, gmask, sdc);
            if (c == 0) loss_acc += r2;
          }
          if (c == 0 && a.r2_out) a.r2_out[pi.pt] = (P.level ? a.r2_out[pi.pt] : 0.f) + r2;
          sdp[c] = sdc * csc;  // seeds in this kernel's column convention
        } else if (valid && train) {
          sdp[c] *= csc;  // cut point: the seeds copied at the start of the tile, rescaled
        } else {
          sdp[c] = 0.f;
        }
      } else if (!kLaneRows && gtid < kHP) {
        // one thread per point (FP32 rows)
        const int p = gtid;
        float o[8];
        {
          const float4* r4 = reinterpret_cast<const float4*>(red) + 2 * p;
          float4 lo = r4[0], hi = r4[1];
#pragma unroll
          for (int qq = 1; qq < 4; ++qq) {
            const float4 l2 = r4[16 * qq], h2 = r4[16 * qq + 1];
            lo.x += l2.x; lo.y += l2.y; lo.z += l2.z; lo.w += l2.w;
            hi.x += h2.x; hi.y += h2.y; hi.z += h2.z; hi.w += h2.w;
          }
          o[0] = lo.x + bo; o[1] = lo.y; o[2] = lo.z; o[3] = lo.w;
          o[4] = hi.x; o[5] = hi.y; o[6] = hi.z; o[7] = hi.w + bo;
        }
        if (!SCALED) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            o[1 + i] *= P.inv_h2f;
            o[4 + i] *= P.inv_hf;
          }
        }
        const PRec pi = pr[p];
        const bool valid = pi.pt >= 0, is_cut = pi.cutj >= 0;
        float4* sd4 = reinterpret_cast<float4*>(seeds + 8 * p);
        if (cutfwd) {
          if (valid) {
            float4* co = reinterpret_cast<float4*>(a.cut_out + (int64_t)(pi.cutj >> 1) * 16 + net * 8);
            co[0] = make_float4(o[0], o[1], o[2], o[3]);
            co[1] = make_float4(o[4], o[5], o[6], o[7]);
          }
        } else if (valid && !is_cut) {
          float sd[8];
          const float r2 = uncut_residual_pt<float>(P, net, pi.x, pi.y, pi.z, pi.gx, o, a.scale, sd);
          loss_acc += r2;
          if (a.r2_out) a.r2_out[pi.pt] = (P.level ? a.r2_out[pi.pt] : 0.f) + r2;
          if (!SCALED) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              sd[1 + i] *= P.inv_h2f;
              sd[4 + i] *= P.inv_hf;
            }
          }
          sd4[0] = make_float4(sd[0], sd[1], sd[2], sd[3]);
          sd4[1] = make_float4(sd[4], sd[5], sd[6], sd[7]);
        } else if (valid && train) {
          // cut point: the seeds copied at the start of the tile, rescaled
          if (!SCALED) {
            float4 lo = sd4[0], hi = sd4[1];
            lo.y *= P.inv_h2f; lo.z *= P.inv_h2f; lo.w *= P.inv_h2f;
            hi.x *= P.inv_hf; hi.y *= P.inv_hf; hi.z *= P.inv_hf;
            sd4[0] = lo;
            sd4[1] = hi;
          }
        } else {
          sd4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
          sd4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      named_sync(gbar, 256);
      if (!train) continue;

      // ---- backward: adjoint of the last tanh layer (FP32 state in registers)
      if constexpr (!SCALED) {
        // two points per packed FP32 instruction
#pragma unroll
        for (int pp = 0; pp < kPPT; pp += 2) {
          float sA[8], sB[8];
          {
            const float4* s4 = reinterpret_cast<const float4*>(seeds + 8 * (4 * cgl + pp));
            const float4 a0 = s4[0], a1 = s4[1], b0 = s4[2], b1v = s4[3];
            sA[0] = a0.x; sA[1] = a0.y; sA[2] = a0.z; sA[3] = a0.w;
            sA[4] = a1.x; sA[5] = a1.y; sA[6] = a1.z; sA[7] = a1.w;
            sB[0] = b0.x; sB[1] = b0.y; sB[2] = b0.z; sB[3] = b0.w;
            sB[4] = b1v.x; sB[5] = b1v.y; sB[6] = b1v.z; sB[7] = b1v.w;
          }
          const float* stA = last + 8 * pp;
          const float* stB = stA + 8;
          F2 sw = mul2(f2(sA[0], sB[0]), f2(stA[0], stB[0]));
#pragma unroll
          for (int c = 1; c < 8; ++c) sw = fma2(f2(sA[c], sB[c]), f2(stA[c], stB[c]), sw);
          {
            float x, y;
            f2get(sw, x, y);
            gwo += x;
            gwo += y;
          }
          const F2 WO = f2s(wo);
          const F2 T = f2(stA[0], stB[0]);
          const F2 S0 = fma2(mul2(T, f2s(-1.0f)), T, f2s(1.0f));
          float gA[8], gB[8];
          F2 gzc = mul2(S0, mul2(WO, f2(sA[0], sB[0])));
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            F2 gm, gd;
            gzc = add2(gzc, tanh_stencil_bwd_pair(T, S0, f2(stA[1 + i], stB[1 + i]),
                                                  f2(stA[4 + i], stB[4 + i]),
                                                  mul2(WO, f2(sA[1 + i], sB[1 + i])),
                                                  mul2(WO, f2(sA[4 + i], sB[4 + i])), gm, gd));
            f2get(gm, gA[1 + i], gB[1 + i]);
            f2get(gd, gA[4 + i], gB[4 + i]);
          }
          f2get(gzc, gA[0], gB[0]);
          const F2 T7 = f2(stA[7], stB[7]);
          f2get(mul2(fma2(mul2(T7, f2s(-1.0f)), T7, f2s(1.0f)), mul2(WO, f2(sA[7], sB[7]))), gA[7],
                gB[7]);
          gbh[NG - 1] += gA[0] + gA[7];
          gbh[NG - 1] += gB[0] + gB[7];
          store8o<BF>(Aimg + (L - 1) * kImgH, poff(pp), gA);
          store8o<BF>(Aimg + (L - 1) * kImgH, poff(pp + 1), gB);
        }
      } else {
#pragma unroll
      for (int pp = 0; pp < kPPT; ++pp) {
        const int p = 4 * cgl + pp;
        float sd[8];
        {
          const float4 lo = *reinterpret_cast<const float4*>(seeds + 8 * p);
          const float4 hi = *reinterpret_cast<const float4*>(seeds + 8 * p + 4);
          sd[0] = lo.x; sd[1] = lo.y; sd[2] = lo.z; sd[3] = lo.w;
          sd[4] = hi.x; sd[5] = hi.y; sd[6] = hi.z; sd[7] = hi.w;
        }
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
        store8o<BF>(Aimg + (L - 1) * kImgH, poff(pp), gz);
      }
      }
      if (gtid == 0) {
        float s = 0.f;
        for (int p = 0; p < kHP; ++p) s += seeds[8 * p] + seeds[8 * p + 7];
        gbo += s;
      }
      fence_proxy_async();
      named_sync(gbar, 256);

      // ---- backward through the hidden GEMMs g = NG .. 1.  Phase n of this
      // group's tile i is n = i NG + (NG - g); group 0 issues it after group 1
      // completed its phase n - NG (tile i-1), group 1 after group 0 completed
      // phase n (tile i): the shared weight-gradient accumulators receive the
      // half-tiles in segment order.
#pragma unroll 1
      for (int g = NG; g >= 1; --g) {
        const int nph = tile_i * NG + (NG - g);
        const int order = grp == 0 ? nph - NG + 1 : nph + 1;
        const uint32_t acc_w = (grp == 0 && tile_i == 0) ? 0u : 1u;
        if (gtid == 0 && gate(order)) {
          const uint32_t wa = smem_u32(Wimg + (g - 1) * kImg);
          const uint32_t gzb = smem_u32(Aimg + g * kImgH);        // gz of act[g]
          const uint32_t ain = smem_u32(Aimg + (g - 1) * kImgH);  // act[g-1]
#pragma unroll
          for (int k = 0; k < 8; ++k)  // input gradient: D = W^T gz
            mma_f16(d_tm, desc_mnmajor(wa, k), desc_mnmajor(gzb, k), id_dgr, k > 0);
#pragma unroll
          for (int k = 0; k < kHP / 2; ++k)  // weight gradient: Wacc += gz act^T (K = 8 kHP)
            mma_f16(tmem + 128u * g, desc_kmajor(gzb, k), desc_kmajor(ain, k), id_wgr,
                    (k > 0 || acc_w) ? 1u : 0u);
          mma_commit(smem_u32(bar_mma));
        }
        const bool ok_w = wait_mma();
        if (gtid == 0 && ok_w) st_release_s32(done_cnt + grp, nph + 1);
        unsigned char* img = Aimg + (g - 1) * kImgH;  // state of act[g-1]
        float G[16];  // two points at a time: registers are short here
        float gzP[8];  // the second point's adjoint of a packed pair
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
          if ((j & 1) == 0) tmem_ld16(d_tm + lane_base + col0 + 8 * j, G);
          const int p = 4 * cgl + j;
          float st[8];
          load8o<BF>(img, poff(j), st);
          float gz[8];
          if constexpr (!SCALED) {
            if ((j & 1) == 0) {
              // this point and the next one on packed FP32 pairs
              float sB[8];
              load8o<BF>(img, poff(j + 1), sB);
              const F2 T = f2(st[0], sB[0]);
              const F2 S0 = fma2(mul2(T, f2s(-1.0f)), T, f2s(1.0f));
              F2 gzc = mul2(S0, f2(G[0], G[8]));
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                F2 gm, gd;
                gzc = add2(gzc, tanh_stencil_bwd_pair(T, S0, f2(st[1 + i], sB[1 + i]),
                                                      f2(st[4 + i], sB[4 + i]),
                                                      f2(G[1 + i], G[9 + i]),
                                                      f2(G[4 + i], G[12 + i]), gm, gd));
                f2get(gm, gz[1 + i], gzP[1 + i]);
                f2get(gd, gz[4 + i], gzP[4 + i]);
              }
              f2get(gzc, gz[0], gzP[0]);
              const F2 T7 = f2(st[7], sB[7]);
              f2get(mul2(fma2(mul2(T7, f2s(-1.0f)), T7, f2s(1.0f)), f2(G[7], G[15])), gz[7], gzP[7]);
            } else {
#pragma unroll
              for (int c2 = 0; c2 < 8; ++c2) gz[c2] = gzP[c2];
            }
          } else {
          const float* Gp = G + 8 * (j & 1);
          const float t = st[0], s0 = fmaf(-t, t, 1.f);
          float gzc = s0 * Gp[0];
#pragma unroll
          for (int i = 0; i < 3; ++i)
            gzc += tanh_stencil_bwd(t, s0, st[1 + i], st[4 + i], Gp[1 + i], Gp[4 + i], hs, h2s,
                                    ihs, ih2s, gz[1 + i], gz[4 + i]);
          gz[0] = gzc;
          gz[7] = fmaf(-st[7], st[7], 1.f) * Gp[7];
          }
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
        if (!end_phase(ok_w)) {
          aborted = true;
          break;
        }
      }
      if (aborted) break;
    }
    // ---- end of the segment: both groups are done with this network
    if (__syncthreads_or(aborted)) {
      aborted = true;
      break;
    }
    fence_after_sync();
    if (train) flush(net);
  }

  double lsum = (double)loss_acc + loss_acc_d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) loss_red[w] = lsum;
  fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int ww = 0; ww < 16; ++ww) s += loss_red[ww];
    if (!cutfwd) a.loss_part[blockIdx.x] = s;
    if (train) {
      a.gpart_flag[2 * blockIdx.x] = aborted ? 0 : wrote0;
      a.gpart_flag[2 * blockIdx.x + 1] = aborted ? 0 : wrote1;
    }
  }
  if (aborted) {
    // an MMA or record copy of this group may still be in flight: give it a
    // short bounded wait (about 1 ms) before TMEM and shared memory are released
    (void)mbar_wait_bounded(smem_u32(bar_mma), ph_mma, 2000000LL);
    (void)mbar_wait_bounded(smem_u32(bar_p), ph_p, 2000000LL);
    (void)mbar_wait_bounded(smem_u32(bar_w), ph_w, 2000000LL);
    fence_before_sync();
    __syncthreads();
  }
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, NCOLS);
}

// Diagnostics: one warp waits, with the bounded wait every kernel of the
// library uses, on a barrier that nothing completes.  Every thread's wait must
// give up after about `budget` clock cycles; *out = 2 (the status bit of a
// wait that ran out) if all gave up, 0 if the barrier completed.
__global__ void k_selftest_wait(long long budget, int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(smem_u32(&bar), 0, budget);
  const bool any = __syncthreads_or(ok);
  if (threadIdx.x == 0) *out = any ? 0 : 2;
}

cudaError_t launch_selftest_wait(long long budget, int* out, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(budget, out);
  return cudaGetLastError();
}

template <int L, bool BF, bool FAST>
static cudaError_t launch_tc_t(const ProbDev& P, const StepArgs& a, int grid, cudaStream_t st) {
  constexpr bool SCALED = !BF;  // FP16 operands need the 1/h^2, 1/h column scaling
  const size_t smem = tc_smem_bytes(L);
  cudaError_t e = cudaFuncSetAttribute(k_step_tc<L, BF, FAST, SCALED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_step_tc<L, BF, FAST, SCALED>, dim3(grid), dim3(512), smem, st, P, a);
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
