// nbm_eval.cu -- evaluation of the trained surrogate on a dense grid (the
// use of a trained model in arXiv 2210.14907, Fig. 1: train once, then evaluate):
// u at the (n+1)^3 nodes -1 + i 2/n, each node with the network of its side
// of the interface (phi <= 0: minus).
//
// Tensor-core path: a persistent CTA per SM walks its tiles of 64 nodes once
// per network (the network's hidden weights are staged in shared memory once
// per pass; tiles without a node of that side are skipped), in two
// independent warp groups with three tiles in flight each.  Layer 1 (K = 3)
// and the output layer run in FP32; every hidden layer is one 128x64x128
// tcgen05 MMA per tile with 16-bit operands (FP16 or BF16) and FP32
// accumulation in TMEM.  The FP32 path is a plain SIMT evaluation (reference
// precision).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "nbm_device.cuh"
#include "nbm_f32x2.cuh"
#include "nbm_tc_ptx.cuh"

namespace nbm {
namespace {

using namespace tc;

constexpr int kImgE = 32768;
// 64-point tiles in flight per warp group of the tensor-core evaluation, and the
// TMEM columns they take (2 groups x kEvalTiles x 64, rounded up to a power of 2)
constexpr int kEvalTiles = 3;
constexpr int kEvalTmemCols = 512;  // the tiles' D, then weights (see kWT)

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

// tanh of two values into one packed 16-bit pair.  FP16: the pair is packed
// first and tanh.approx.f16x2 takes both in one SFU operation (the result is
// the GEMM operand, rounded to FP16 either way).  BF16 keeps the FP32 tanh:
// a BF16 argument would lose 3 more bits than the output rounding.
template <bool BF>
__device__ __forceinline__ uint32_t tanh_pack2(float a, float b) {
  if constexpr (BF) {
    return pack2<true>(fast_tanh(a), fast_tanh(b));
  } else {
    uint32_t x = pack2<false>(a, b), y;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
  }
}

// Points: the (n+1)^3 grid nodes, or (pts != nullptr) npts points pts[3i..3i+2].
//
// Two warp groups of 8 warps run independently, each on its own sets of kX
// 64-point tiles (the CTA's tiles alternate between the groups: group g takes
// tiles tb + g, tb + g + 2, ..., kX at a time).  Each tile X (0 .. kX-1) of a group
// has its own activation image (128 units x 64 points, 16 KB), 64 TMEM
// accumulator columns and MMA barrier, so the tensor pipe runs one tile's
// 128 x 64 x 128 GEMM while the CUDA cores run the other tile's epilogue, and
// the two groups (each on its own named barrier) fill each other's waits.  In
// a group, thread (q = warp & 3, cg = (warp >> 2) & 1) owns unit 32 q + lane
// (its TMEM lane) and the tile's points 32 cg .. 32 cg + 31.
//
// Pass 0 (the minus network) decides every point's side and keeps it in
// `side` (per 128 points, bit c: point c is in Omega-; each 64-point tile owns
// two of the four words); pass 1 reads it back instead of evaluating the
// level set again.  A tile without a point of the pass's side is skipped.
template <int L, bool BF>
__global__ void __launch_bounds__(512, 1) k_eval_tc(ProbDev P, const float* __restrict__ params,
                                                    const unsigned char* __restrict__ wimg, int n,
                                                    const float* __restrict__ pts, int64_t npts,
                                                    float* __restrict__ u_out, uint4* side,
                                                    int* status) {
  constexpr int H = 128, NG = L - 1, kTP = 64, kImgG = 16384, kX = kEvalTiles;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int grp = tid >> 8, gtid = tid & 255, gw = gtid >> 5;
  const int q = w & 3, cg = (w >> 2) & 1, u = 32 * q + lane, col0 = 32 * cg;
  const uint32_t gbar = 1u + (uint32_t)grp;
  unsigned char* Wimg = sm;                                    // [NG] 32 KB
  unsigned char* Aimg = sm + NG * kImgE + grp * kX * kImgG;    // this group's [kX] images
  unsigned char* misc = sm + NG * kImgE + 2 * kX * kImgG;
  uint64_t* bar_w = (uint64_t*)misc;
  uint64_t* bar_mma = (uint64_t*)(misc + 8) + kX * grp;        // this group's [kX]
  uint32_t* tslot = (uint32_t*)(misc + 8 + 16 * kX);
  volatile int* abort_f = (volatile int*)(misc + 12 + 16 * kX);
  int* actw = (int*)(misc + 128) + grp * 4 * kX;               // [2 set parities][2 kX warps]
  constexpr int kRed = 256, kXs = kRed + 2 * kX * 4 * kTP * 4, kFlag = kXs + 2 * kX * 3 * kTP * 4;
  float* red = (float*)(misc + kRed) + grp * kX * 4 * kTP;     // [kX][4][64] output partials
  float* xs = (float*)(misc + kXs) + grp * kX * 3 * kTP;       // [kX][3][64] coordinates
  int* flag = (int*)(misc + kFlag) + grp * kX * kTP;           // [kX][64]

  const uint32_t idf = idesc_f16_n(BF, false, true, kTP);
  if (tid == 0) {
    mbar_init(smem_u32(bar_w), 1);
    for (int b = 0; b < 2 * kX; ++b) mbar_init(smem_u32((uint64_t*)(misc + 8) + b), 1);
    *abort_f = 0;
    fence_mbar_init();
  }
  if (w == 0) tmem_alloc(smem_u32(tslot), kEvalTmemCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t d_tm = tmem + (uint32_t)(kX * kTP * grp);  // tile X: d_tm + 64 X
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  // per-tile state as bit X: MMA barrier phase, and a commit not yet waited for
  uint32_t ph_w = 0, ph_bits = 0, pending_bits = 0;
  const int64_t N1 = n + 1, total = pts ? npts : N1 * N1 * N1;
  const int64_t T = (total + kTP - 1) / kTP;
  const int64_t tb = (int64_t)blockIdx.x * T / gridDim.x, te = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  const float hg = 2.0f / (float)n;
  bool aborted = false;

  // The weights of the first kWT hidden layers sit in the TMEM columns past
  // the tiles' D (64 columns per layer; the GEMMs' A operand), which spares
  // those GEMMs the 32 KB weight read from shared memory.
  constexpr uint32_t kWCol = 2 * kX * kTP;  // first column past the tiles' D
  constexpr int kFreeLayers = (kEvalTmemCols - (int)kWCol) / 64;
  constexpr int kWT = NG < kFreeLayers ? NG : kFreeLayers;
  // the layer-g GEMM of tile X: weights g (K-major; TMEM for g < kWT) x image X
  // (MN-major)
  auto issue = [&](int X, int g) {
    if (gtid == 0) {
      fence_after_sync();
      const uint32_t ab = smem_u32(Aimg + X * kImgG);
      if (g < kWT) {
        const uint32_t wt = tmem + kWCol + 64u * (uint32_t)g;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          mma_f16_ta(d_tm + kTP * X, wt + 8u * (uint32_t)k, desc_mnmajor(ab, k), idf, k > 0);
      } else {
        const uint32_t wa = smem_u32(Wimg + g * kImgE);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          mma_f16(d_tm + kTP * X, desc_kmajor(wa, k), desc_mnmajor(ab, k), idf, k > 0);
      }
      mma_commit(smem_u32(bar_mma + X));
    }
    pending_bits |= 1u << X;
  };
  // bounded wait for tile X's GEMM; false if it gave up
  auto wait_mma = [&](int X) -> bool {
    const bool ok = mbar_wait_bounded(smem_u32(bar_mma + X), (ph_bits >> X) & 1u);
    if (ok) {  // a wait that gave up leaves the GEMM pending for the exit path
      ph_bits ^= 1u << X;
      pending_bits &= ~(1u << X);
    }
    fence_after_sync();
    return ok;
  };
  // the group barrier that ends a phase; it agrees on an abort.  False: abort.
  auto end_phase = [&](bool ok) -> bool {
    fence_before_sync();
    fence_proxy_async();
    const bool bad = named_sync_or(gbar, 256, !ok || *abort_f != 0);
    if (bad && gtid == 0) {
      if (!ok) atomicOr(status, 2);
      *abort_f = 1;
    }
    return !bad;
  };

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
      if (ok) ph_w ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(status, 2);
        aborted = true;
        break;
      }
    }
    // this network's first kWT weight layers into TMEM (the previous pass's
    // GEMMs have all completed)
    if (w < 4) stage_weights_tmem(Wimg, kImgE, tmem + ((uint32_t)(32 * w) << 16) + kWCol, u, kWT);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    int set = 0;
#pragma unroll 1
    for (int64_t t = tb + grp; t < te; t += 2 * kX, ++set) {
      // tile X of this set is t + 2 X; actw alternates between two halves: a
      // set without active tiles has no barrier after its reads
      int* aw = actw + 2 * kX * (set & 1);
      // coordinates and side flags of the tiles' 64 points (threads 0 .. 64 kX - 1)
      if (gtid < kX * kTP) {
        const int X = gtid >> 6, c = gtid & 63;
        const int64_t tx = t + 2 * X;
        const int64_t id = tx * kTP + c;
        const bool valid = tx < te && id < total;
        int f = 0, minus = 0;
        uint32_t* sw = valid ? reinterpret_cast<uint32_t*>(&side[tx >> 1]) + 2 * (tx & 1) + (c >> 5)
                             : nullptr;
        if (s == 1 && valid) {  // the side decided in pass 0
          minus = (*sw >> (c & 31)) & 1u;
          f = !minus;
        }
        float x = 0.f, y = 0.f, z = 0.f;
        if (valid && (s == 0 || f)) {
          if (pts) {
            x = pts[3 * id];
            y = pts[3 * id + 1];
            z = pts[3 * id + 2];
          } else if (total <= 0xffffffffll) {  // 32-bit index arithmetic
            const uint32_t id32 = (uint32_t)id, n1 = (uint32_t)N1, r = id32 / n1;
            x = -1.f + hg * (float)(id32 - r * n1);
            y = -1.f + hg * (float)(r % n1);
            z = -1.f + hg * (float)(r / n1);
          } else {
            const int i = (int)(id % N1), j = (int)((id / N1) % N1), k = (int)(id / (N1 * N1));
            x = -1.f + hg * (float)i;
            y = -1.f + hg * (float)j;
            z = -1.f + hg * (float)k;
          }
        }
        if (s == 0) {
          minus = valid && node_phase(P, x, y, z) == 0;
          f = minus;
          const uint32_t bits = __ballot_sync(0xffffffffu, minus);
          if (lane == 0 && valid) *sw = bits;
        }
        float* xx = xs + X * 3 * kTP;
        xx[c] = x;
        xx[kTP + c] = y;
        xx[2 * kTP + c] = z;
        flag[X * kTP + c] = f;
        const uint32_t any = __ballot_sync(0xffffffffu, f);
        if (lane == 0) aw[gw] = any != 0u;
      }
      named_sync(gbar, 256);
      uint32_t act = 0;
#pragma unroll
      for (int X = 0; X < kX; ++X) act |= ((aw[2 * X] | aw[2 * X + 1]) ? 1u : 0u) << X;
      if (!act) continue;
      // layer 1 (FP32, K = 3) of each active tile -> its image; then its GEMM
#pragma unroll
      for (int X = 0; X < kX; ++X) {
        if (!((act >> X) & 1u)) continue;
        const float* xx = xs + X * 3 * kTP;
        unsigned char* dst = Aimg + X * kImgG;
#pragma unroll
        for (int c8 = 0; c8 < 4; ++c8) {
          float z[8];
#pragma unroll
          for (int h4 = 0; h4 < 2; ++h4) {  // four points per 16-byte shared load
            const int c = col0 + 8 * c8 + 4 * h4;
            const float4 px = *reinterpret_cast<const float4*>(xx + c);
            const float4 py = *reinterpret_cast<const float4*>(xx + kTP + c);
            const float4 pz = *reinterpret_cast<const float4*>(xx + 2 * kTP + c);
            z[4 * h4 + 0] = fmaf(w10, px.x, fmaf(w11, py.x, fmaf(w12, pz.x, b1)));
            z[4 * h4 + 1] = fmaf(w10, px.y, fmaf(w11, py.y, fmaf(w12, pz.y, b1)));
            z[4 * h4 + 2] = fmaf(w10, px.z, fmaf(w11, py.z, fmaf(w12, pz.z, b1)));
            z[4 * h4 + 3] = fmaf(w10, px.w, fmaf(w11, py.w, fmaf(w12, pz.w, b1)));
          }
          *reinterpret_cast<uint4*>(dst + img_off(u, col0 + 8 * c8)) =
              make_uint4(tanh_pack2<BF>(z[0], z[1]), tanh_pack2<BF>(z[2], z[3]),
                         tanh_pack2<BF>(z[4], z[5]), tanh_pack2<BF>(z[6], z[7]));
        }
      }
      if (!end_phase(true)) {
        aborted = true;
        break;
      }
      for (int X = 0; X < kX; ++X)
        if ((act >> X) & 1u) issue(X, 0);
      // hidden layers: while one tile's epilogue runs, the other tile's GEMM does
      bool ok_all = true;  // this thread's MMA waits of the pair
#pragma unroll 1
      for (int g = 1; g <= NG && !aborted; ++g) {
        float bb = bh[0];
#pragma unroll
        for (int i = 1; i < NG; ++i) bb = (g - 1 == i) ? bh[i] : bb;
#pragma unroll 1
        for (int X = 0; X < kX; ++X) {
          if (!((act >> X) & 1u)) continue;
          ok_all = wait_mma(X) && ok_all;
          float acc[32];
          tmem_ld32(d_tm + kTP * X + lane_base + col0, acc);
          const F2 BB = f2s(bb);
          if (g < NG) {
            unsigned char* dst = Aimg + X * kImgG;
#pragma unroll
            for (int c8 = 0; c8 < 4; ++c8) {
              // the bias on packed FP32 pairs, then tanh and the 16-bit operand
              float z[8];
#pragma unroll
              for (int i = 0; i < 8; i += 2)
                f2get(add2(f2(acc[8 * c8 + i], acc[8 * c8 + i + 1]), BB), z[i], z[i + 1]);
              *reinterpret_cast<uint4*>(dst + img_off(u, col0 + 8 * c8)) =
                  make_uint4(tanh_pack2<BF>(z[0], z[1]), tanh_pack2<BF>(z[2], z[3]),
                             tanh_pack2<BF>(z[4], z[5]), tanh_pack2<BF>(z[6], z[7]));
            }
            if (!end_phase(ok_all)) {
              aborted = true;
              break;
            }
            issue(X, g);
          } else {
            // output layer (FP32): the sum over units of wo * tanh
            float v[32], sres;
            const F2 WO = f2s(wo);
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
              float za, zb;
              f2get(add2(f2(acc[i], acc[i + 1]), BB), za, zb);
              f2get(mul2(WO, f2(fast_tanh(za), fast_tanh(zb))), v[i], v[i + 1]);
            }
            reduce32(v, lane, sres);
            red[(X * 4 + q) * kTP + col0 + lane] = sres;
          }
        }
      }
      if (aborted) break;
      if (!end_phase(ok_all)) {
        aborted = true;
        break;
      }
      if (gtid < kX * kTP) {
        const int X = gtid >> 6, c = gtid & 63;
        if (((act >> X) & 1u) && flag[X * kTP + c]) {
          const float* r = red + X * 4 * kTP;
          u_out[(t + 2 * X) * kTP + c] = r[c] + r[kTP + c] + r[2 * kTP + c] + r[3 * kTP + c] + bo;
        }
      }
      // no barrier here: each thread rewrites only its own coordinate and flag
      // slots in the next staging, and red, the images and TMEM are next
      // written after the next pair's barriers
    }
    // both groups are done with this network before its weights are replaced
    if (__syncthreads_or(aborted)) aborted = true;
  }
  if (aborted) {
    if (tid == 0) atomicOr(status, 2);
    // let any GEMM still committed, and a weight copy that a wait gave up on,
    // finish (bounded) before TMEM and shared memory are released
    for (int X = 0; X < kX; ++X)
      if ((pending_bits >> X) & 1u)
        (void)mbar_wait_bounded(smem_u32(bar_mma + X), (ph_bits >> X) & 1u, 2000000LL);
    (void)mbar_wait_bounded(smem_u32(bar_w), ph_w, 2000000LL);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, kEvalTmemCols);
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
                             int n, const float* pts, int64_t npts, float* u, uint4* side,
                             int grid, int* status, cudaStream_t st) {
  // weights (L-1) x 32 KB, 2 kEvalTiles 16 KB tile images, barriers, partials,
  // coordinates and flags (256 + 4608 kEvalTiles bytes), 1 KB of alignment slack
  const size_t smem = (size_t)(L - 1) * kImgE + 2 * kEvalTiles * 16384 + 256 +
                      4608 * kEvalTiles + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_eval_tc<L, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_eval_tc<L, BF><<<grid, 512, smem, st>>>(P, params, wimg, n, pts, npts, u, side, status);
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
    uint4* side = nullptr;  // per 128-point tile: bit c set if point c is in Omega-
    const int64_t total = pts ? npts : (int64_t)(n + 1) * (n + 1) * (n + 1);
    e = cudaMalloc((void**)&wimg, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&side, sizeof(uint4) * (size_t)((total + 127) / 128));
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    Workspace tmp;
    tmp.wtc = wimg;
    if (e == cudaSuccess) e = launch_prep_weights(P, params, precision, tmp, st);
    const int grid = problem_num_sms(p);
    const bool bf = precision == NBM_PREC_BF16;
    if (e == cudaSuccess) {
      if (d.n_hidden == 2) e = bf ? launch_eval_tc_t<2, true>(P, params, wimg, n, pts, npts, u_out, side, grid, status, st)
                                  : launch_eval_tc_t<2, false>(P, params, wimg, n, pts, npts, u_out, side, grid, status, st);
      else if (d.n_hidden == 3) e = bf ? launch_eval_tc_t<3, true>(P, params, wimg, n, pts, npts, u_out, side, grid, status, st)
                                       : launch_eval_tc_t<3, false>(P, params, wimg, n, pts, npts, u_out, side, grid, status, st);
      else e = bf ? launch_eval_tc_t<4, true>(P, params, wimg, n, pts, npts, u_out, side, grid, status, st)
                  : launch_eval_tc_t<4, false>(P, params, wimg, n, pts, npts, u_out, side, grid, status, st);
    }
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (wimg) cudaFree(wimg);
    if (status) cudaFree(status);
    if (side) cudaFree(side);
    if (e == cudaSuccess && (hs & 2)) {
      set_error_message("grid evaluation: a bounded device wait gave up");
      return NBM_ERR_DEVICE_TIMEOUT;
    }
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "grid evaluation: %s", cudaGetErrorString(e));
    set_error_message(msg);
    return e == cudaErrorMemoryAllocation ? NBM_ERR_OOM : NBM_ERR_CUDA;
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
