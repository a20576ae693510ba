// nbm_eval.cu -- evaluation of the trained surrogate on a dense grid (the
// use of a trained model in arXiv 2210.14907, Fig. 1: train once, then evaluate):
// u at the (n+1)^3 nodes -1 + i 2/n, each node with the network of its side
// of the interface (phi <= 0: minus).
//
// Tensor-core path: a persistent CTA per SM walks its tiles of 128 nodes, two
// at a time, once per network (the network's hidden weights are staged in
// shared memory once per pass; tiles without a node of that side are
// skipped).  Layer 1 (K = 3) and the output layer run in FP32; every hidden
// layer is one 128x128x128 tcgen05 MMA with 16-bit operands (FP16 or BF16)
// and FP32 accumulation in TMEM.  The FP32 path is a plain SIMT evaluation
// (reference precision).
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
// Two tiles of 128 points are in flight per CTA.  Tile X (0, 1) has its own
// TMEM accumulator (columns 128 X .. 128 X + 127), activation image,
// coordinates, flags, output partials and MMA barrier, so the tensor core
// runs one tile's layer-g GEMM while the CUDA cores run the other tile's
// epilogue.  Thread (q = warp & 3, cg = warp >> 2) owns unit 32 q + lane
// (its TMEM lane) and the tile's columns 32 cg .. 32 cg + 31.
//
// Pass 0 (the minus network) decides every point's side and keeps it as a
// 128-bit mask per tile in `side` (bit c: point c is in Omega-); pass 1 reads
// the mask back instead of evaluating the level set again.
template <int L, bool BF>
__global__ void __launch_bounds__(512, 1) k_eval_tc(ProbDev P, const float* __restrict__ params,
                                                    const unsigned char* __restrict__ wimg, int n,
                                                    const float* __restrict__ pts, int64_t npts,
                                                    float* __restrict__ u_out, uint4* side,
                                                    int* status) {
  constexpr int H = 128, NG = L - 1;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Wimg = sm;                       // [NG]
  unsigned char* Aimg = sm + NG * kImgE;          // [2] one activation image per tile
  unsigned char* misc = sm + (NG + 2) * kImgE;
  uint64_t* bar_w = (uint64_t*)misc;
  uint64_t* bar_mma = (uint64_t*)(misc + 8);      // [2]
  uint32_t* tslot = (uint32_t*)(misc + 24);
  float* red = (float*)(misc + 64);               // [2][4][128] output partials
  float* xs = red + 1024;                         // [2][3][128] coordinates
  int* flag = (int*)(xs + 768);                   // [2][128]
  int* actw = flag + 256;  // [2][8] staging warps with a point of the side, by pair parity

  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int q = w & 3, cg = w >> 2, u = 32 * q + lane, col0 = 32 * cg;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  const uint32_t idf = idesc_f16(BF, false, true);
  if (tid == 0) {
    mbar_init(smem_u32(bar_w), 1);
    mbar_init(smem_u32(bar_mma), 1);
    mbar_init(smem_u32(bar_mma + 1), 1);
    fence_mbar_init();
  }
  if (w == 0) tmem_alloc(smem_u32(tslot), 256);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  // per-tile state as bit X of a register: MMA barrier phase, and a commit on
  // bar_mma[X] not yet waited for
  uint32_t ph_w = 0, ph_bits = 0, pending_bits = 0;
  const int64_t N1 = n + 1, total = pts ? npts : N1 * N1 * N1;
  const int64_t T = (total + 127) / 128;
  const int64_t tb = (int64_t)blockIdx.x * T / gridDim.x, te = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  const float hg = 2.0f / (float)n;
  bool aborted = false;

  // the layer-g GEMM of tile X: weights g (K-major) x image X (MN-major)
  auto issue = [&](int X, int g) {
    if (tid == 0) {
      fence_after_sync();
      const uint32_t wa = smem_u32(Wimg + g * kImgE);
      const uint32_t ab = smem_u32(Aimg + X * kImgE);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        mma_f16(tmem + 128 * X, desc_kmajor(wa, k), desc_mnmajor(ab, k), idf, k > 0);
      mma_commit(smem_u32(bar_mma + X));
    }
    pending_bits |= 1u << X;
  };
  // bounded wait for tile X's GEMM (this thread's result; the CTA agrees on an
  // abort at the barrier that ends the epilogue)
  auto wait_mma = [&](int X) {
    const bool ok = mbar_wait_bounded(smem_u32(bar_mma + X), (ph_bits >> X) & 1u);
    if (ok) {  // a wait that gave up leaves the GEMM pending for the exit path
      ph_bits ^= 1u << X;
      pending_bits &= ~(1u << X);
    }
    fence_after_sync();
    return ok;
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
    for (int64_t t = tb, pair = 0; t < te && !aborted; t += 2, ++pair) {
      // actw alternates between two halves: a pair without active tiles has no
      // barrier after its reads, so the next pair must not overwrite them
      int* aw = actw + 8 * (int)(pair & 1);
      // coordinates and side flags of both tiles (threads 0..255)
      int f = 0;
      if (tid < 256) {
        const int X = tid >> 7, c = tid & 127;
        const int64_t id = (t + X) * 128 + c;
        const bool valid = t + X < te && id < total;
        int minus = 0;
        if (s == 1 && valid) {  // the side decided in pass 0
          const uint4 m = side[t + X];
          const uint32_t word = (c >> 5) == 0 ? m.x : (c >> 5) == 1 ? m.y : (c >> 5) == 2 ? m.z : m.w;
          minus = (word >> (c & 31)) & 1u;
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
          if (lane == 0 && t + X < te) ((uint32_t*)&side[t + X])[c >> 5] = bits;  // own tiles only
        }
        xs[X * 384 + c] = x;
        xs[X * 384 + 128 + c] = y;
        xs[X * 384 + 256 + c] = z;
        flag[X * 128 + c] = f;
        const uint32_t any = __ballot_sync(0xffffffffu, f);
        if (lane == 0) aw[w] = any != 0u;
      }
      __syncthreads();
      const uint32_t act = ((aw[0] | aw[1] | aw[2] | aw[3]) ? 1u : 0u) |
                           ((aw[4] | aw[5] | aw[6] | aw[7]) ? 2u : 0u);
      if (!act) continue;
      // layer 1 (FP32 K = 3) of each active tile -> its image; then its GEMM
#pragma unroll
      for (int X = 0; X < 2; ++X) {
        if (!((act >> X) & 1u)) continue;
        const float* xx = xs + X * 384;
        unsigned char* dst = Aimg + X * kImgE;
#pragma unroll
        for (int c8 = 0; c8 < 4; ++c8) {
          float z[8];
#pragma unroll
          for (int h4 = 0; h4 < 2; ++h4) {  // four columns per 16-byte shared load
            const int c = col0 + 8 * c8 + 4 * h4;
            const float4 px = *reinterpret_cast<const float4*>(xx + c);
            const float4 py = *reinterpret_cast<const float4*>(xx + 128 + c);
            const float4 pz = *reinterpret_cast<const float4*>(xx + 256 + c);
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
      fence_proxy_async();
      __syncthreads();
      for (int X = 0; X < 2; ++X)
        if ((act >> X) & 1u) issue(X, 0);
      // hidden layers: while one tile's epilogue runs, the other tile's GEMM does
      bool ok_all = true;  // this thread's MMA waits of the pair
#pragma unroll 1
      for (int g = 1; g <= NG && !aborted; ++g) {
        float bb = bh[0];
#pragma unroll
        for (int i = 1; i < NG; ++i) bb = (g - 1 == i) ? bh[i] : bb;
#pragma unroll 1
        for (int X = 0; X < 2; ++X) {
          if (!((act >> X) & 1u)) continue;
          ok_all = wait_mma(X) && ok_all;
          float acc[32];
          tmem_ld32(tmem + lane_base + 128 * X + col0, acc);
          if (g < NG) {
            unsigned char* dst = Aimg + X * kImgE;
#pragma unroll
            for (int c8 = 0; c8 < 4; ++c8) {
              const float* a8 = acc + 8 * c8;
              *reinterpret_cast<uint4*>(dst + img_off(u, col0 + 8 * c8)) =
                  make_uint4(tanh_pack2<BF>(a8[0] + bb, a8[1] + bb), tanh_pack2<BF>(a8[2] + bb, a8[3] + bb),
                             tanh_pack2<BF>(a8[4] + bb, a8[5] + bb), tanh_pack2<BF>(a8[6] + bb, a8[7] + bb));
            }
            fence_before_sync();
            fence_proxy_async();
            if (__syncthreads_or(!ok_all)) {
              aborted = true;
              break;
            }
            issue(X, g);
          } else {
            // output layer (FP32): the sum over units of wo * tanh
            float v[32], sres;
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = wo * fast_tanh(acc[i] + bb);
            reduce32(v, lane, sres);
            red[X * 512 + q * 128 + col0 + lane] = sres;
          }
        }
      }
      if (aborted) break;
      fence_before_sync();
      if (__syncthreads_or(!ok_all)) {
        aborted = true;
        break;
      }
      if (tid < 256) {
        const int X = tid >> 7, c = tid & 127;
        if (((act >> X) & 1u) && flag[X * 128 + c]) {
          const float* r = red + X * 512;
          u_out[(t + X) * 128 + c] = r[c] + r[128 + c] + r[256 + c] + r[384 + c] + bo;
        }
      }
      // no barrier here: each thread rewrites only its own flag slot in the
      // next staging, and xs, red, the images and TMEM are next written after
      // the next pair's barriers
    }
  }
  if (aborted) {
    if (tid == 0) atomicOr(status, 2);
    // let any GEMM still committed, and a weight copy that a wait gave up on,
    // finish (bounded) before TMEM and shared memory are released
    for (int X = 0; X < 2; ++X)
      if ((pending_bits >> X) & 1u) (void)mbar_wait_bounded(smem_u32(bar_mma + X), (ph_bits >> X) & 1u);
    (void)mbar_wait_bounded(smem_u32(bar_w), ph_w, 2000000LL);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, 256);
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
  const size_t smem = (size_t)(L + 1) * kImgE + 1024 + 12288;
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
