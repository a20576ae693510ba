// nbm_prep.cu -- the light stages of the NBM step (arXiv 2210.14907, Sec. 3):
//   sample + classify  : Philox collocation points, cut/uncut decision of the
//                        implicit cell from the level set at its 8 corners
//   scan + scatter     : stable phase partition (two networks -> two lists;
//                        cut cells go into both and into the cut list) and
//                        the tensor-core tile records of the uncut points
//   cut geometry       : Kuhn-split volume / face / interface fractions and
//                        the interface point of every cut cell (FP32 on
//                        cell-local coordinates, FP64 in the FP64-row mode),
//                        and the cut cells' tile records
//   gather             : the tile records in list order (large batches)
//   cut residual       : balance + jump rows of cut cells (both networks)
//   weight staging     : FP32 transposed and 16-bit tensor-core copies
//   finish             : deterministic loss / gradient reduction (8 slice
//                        groups per 32 parameters, fixed order) and Adam,
//                        one launch
#include <cmath>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nbm_device.cuh"
#include "nbm_geom.cuh"
#include "nbm_tc_ptx.cuh"

namespace nbm {

constexpr int kBlk = 256;
// Batches of up to this many point blocks: the scatter sums the block counts
// itself and writes the tile records (else k_scan_counts and k_gather_tiles).
constexpr int kScatterPrefixBlocks = 2048;

// ------------------------------------------------------------------------
// Collocation points.  Uniform: lattice -1 + k 2^-22, k = 1 + floor(r (2^23-1)
// / 2^32) per axis (integer arithmetic, identical everywhere).  Band: a ray
// direction uniform on the sphere and an offset t in (-4h, 4h) from the
// interface radius along it, in FP64, quantised to the same lattice.
// ------------------------------------------------------------------------
__device__ inline double quantize_coord(double v) {
  double k = floor((v + 1.0) * 4194304.0 + 0.5);
  k = fmin(fmax(k, 1.0), 8388607.0);
  return -1.0 + k / 4194304.0;
}

__device__ inline void draw_point(const ProbDev& P, uint64_t seed, int64_t step, int64_t i,
                                  bool band, float p[3]) {
  uint32_t r[4];
  philox4x32_10((uint32_t)i, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), kPointStream,
                (uint32_t)seed, (uint32_t)(seed >> 32), r);
  if (!band) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      uint32_t k = 1u + (uint32_t)(((uint64_t)r[j] * 8388607ull) >> 32);
      p[j] = -1.0f + (float)k * (1.0f / 4194304.0f);
    }
    return;
  }
  double u0 = ((double)(r[0] >> 8) + 0.5) / 16777216.0;
  double u1 = ((double)(r[1] >> 8) + 0.5) / 16777216.0;
  double u2 = ((double)(r[2] >> 8) + 0.5) / 16777216.0;
  double cth = 1.0 - 2.0 * u0;
  double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
  // azimuth psi = 2 pi u1: its cosine and sine by sincospi (no argument
  // reduction of 2 pi u1)
  double sps, cps;
  sincospi(2.0 * u1, &sps, &cps);
  double t = (2.0 * u2 - 1.0) * 4.0 * P.h_band;
  double R = P.r0;
  if (P.geometry == NBM_GEOM_FLOWER) {
    // theta = acos(cth), sin(theta) = sth >= 0
    double st, ct, cp, sp;
    flower_factors<double>(P, cth, sth, cps, sps, st, ct, cp, sp);
    // a lobe count that is not an integer: the factor of the draw's own
    // azimuth 2 pi u1 in (0, 2 pi) (not periodic in 2 pi)
    if (P.lp_i < 0) cp = cos(P.lp * (2.0 * 3.14159265358979323846 * u1));
    R += P.amp * st * cp;
  }
  p[0] = (float)quantize_coord((R + t) * sth * cps);
  p[1] = (float)quantize_coord((R + t) * sth * sps);
  p[2] = (float)quantize_coord((R + t) * cth);
}

// Number of corners of the cell p + [-h/2, h/2]^3 with phi <= 0.  FP32 first;
// a corner whose FP32 value is within the FP32 error band of 0 is redone in
// FP64, so that every decision is the FP64 one.
__device__ inline int count_neg_corners(const ProbDev& P, const float p[3]) {
  const float hh = 0.5f * P.hf;
  int nneg = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float cx = p[0] + ((c & 1) ? hh : -hh), cy = p[1] + ((c & 2) ? hh : -hh),
                cz = p[2] + ((c & 4) ? hh : -hh);
    const float f = phi_f(P, cx, cy, cz);
    bool neg = f <= 0.f;
    if (fabsf(f) < 2e-5f) {
      // within the FP32 error band of 0: the FP64 sign (a corner outside the
      // band has the same sign in both precisions)
      const double hd = 0.5 * P.h;
      neg = phi_d(P, (double)p[0] + ((c & 1) ? hd : -hd), (double)p[1] + ((c & 2) ? hd : -hd),
                  (double)p[2] + ((c & 4) ? hd : -hd)) <= 0.0;
    }
    nneg += neg;
  }
  return nneg;
}

// ------------------------------------------------------------------------
// Weight staging.  Hidden layer l of net s (W[u][k], u = output unit):
//   wt  : FP32 transpose, wt[((s*(L-1) + l-1)*H + k)*H + u] = W[u][k]
//   wtc : 16-bit copy in the tensor-core shared-memory image (H = 128):
//         8-row x 128-byte atoms with the 128-byte XOR swizzle,
//         atom (cb, ug) at (cb*16 + ug)*1024 for column block cb = k/64 and
//         row group ug = u/8.
// ------------------------------------------------------------------------
__host__ __device__ inline uint32_t tc_tile_offset(int u, int c) { return tc::img_off(u, c); }

// Hidden weights of both networks restaged from the parameter vector: the
// FP32 transposed copy wt [net][layer][k][u] and, for the tensor-core path,
// the 16-bit image in the tcgen05 tile layout.  Element e of block (net,
// layer) in (u, k) order; blocks b of nblk share the elements.
__device__ inline void prep_weights_blocks(const ProbDev& P, const float* params, float* wt,
                                           void* wtc, int prec, int b, int nblk) {
  const int H = P.H, L = P.L, per = H * H;
  const int total = 2 * (L - 1) * per;
  for (int e = b * blockDim.x + threadIdx.x; e < total; e += nblk * blockDim.x) {
    const int blk = e / per, s = blk / (L - 1), l = blk - s * (L - 1) + 1;
    const int rem = e - blk * per, u = rem / H, k = rem - u * H;
    const float w = params[(int64_t)s * P.p_net + 4 * H + (int64_t)(l - 1) * (per + H) + rem];
    if (wt) wt[(int64_t)blk * per + (int64_t)k * H + u] = w;
    if (wtc && H == 128) {
      char* base = (char*)wtc + (int64_t)blk * per * 2;
      if (prec == NBM_PREC_FP16)
        *(__half*)(base + tc_tile_offset(u, k)) = __float2half_rn(w);
      else
        *(__nv_bfloat16*)(base + tc_tile_offset(u, k)) = __float2bfloat16_rn(w);
    }
  }
}

// blocks of a weight restage
static int prep_weight_blocks(const ProbDev& P) { return 2 * (P.L - 1) * 16; }

__global__ void __launch_bounds__(kBlk) k_sample_classify(ProbDev P, const float* pts_in,
                                                          uint64_t seed, const int64_t* step_dev,
                                                          int64_t step_host, int64_t n,
                                                          int64_t n_band, float* X, float* Y,
                                                          float* Z, uint8_t* cls, int* blockcnt,
                                                          int nb, int64_t first, int64_t n_total,
                                                          const float* prep_params, float* wt,
                                                          void* wtc, int prec) {
  pdl_enter();
  if ((int)blockIdx.x >= nb) {
    // the blocks past the points restage the hidden weights (first step of a call)
    prep_weights_blocks(P, prep_params, wt, wtc, prec, blockIdx.x - nb, gridDim.x - nb);
    return;
  }
  int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x;
  int c = -1;
  if (i < n) {
    float p[3];
    if (pts_in) {
      p[0] = pts_in[3 * i];
      p[1] = pts_in[3 * i + 1];
      p[2] = pts_in[3 * i + 2];
    } else {
      // point first + i of the step's n_total-point batch (band points last)
      int64_t step = step_dev ? (*step_dev + 1) : step_host;
      bool iface = P.geometry == NBM_GEOM_SPHERE || P.geometry == NBM_GEOM_FLOWER;
      const int64_t ig = first + i;
      draw_point(P, seed, step, ig, iface && ig >= n_total - n_band, p);
    }
    X[i] = p[0];
    Y[i] = p[1];
    Z[i] = p[2];
    int nneg = count_neg_corners(P, p);
    c = nneg == 8 ? 0 : (nneg == 0 ? 1 : 2);
    cls[i] = (uint8_t)c;
  }
  int cm = __syncthreads_count(c == 0 || c == 2);
  int cp = __syncthreads_count(c == 1 || c == 2);
  int cc = __syncthreads_count(c == 2);
  if (threadIdx.x == 0) {
    blockcnt[blockIdx.x] = cm;
    blockcnt[nb + blockIdx.x] = cp;
    blockcnt[2 * nb + blockIdx.x] = cc;
  }
}

// Exclusive scan of the three per-block count arrays (one CTA).  counters[0..2]
// receive the totals (n-, n+, n_cut).
__global__ void __launch_bounds__(1024) k_scan_counts(int* blockcnt, int nb, int* counters) {
  pdl_enter();
  __shared__ int warp_tot[32];
  for (int m = 0; m < 3; ++m) {
    int* a = blockcnt + (int64_t)m * nb;
    int per = (nb + 1023) / 1024;
    int lo = threadIdx.x * per, hi = min(lo + per, nb);
    int s = 0;
    for (int j = lo; j < hi; ++j) s += a[j];
    // block exclusive scan of s
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      int v = warp_tot[lane], iv = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, iv, o);
        if (lane >= o) iv += t;
      }
      warp_tot[lane] = iv - v;
      if (lane == 31) counters[m] = iv;
    }
    __syncthreads();
    int run = warp_tot[w] + incl - s;
    for (int j = lo; j < hi; ++j) {
      int v = a[j];
      a[j] = run;
      run += v;
    }
    __syncthreads();
  }
}

// Record of an uncut point of phase s (tile layout of the tensor-core kernel):
// the point and the source term f^s(p) of its balance row (Sec. 3), so that
// the fused kernel's residual stage does no transcendental arithmetic.
__device__ inline PRec uncut_record(const ProbDev& P, int s, int pt, float x, float y, float z) {
  PRec o;
  o.x = x;
  o.y = y;
  o.z = z;
  o.pt = pt;
  o.cutj = -1;
  o.gz = 0.f;
  if (P.fp64) {  // FP64 rows: f^s(p) as a two-float sum gx + gy
    const double f = rhs_f<double>(P, s, (double)x, (double)y, (double)z);
    o.gx = (float)f;
    o.gy = (float)(f - (double)o.gx);
  } else {
    o.gx = rhs_f<float>(P, s, x, y, z);
    o.gy = 0.f;
  }
  return o;
}

// A record is 32 bytes at a 32-byte aligned address: two 16-byte stores.
__device__ inline void store_record(PRec* dst, const PRec& o) {
  float4* d = reinterpret_cast<float4*>(dst);
  d[0] = make_float4(o.x, o.y, o.z, o.gx);
  d[1] = make_float4(o.gy, o.gz, __int_as_float(o.pt), __int_as_float(o.cutj));
}

__device__ inline PRec pad_record() {
  PRec o;
  o.x = o.y = o.z = o.gx = o.gy = o.gz = 0.f;
  o.pt = -1;
  o.cutj = -1;
  return o;
}

// Stable scatter: list order = point order.  Entry >= 0: uncut point index;
// entry < 0: cut cell -(cut_id + 1).  scanned: blockcnt holds the exclusive
// offsets (k_scan_counts ran).  Otherwise (few blocks: the scan's launch
// costs more than the sums) each block adds up the per-block counts of the
// blocks before it (integer sums: exact in any order) for its offsets in the
// three lists, and the last block writes the totals counters[0..2].
// rec != nullptr (tensor-core paths): the tile records too.  rec holds the
// minus list, then the plus list, each padded to a multiple of 16 records
// (the plus list starts at 16 ceil(n-/16)); rec_cut the cut list, padded the
// same way.  An uncut point writes its own record; a cut point writes its two
// record slots to cut_rpos, and k_cut_geometry writes the cut cell's three
// records once its interface point is known; the last block writes the
// padding.  Every slot up to the padded ends is written each step.
__global__ void __launch_bounds__(kBlk) k_scatter(const ProbDev P, const uint8_t* cls, int64_t n,
                                                  const int* blockcnt, int nb, int scanned,
                                                  int* list_m, int* list_p, int* cut_pt,
                                                  int* counters, const float* X, const float* Y,
                                                  const float* Z, PRec* rec, PRec* rec_cut,
                                                  int2* cut_rpos) {
  pdl_enter();
  __shared__ int boff[4][kBlk / 32];
  __shared__ int wsum[3][kBlk / 32];
  if (!scanned) {
    // s*: counts of the blocks before this one; t0: all blocks' minus count
    int s0 = 0, s1 = 0, s2 = 0, t0 = 0;
    for (int j = threadIdx.x; j < nb; j += kBlk) {
      const int c0 = blockcnt[j];
      t0 += c0;
      if (j < (int)blockIdx.x) {
        s0 += c0;
        s1 += blockcnt[nb + j];
        s2 += blockcnt[2 * nb + j];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      t0 += __shfl_xor_sync(0xffffffffu, t0, o);
    }
    if ((threadIdx.x & 31) == 0) {
      boff[0][threadIdx.x >> 5] = s0;
      boff[1][threadIdx.x >> 5] = s1;
      boff[2][threadIdx.x >> 5] = s2;
      boff[3][threadIdx.x >> 5] = t0;
    }
  }
  int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x;
  int c = i < n ? (int)cls[i] : -1;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned lt = (1u << lane) - 1u;
  bool f[3] = {c == 0 || c == 2, c == 1 || c == 2, c == 2};
  int rank[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    unsigned b = __ballot_sync(0xffffffffu, f[m]);
    rank[m] = __popc(b & lt);
    if (lane == 0) wsum[m][w] = __popc(b);
  }
  __syncthreads();
  int pos[3], tot[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    int off = 0, own = 0;
    if (scanned) {
      off = blockcnt[(int64_t)m * nb + blockIdx.x];
    } else {
      for (int k = 0; k < kBlk / 32; ++k) off += boff[m][k];
    }
    for (int k = 0; k < kBlk / 32; ++k) own += wsum[m][k];
    tot[m] = off + own;  // the list's length when this is the last block
    if (!scanned && blockIdx.x == nb - 1 && threadIdx.x == 0) counters[m] = tot[m];
    for (int k = 0; k < w; ++k) off += wsum[m][k];
    pos[m] = off + rank[m];
  }
  int nm = 0;  // minus-list length: the plus list's records start at 16 ceil(nm/16)
  if (scanned) {
    nm = counters[0];
  } else {
    for (int k = 0; k < kBlk / 32; ++k) nm += boff[3][k];
  }
  const int base_p = 16 * ((nm + 15) / 16);
  if (rec && blockIdx.x == nb - 1 && threadIdx.x < 48) {
    const int m = threadIdx.x >> 4, k = threadIdx.x & 15;
    const int len = tot[m], slot = len + k;
    if (slot < 16 * ((len + 15) / 16)) {
      store_record(m == 2 ? rec_cut + slot : rec + (m == 1 ? base_p : 0) + slot, pad_record());
    }
  }
  if (c < 0) return;
  int cut_id = pos[2];
  if (c == 2) cut_pt[cut_id] = (int)i;
  int e = c == 2 ? -(cut_id + 1) : (int)i;
  if (f[0]) list_m[pos[0]] = e;
  if (f[1]) list_p[pos[1]] = e;
  if (!rec) return;
  if (c == 2) {
    cut_rpos[cut_id] = make_int2(pos[0], base_p + pos[1]);
  } else {
    store_record(rec + (c == 0 ? pos[0] : base_p + pos[1]),
                 uncut_record(P, c, (int)i, X[i], Y[i], Z[i]));
  }
}

// One cut cell per 8 lanes: corner values, tetrahedra and faces are spread
// over the lanes and combined with shuffles.  FP64 is narrow on this part, so
// the per-cell dependency chain, not the operation count, sets the time.
// Lane k's share of a cut cell's closed forms: tetrahedron k of the Kuhn
// split (k < 6; volume fraction / 6, interface area, area-weighted centroid)
// and face k (k < 6; fraction of Omega-).  Fk is the lane's own corner value
// (corner k of the 8 lanes from `base`); the other corners' values come by
// shuffles, corner(c, a) gives coordinate a of corner c.  Every lane of the
// warp calls it (full-mask shuffles); lanes 6 and 7 return nothing.  No array
// is indexed at run time, so nothing goes to local memory.
template <typename T, typename Corner>
__device__ inline void cell_pieces(int k, T Fk, int base, Corner corner, T& vneg, T& area,
                                   T wc[3], T& Afk) {
  const unsigned full = 0xffffffffu;
  const int q = k < 6 ? k : 0;
  // tetrahedron q: corners 0, v1, v2, 7 along the axis order (q/2, second, third)
  const int second = (q == 0 || q == 5) ? 1 : (q == 1 || q == 3) ? 2 : 0;
  const int v1 = 1 << (q >> 1), v2 = v1 | (1 << second);
  const int idx[4] = {0, v1, v2, 7};
  T Xt[4][3], ft[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    ft[t] = __shfl_sync(full, Fk, base + idx[t]);
#pragma unroll
    for (int a = 0; a < 3; ++a) Xt[t][a] = corner(idx[t], a);
  }
  // face q: axis q/2, side q%2, split along the diagonal c00 - c11
  const int a = q >> 1, sd = q & 1, j = (a + 1) % 3, kx = (a + 2) % 3;
  const int c00 = sd << a, c10 = c00 | (1 << j), c01 = c00 | (1 << kx), c11 = c10 | (1 << kx);
  const T F00 = __shfl_sync(full, Fk, base + c00), F10 = __shfl_sync(full, Fk, base + c10);
  const T F01 = __shfl_sync(full, Fk, base + c01), F11 = __shfl_sync(full, Fk, base + c11);
  if (k >= 6) return;
  vneg = frac_tet<T>(ft) / T(6);
  area = tet_iface<T>(Xt, ft, wc);
  Afk = T(0.5) * (frac_tri<T>(F00, F10, F11) + frac_tri<T>(F00, F01, F11));
}

// Cut cell `id` of the list (nc cells) on the 8 lanes of a warp's quarter; the
// whole warp calls it (full-mask shuffles), lanes past the list compute on
// cell 0's point and store nothing.  rec != nullptr: lanes 0..2 also write the
// cell's three tile records (cut list, minus and plus list slots from rpos).
template <bool FP64>
__device__ __forceinline__ void cut_cell_geometry(const ProbDev& P, const float* X,
                                                  const float* Y,
                                                  const float* Z,
                                                  const int* cut_pt, CutRec* cut,
                                                  int id, int nc, PRec* rec, PRec* rec_cut,
                                                  const int2* rpos) {
  const unsigned full = 0xffffffffu;
  const int k = threadIdx.x & 7, base = (threadIdx.x & 31) & ~7;
  const bool live = id < nc;
  const int i = live ? cut_pt[id] : 0;
  const double h = P.h;
  const double p[3] = {(double)X[i], (double)Y[i], (double)Z[i]};
  // Lane k < 6 takes tetrahedron k (volume fraction, interface area and
  // area-weighted centroid) and face k; the 8 lanes then sum.  Outputs:
  // Vm, S (area / h^2), the centroid cen and face fraction Afk of lane k.
  double vneg_d, S_d, Afk_d, cen[3] = {p[0], p[1], p[2]};
  bool has_area;
  float f0f = 0.f, f1f = 0.f;  // FP32 rows: f- and f+ at p
  if constexpr (FP64) {
    // FP64 rows: FP64 corner values and closed forms on absolute coordinates
    double Ck[3];
    for (int a = 0; a < 3; ++a) Ck[a] = p[a] + h * ((double)((k >> a) & 1) - 0.5);
    const double Fk = phi_d(P, Ck[0], Ck[1], Ck[2]);
    double vneg = 0.0, area = 0.0, wc[3] = {0.0, 0.0, 0.0}, Afk = 0.0;
    cell_pieces<double>(
        k, Fk, base, [&](int c, int a) { return p[a] + h * ((double)((c >> a) & 1) - 0.5); },
        vneg, area, wc, Afk);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      vneg += __shfl_xor_sync(full, vneg, o);
      area += __shfl_xor_sync(full, area, o);
      for (int a = 0; a < 3; ++a) wc[a] += __shfl_xor_sync(full, wc[a], o);
    }
    vneg_d = vneg;
    S_d = area / (h * h);
    Afk_d = Afk;
    has_area = area > 0.0;
    if (has_area)
      for (int a = 0; a < 3; ++a) cen[a] = wc[a] / area;
  } else {
    // FP32 rows: corner values with the classifier's rule (FP32 at the same
    // FP32 coordinates; a corner within the FP32 error band of 0 in FP64), so
    // the signs are those that made the cell cut; the closed forms in FP32 on
    // cell-local coordinates (corners at exactly +-1/2, lengths in units of
    // h), where nothing cancels
    const float pf[3] = {X[i], Y[i], Z[i]};
    // f- and f+ at p on every lane (they depend on p only, so their chains
    // overlap the corner values below)
    f0f = rhs_f<float>(P, 0, pf[0], pf[1], pf[2]);
    f1f = rhs_f<float>(P, 1, pf[0], pf[1], pf[2]);
    const float hh = 0.5f * P.hf;
    float Fk = phi_f(P, pf[0] + ((k & 1) ? hh : -hh), pf[1] + ((k & 2) ? hh : -hh),
                     pf[2] + ((k & 4) ? hh : -hh));
    if (fabsf(Fk) < 2e-5f) {  // this corner within the FP32 error band of 0
      const double hd = 0.5 * P.h;
      const double fd = phi_d(P, (double)pf[0] + ((k & 1) ? hd : -hd),
                              (double)pf[1] + ((k & 2) ? hd : -hd),
                              (double)pf[2] + ((k & 4) ? hd : -hd));
      Fk = (float)fd;
      if (Fk == 0.f && fd > 0.0) Fk = __int_as_float(1);  // keep a positive sign
    }
    float vneg = 0.f, area = 0.f, wc[3] = {0.f, 0.f, 0.f}, Afk = 0.f;
    cell_pieces<float>(
        k, Fk, base, [](int c, int a) { return (float)((c >> a) & 1) - 0.5f; }, vneg, area, wc,
        Afk);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      vneg += __shfl_xor_sync(full, vneg, o);
      area += __shfl_xor_sync(full, area, o);
      for (int a = 0; a < 3; ++a) wc[a] += __shfl_xor_sync(full, wc[a], o);
    }
    vneg_d = vneg;
    S_d = area;  // already in units of h^2
    Afk_d = Afk;
    has_area = area > 0.f;
    if (has_area)
      for (int a = 0; a < 3; ++a) cen[a] = p[a] + h * (double)(wc[a] / area);
  }
  double xg[3] = {cen[0], cen[1], cen[2]};
  if (has_area) {
    if constexpr (FP64) {
      for (int it = 0; it < 3; ++it) {  // Newton projection onto phi = 0
        double g[3];
        const double ph = phi_d(P, xg[0], xg[1], xg[2]);
        grad_phi_d(P, xg, g);
        const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        if (gg <= 1e-300) break;
        for (int a = 0; a < 3; ++a) xg[a] -= ph * g[a] / gg;
      }
    } else {
      // FP32 rows: the projection in FP32 (x_G to ~1e-7; both networks and
      // alpha are evaluated at the same x_G)
      float xf[3] = {(float)xg[0], (float)xg[1], (float)xg[2]};
      for (int it = 0; it < 3; ++it) {
        float g[3];
        const float ph = phi_f(P, xf[0], xf[1], xf[2]);
        grad_phi_f(P, xf, g);
        const float gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        if (gg <= 1e-30f) break;
        for (int a = 0; a < 3; ++a) xf[a] -= ph * g[a] / gg;
      }
      for (int a = 0; a < 3; ++a) xg[a] = xf[a];
    }
  }
  // beta, alpha (at x_G), f- and f+ (at p)
  double beta, alpha, f0, f1;
  if constexpr (FP64) {
    // FP64: four functions on four lanes
    double val = 0.0;
    if (k == 0 && has_area) val = beta_d(P, xg);
    else if (k == 1 && has_area) val = alpha_d(P, xg);
    else if (k == 2) val = rhs_f<double>(P, 0, p[0], p[1], p[2]);
    else if (k == 3) val = rhs_f<double>(P, 1, p[0], p[1], p[2]);
    beta = __shfl_sync(full, val, base + 0);
    alpha = __shfl_sync(full, val, base + 1);
    f0 = __shfl_sync(full, val, base + 2);
    f1 = __shfl_sync(full, val, base + 3);
  } else {
    // FP32: beta and alpha on every lane, without branches on the lane, so
    // that their independent chains overlap
    const float xf[3] = {(float)xg[0], (float)xg[1], (float)xg[2]};
    float bt = 0.f, al = 0.f;
    if (has_area) {
      bt = beta_f(P, xf);
      al = alpha_f(P, xf);
    }
    beta = bt;
    alpha = al;
    f0 = f0f;
    f1 = f1f;
  }
  if (!live) return;
  if (rec && k < 3) {
    // the interface point rounded as the fused kernel reads it
    PRec o;
    o.x = X[i];
    o.y = Y[i];
    o.z = Z[i];
    o.gx = (float)xg[0];
    o.gy = (float)xg[1];
    o.gz = (float)xg[2];
    o.pt = i;
    o.cutj = 2 * id + (has_area ? 1 : 0);
    store_record(k == 0 ? rec_cut + id : rec + (k == 1 ? rpos[id].x : rpos[id].y), o);
  }
  CutRec* r = cut + id;
  if (k < 6) r->Am[k] = Afk_d;
  if (k == 0) {
    r->Vm = vneg_d;
    r->S = S_d;
    r->has_jump = has_area;
    for (int a = 0; a < 3; ++a) r->xg[a] = xg[a];
    r->beta = beta;
    r->alpha = alpha;
    r->f[0] = f0;
    r->f[1] = f1;
    r->point = i;
  }
}

// Grid-stride over the cut list in groups of 16 cells (4 per warp), so that
// the grid need not cover the worst case of every point being cut.
// FP64: the FP64-row mode (its own instance: the FP32 one needs fewer
// registers, so more of its warps are resident).
template <bool FP64>
__global__ void __launch_bounds__(128) k_cut_geometry(ProbDev P, const float* X,
                                                      const float* Y,
                                                      const float* Z,
                                                      const int* cut_pt,
                                                      const int* counters,
                                                      CutRec* cut, PRec* rec,
                                                      PRec* rec_cut,
                                                      const int2* rpos) {
  pdl_enter();
  const int nc = counters[2];
  for (int cell0 = blockIdx.x * 16; cell0 < nc; cell0 += gridDim.x * 16) {
    if (cell0 + 4 * (int)(threadIdx.x >> 5) >= nc) break;  // this warp's cells are past the list
    cut_cell_geometry<FP64>(P, X, Y, Z, cut_pt, cut, cell0 + (int)(threadIdx.x >> 3), nc, rec,
                            rec_cut, rpos);
  }
}

// ------------------------------------------------------------------------
// Rows of a cut cell from the outputs of both networks (FP64):
//   B = h^2 sum_s V^s (k^s U^s - f^s) - sum_s sum_f A^s_f mu^s dU^s_f + h S beta,
//   dU^s_{sigma i} = h^2 Mt_i + sigma h Dt_i  or  g(q) - U^s  at the cube boundary,
//   D = sum_s sum_f A^s_f mu^s + h^2 sum_s V^s k^s,   J = U+(xg) - U-(xg) - alpha,
//   r^2 = (B/D)^2 + lambda J^2;   seeds = d(scale r^2)/d(outputs).
// ------------------------------------------------------------------------
// One warp per block.  The row is FP64 (its balance B cancels), and GB300's
// FP64 pipe is narrow.  When the cut list fits in one pass of 4 cells per
// warp (a few thousand cells), each cell takes 8 lanes: lane f < 6 face f of
// both phases, lane 6 the volume terms, the row's sums added by shuffles,
// which cuts each cell's dependency chain to about a sixth.  A longer list is
// bound by the FP64 pipe instead, and takes one cell per thread
// (cut_row_one), so that every lane of each FP64 instruction is busy.  (Rows in
// FP32 were tried: the cancellation in B made the seeds, and so the gradient,
// depend at 1e-5 on how a batch is split into shards.)
// The same row on one thread (cut cell `id`): with many cut cells per warp
// the FP64 pipe, not the chain, is the bound, and one cell per lane keeps
// every lane of each FP64 instruction busy.  Returns r^2.
__device__ inline double cut_row_one(const ProbDev& P, const float* X, const float* Y,
                                     const float* Z, const CutRec* c, const float* o,
                                     float* sd, float scale, float* r2_out) {
  const int i = c->point;
  const double h = P.h, h2 = h * h;
  const double p[3] = {(double)X[i], (double)Y[i], (double)Z[i]};
  double B = 0.0, D = 0.0, dU[2], dM[2][3], dD[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double V = s ? 1.0 - c->Vm : c->Vm;
    const double k = P.k[s];
    const double U = (double)o[8 * s];
    B += h2 * V * (k * U - c->f[s]);
    D += h2 * V * k;
    dU[s] = h2 * V * k;
#pragma unroll
    for (int a = 0; a < 3; ++a) dM[s][a] = dD[s][a] = 0.0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1;
      const double sg = (f & 1) ? 1.0 : -1.0;
      double q[3] = {p[0], p[1], p[2]}, fc[3] = {p[0], p[1], p[2]};
      q[a] += sg * h;
      fc[a] += 0.5 * sg * h;
      const double A = s ? 1.0 - c->Am[f] : c->Am[f];
      const double w = A * mu_at<double>(P, s, fc[0], fc[1], fc[2]);
      D += w;
      if (fabs(q[a]) >= 1.0) {
        B -= w * (dirichlet_g<double>(P, q[0], q[1], q[2]) - U);
        dU[s] += w;
      } else {
        B -= w * (h2 * (double)o[8 * s + 1 + a] + sg * h * (double)o[8 * s + 4 + a]);
        dM[s][a] -= w * h2;
        dD[s][a] -= w * sg * h;
      }
    }
  }
  const bool jump = c->has_jump;
  if (jump) B += h * c->S * c->beta;
  const double J = jump ? (double)o[15] - (double)o[7] - c->alpha : 0.0;
  const double rB = B / D;
  const double r2 = rB * rB + P.lambda * J * J;
  if (sd) {
    const double cB = (double)scale * 2.0 * rB / D;
    const double cJ = (double)scale * 2.0 * P.lambda * J;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      sd[8 * s] = (float)(cB * dU[s]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        sd[8 * s + 1 + a] = (float)(cB * dM[s][a]);
        sd[8 * s + 4 + a] = (float)(cB * dD[s][a]);
      }
      sd[8 * s + 7] = jump ? (float)(s ? cJ : -cJ) : 0.f;
    }
  }
  if (r2_out) r2_out[i] = (P.level ? r2_out[i] : 0.f) + (float)r2;
  return r2;
}

__global__ void __launch_bounds__(32) k_cut_residual(ProbDev P, const float* X, const float* Y,
                                                      const float* Z, const int* counters,
                                                      const CutRec* cut, const float* out,
                                                      float* seeds, float scale, float* r2_out,
                                                      double* loss_part) {
  pdl_enter();
  const unsigned full = 0xffffffffu;
  const int nc = counters[2];
  const int l = threadIdx.x & 7, sub = threadIdx.x >> 3;
  const double h = P.h, h2 = h * h;
  double r2_sum = 0.0;  // this lane's cells' r^2, then the block partial
  if (nc > 4 * (int)gridDim.x) {
    // more cells than one pass of 4 per warp: one cell per thread
    for (int id = blockIdx.x * 32 + threadIdx.x; id < nc; id += gridDim.x * 32)
      r2_sum += cut_row_one(P, X, Y, Z, cut + id, out + (int64_t)id * 16,
                            seeds ? seeds + (int64_t)id * 16 : nullptr, scale, r2_out);
  } else {
    // 4 cells per warp, 8 lanes per cell
    for (int first = blockIdx.x * 4; first < nc; first += gridDim.x * 4) {  // warp-uniform
      const int id = first + sub;
      const bool live = id < nc;
      const CutRec* c = cut + (live ? id : first);  // fields read where needed (no local copy)
      const int i = c->point;
      const double p[3] = {(double)X[i], (double)Y[i], (double)Z[i]};
      const float* o = out + (int64_t)(live ? id : first) * 16;
      // this lane's share of B, D, dU^s and (faces) dM^s, dD^s of its axis
      double B = 0.0, D = 0.0, dU0 = 0.0, dU1 = 0.0, dm0 = 0.0, dm1 = 0.0, dd0 = 0.0, dd1 = 0.0;
      if (l < 6) {
        const int ax = l >> 1;
        const double sg = (l & 1) ? 1.0 : -1.0;
        // neighbour q and face centre fc (selects: the arrays stay in registers)
        const double dq = sg * h, df = 0.5 * sg * h;
        const double q0 = ax == 0 ? p[0] + dq : p[0], q1 = ax == 1 ? p[1] + dq : p[1],
                     q2 = ax == 2 ? p[2] + dq : p[2];
        const double f0 = ax == 0 ? p[0] + df : p[0], f1 = ax == 1 ? p[1] + df : p[1],
                     f2 = ax == 2 ? p[2] + df : p[2];
        const bool bnd = fabs(ax == 0 ? q0 : ax == 1 ? q1 : q2) >= 1.0;
        const double g = bnd ? dirichlet_g<double>(P, q0, q1, q2) : 0.0;
        const double Aml = c->Am[l];
  #pragma unroll
        for (int s = 0; s < 2; ++s) {
          const double A = s ? 1.0 - Aml : Aml;
          // mu^s at the face centre (constant for the benchmark pair)
          const double w = A * mu_at<double>(P, s, f0, f1, f2);
          const double U = (double)o[8 * s];
          D += w;
          double du = 0.0, dm = 0.0, dd = 0.0;
          if (bnd) {
            // U^s(p) enters the row directly only through Dirichlet faces: the
            // interior faces carry it inside the increments Mt, Dt
            B -= w * (g - U);
            du = w;
          } else {
            B -= w * (h2 * (double)o[8 * s + 1 + ax] + sg * h * (double)o[8 * s + 4 + ax]);
            dm = -w * h2;
            dd = -w * sg * h;
          }
          if (s == 0) { dU0 = du; dm0 = dm; dd0 = dd; }
          else { dU1 = du; dm1 = dm; dd1 = dd; }
        }
      } else if (l == 6) {
  #pragma unroll
        for (int s = 0; s < 2; ++s) {
          const double V = s ? 1.0 - c->Vm : c->Vm;
          const double k = P.k[s];
          const double U = (double)o[8 * s];
          B += h2 * V * (k * U - c->f[s]);
          D += h2 * V * k;
          if (s == 0) dU0 = h2 * V * k;
          else dU1 = h2 * V * k;
        }
        if (c->has_jump) B += h * c->S * c->beta;
      }
      // the two faces of an axis: lanes 2a, 2a + 1
      dm0 += __shfl_xor_sync(full, dm0, 1, 8);
      dm1 += __shfl_xor_sync(full, dm1, 1, 8);
      dd0 += __shfl_xor_sync(full, dd0, 1, 8);
      dd1 += __shfl_xor_sync(full, dd1, 1, 8);
  #pragma unroll
      for (int m = 1; m < 8; m <<= 1) {
        B += __shfl_xor_sync(full, B, m, 8);
        D += __shfl_xor_sync(full, D, m, 8);
        dU0 += __shfl_xor_sync(full, dU0, m, 8);
        dU1 += __shfl_xor_sync(full, dU1, m, 8);
      }
      const bool jump = c->has_jump;
      const double J = jump ? (double)o[15] - (double)o[7] - c->alpha : 0.0;
      const double rB = B / D;
      const double r2 = rB * rB + P.lambda * J * J;
      // seed column l of both networks: 0 dU, 1..3 dM of axis l-1, 4..6 dD of
      // axis l-4 (held by lane 2 axis), 7 the jump
      const int src = (l >= 1 && l <= 3) ? 2 * (l - 1) : (l >= 4 && l <= 6) ? 2 * (l - 4) : 0;
      const double m0 = __shfl_sync(full, dm0, src, 8), m1 = __shfl_sync(full, dm1, src, 8);
      const double e0 = __shfl_sync(full, dd0, src, 8), e1 = __shfl_sync(full, dd1, src, 8);
      if (!live) continue;
      if (seeds) {
        const double cB = (double)scale * 2.0 * rB / D;
        const double cJ = (double)scale * 2.0 * P.lambda * J;
        float* sd = seeds + (int64_t)id * 16;
        if (l == 7) {
          sd[7] = jump ? (float)(-cJ) : 0.f;
          sd[15] = jump ? (float)cJ : 0.f;
        } else {
          const double v0 = l == 0 ? dU0 : l <= 3 ? m0 : e0;
          const double v1 = l == 0 ? dU1 : l <= 3 ? m1 : e1;
          sd[l] = (float)(cB * v0);
          sd[8 + l] = (float)(cB * v1);
        }
      }
      if (l == 0) {
        if (r2_out) r2_out[i] = (P.level ? r2_out[i] : 0.f) + (float)r2;
        r2_sum += r2;
      }
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) r2_sum += __shfl_xor_sync(full, r2_sum, m);
  if (threadIdx.x == 0) loss_part[blockIdx.x] = r2_sum;
}

// ------------------------------------------------------------------------
// Tile records in list order, one thread per record, for batches of more
// than 2048 point blocks (the scan path).  There the records and the cut
// cells' geometry together outgrow L2, and records written in list order
// right before the cut-cell forward and the fused kernel read them cost less
// than records written by the scatter and the cut geometry as they go.  The
// same records as those two write: rec = minus list, then plus list (each
// padded to a multiple of 16), rec_cut = cut list (padded).
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather_tiles(const ProbDev P, const int* counters,
                                                      const int* list_m, const int* list_p,
                                                      const int* cut_pt, const float* X,
                                                      const float* Y, const float* Z,
                                                      const CutRec* cut, PRec* rec,
                                                      PRec* rec_cut) {
  pdl_enter();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nm = counters[0], np = counters[1], nc = counters[2];
  const int64_t base_p = 16 * (int64_t)((nm + 15) / 16);
  const int64_t end_p = base_p + 16 * (int64_t)((np + 15) / 16);
  // the record of list entry e (>= 0 uncut point of phase s, < 0 cut cell)
  auto entry = [&](int e, int s) {
    if (e >= 0) return uncut_record(P, s, e, X[e], Y[e], Z[e]);
    const int id = -e - 1, pt = cut_pt[id];
    const CutRec& c = cut[id];
    PRec o;
    o.x = X[pt];
    o.y = Y[pt];
    o.z = Z[pt];
    o.gx = (float)c.xg[0];
    o.gy = (float)c.xg[1];
    o.gz = (float)c.xg[2];
    o.pt = pt;
    o.cutj = 2 * id + (c.has_jump ? 1 : 0);
    return o;
  };
  if (r < end_p) {
    const bool minus = r < base_p;
    const int64_t slot = minus ? r : r - base_p;
    const bool live = slot < (minus ? nm : np);
    store_record(rec + r, live ? entry((minus ? list_m : list_p)[slot], minus ? 0 : 1)
                                : pad_record());
  }
  if (r < 16 * (int64_t)((nc + 15) / 16))
    store_record(rec_cut + r, r < nc ? entry(-(int)r - 1, 0) : pad_record());
}

// Standalone restage (grid evaluation); the training paths restage inside
// their sampling launch (k_sample_classify's extra blocks).
__global__ void k_prep_weights(ProbDev P, const float* params, float* wt, void* wtc,
                               int prec) {
  pdl_enter();
  prep_weights_blocks(P, params, wt, wtc, prec, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------------
// Finish: loss (fixed-order sums), then gradient reduction over CTA partials
// (fixed order) and, when training, Adam (Kingma & Ba, bias-corrected).
// ------------------------------------------------------------------------
// Where the loss of the step goes.  With refinement levels, the levels' losses
// are summed in *loss_acc (acc_in: add the levels done so far; last == 0: only
// accumulate) and the step is finished after the last level.
struct LossOut {
  const double* lp;  // [nlp] loss partials of the fused kernel's CTAs
  int nlp;
  const double* clp;  // [nclp] loss partials of the cut-row blocks
  int nclp;
  double scale;       // 1/N
  double* loss;
  int64_t* step;      // non-NULL: advance the device step counter
  float* loss_hist;
  int64_t hist_base;
  int* status;
  double* loss_acc;
  int acc_in, last;
};

// Sum of the step's loss partials on a block of 256 threads, in three parts
// so that a caller can overlap the loads with other work: thread-strided
// partial sums (loss_thread_sum), warp shuffles into red8 (loss_warp_sum), a
// __syncthreads by the caller, then the 8 warp sums in a fixed order
// (finish_loss).  Every block that does this gets the same value.
__device__ inline double loss_thread_sum(const LossOut& o) {
  double s = 0.0;
  for (int j = threadIdx.x; j < o.nlp; j += 256) s += o.lp[j];
  for (int j = threadIdx.x; j < o.nclp; j += 256) s += o.clp[j];
  return s;
}

__device__ inline void loss_warp_sum(double s, double* red8) {
#pragma unroll
  for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
  if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = s;
}

// L = scale * (sum of the partials) (+ the earlier levels' sum) from the warp
// sums in red8; with `store`, thread 0 stores it (and finishes the step when
// `last`).
__device__ inline double finish_loss(const LossOut& o, const double* red8, bool store) {
  double t8 = red8[0];
  for (int w = 1; w < 8; ++w) t8 += red8[w];
  double L = t8 * o.scale;
  if (o.acc_in) L += *o.loss_acc;
  if (!store || threadIdx.x != 0) return L;
  if (!o.last) {
    *o.loss_acc = L;
    return L;
  }
  *o.loss = L;
  if (!isfinite(L)) atomicOr(o.status, 1);
  if (o.step) {
    const int64_t t = *o.step + 1;
    *o.step = t;
    if (o.loss_hist) o.loss_hist[t - o.hist_base - 1] = (float)L;
  }
  return L;
}

// Loss only (a step with neither gradient nor update).
__global__ void k_loss(LossOut o) {
  pdl_enter();
  __shared__ double red[8];
  loss_warp_sum(loss_thread_sum(o), red);
  __syncthreads();
  finish_loss(o, red, true);
}

// Loss and gradient of the step (fixed CTA order), then Adam.  Block 0 stores
// the loss (finish_loss); every block of an Adam step that is the last level
// sums the same partials in the same order itself, to skip the update of a
// non-finite step without waiting for block 0.  With refinement levels the
// levels' gradients are summed in gacc: gacc_in (levels done so far) is
// added, and a level that is not the last stores the sum in gacc_out and stops
// (only block 0 then touches the loss: it alone reads and writes *loss_acc).
// Block of 256 threads on 128 consecutive parameters of one network: warp cg
// sums the per-CTA partial slices cg, cg + 8, ... (lane l: parameters 4l..4l+3
// of the block, one float4 per slice, every slice loaded and the slice of a
// CTA that stopped early dropped by a select, so the loads do not wait for the
// flags); then thread t < 128 adds the 8 group sums of parameter t in a fixed
// order, so the sum is deterministic, and applies the update.
__global__ void __launch_bounds__(256) k_reduce_adam(ProbDev P, int grid, int nb_net,
                                                     const float* gpart,
                                                     const int* flag,
                                                     float* grad_out, float* params, float* m,
                                                     float* v, float lr, float b1, float b2,
                                                     float eps, float c1, float c2,
                                                     LossOut lo, float* wt, void* wtc,
                                                     int prec, const float* gacc_in,
                                                     float* gacc_out) {
  pdl_enter();
  __shared__ float4 red[8][32];
  __shared__ double red8[8];
  // the loss partials' loads overlap the gradient slices' loads
  const bool want_loss = blockIdx.x == 0 || (params && lo.last);  // block-uniform
  const double ls = want_loss ? loss_thread_sum(lo) : 0.0;
  const int pn = (int)P.p_net;
  const int s = blockIdx.x >= nb_net ? 1 : 0;
  const int blk = blockIdx.x - s * nb_net;
  const int lane = threadIdx.x & 31, cg = threadIdx.x >> 5;
  const int j4 = (blk * 32 + lane) * 4;  // within the network; < gstride when < pn
  float4 part = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j4 < pn) {
    const float* src = gpart + (int64_t)s * P.gstride + j4;
#pragma unroll 8
    for (int c = cg; c < grid; c += 8) {
      const float4 g = __ldcg(reinterpret_cast<const float4*>(src + (int64_t)c * 2 * P.gstride));
      const bool f = flag[2 * c + s] != 0;
      part.x += f ? g.x : 0.f;
      part.y += f ? g.y : 0.f;
      part.z += f ? g.z : 0.f;
      part.w += f ? g.w : 0.f;
    }
  }
  red[cg][lane] = part;
  if (want_loss) loss_warp_sum(ls, red8);
  __syncthreads();
  const double L = want_loss ? finish_loss(lo, red8, blockIdx.x == 0) : 0.0;
  const int t = threadIdx.x;
  const int jj = blk * 128 + t;
  if (t >= 128 || jj >= pn) return;
  float g = reinterpret_cast<const float*>(red[0])[t];
#pragma unroll
  for (int q = 1; q < 8; ++q) g += reinterpret_cast<const float*>(red[q])[t];
  const int64_t j = (int64_t)s * pn + jj;
  if (gacc_in) g += gacc_in[j];
  if (gacc_out) {
    gacc_out[j] = g;
    return;
  }
  if (grad_out) grad_out[j] = g;
  if (!params) return;
  if (!isfinite(L)) return;  // non-finite step: skip the update
  float mj = b1 * m[j] + (1.f - b1) * g;
  float vj = b2 * v[j] + (1.f - b2) * g * g;
  m[j] = mj;
  v[j] = vj;
  float mh = mj / c1, vh = vj / c2;
  float w = params[j] - lr * mh / (sqrtf(vh) + eps);
  params[j] = w;
  // restage hidden weights for the next step
  const int H = P.H;
  const int per = H * H;
  if (jj >= 4 * H && jj < 4 * H + (P.L - 1) * (per + H)) {
    const int q = jj - 4 * H;
    const int l = q / (per + H) + 1;
    const int rem = q - (l - 1) * (per + H);
    if (rem < per) {
      const int u = rem / H, k = rem - u * H;
      const int64_t wb = (int64_t)s * (P.L - 1) + (l - 1);
      if (wt) wt[wb * per + (int64_t)k * H + u] = w;
      if (wtc && H == 128) {
        char* base = (char*)wtc + wb * per * 2;
        if (prec == NBM_PREC_FP16) *(__half*)(base + tc_tile_offset(u, k)) = __float2half_rn(w);
        else *(__nv_bfloat16*)(base + tc_tile_offset(u, k)) = __float2bfloat16_rn(w);
      }
    }
  }
}

// One Adam update (Kingma & Ba, bias-corrected) with a gradient the caller
// supplies, e.g. the sum of the data-parallel shards' gradients (Sec. 3: the
// locally computed gradient updates are aggregated).  Element for element the
// arithmetic of the update in k_reduce_adam, so one shard covering the whole
// batch reproduces nbm_train_steps bitwise.
__global__ void k_adam(int64_t n, float* params, float* m,
                       float* v, const float* grad, float lr, float b1,
                       float b2, float eps, float c1, float c2,
                       const double* loss) {
  pdl_enter();
  if (loss && !isfinite(*loss)) return;  // non-finite step: skip the update
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float g = grad[j];
    const float mj = b1 * m[j] + (1.f - b1) * g;
    const float vj = b2 * v[j] + (1.f - b2) * g * g;
    m[j] = mj;
    v[j] = vj;
    const float mh = mj / c1, vh = vj / c2;
    params[j] = params[j] - lr * mh / (sqrtf(vh) + eps);
  }
}

// ------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------
float adam_correction(float beta, int64_t t) {
  return (float)(1.0 - std::pow((double)beta, (double)t));
}

cudaError_t launch_adam(int64_t n, float* params, float* m, float* v, const float* grad, float lr,
                        float b1, float b2, float eps, int64_t t, const double* loss,
                        cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  return launch_pdl(k_adam, dim3((unsigned)(blocks < 1024 ? blocks : 1024)), dim3(256), 0, st, n,
                    params, m, v, grad, lr, b1, b2, eps, adam_correction(b1, t),
                    adam_correction(b2, t), loss);
}

cudaError_t launch_sample_classify(const ProbDev& P, const float* pts_in, uint64_t seed,
                                   const int64_t* step_dev, int64_t step_host, int64_t n,
                                   int64_t n_band, Workspace& ws, cudaStream_t st,
                                   int64_t first, int64_t n_total, const float* prep_params,
                                   int prec, bool tiles) {
  int nb = (int)((n + kBlk - 1) / kBlk);
  const int npb = prep_params ? prep_weight_blocks(P) : 0;
  cudaError_t e = launch_pdl(k_sample_classify, dim3(nb + npb), dim3(kBlk), 0, st, P, pts_in,
                             seed, step_dev, step_host, n, n_band, ws.x, ws.y, ws.z, ws.cls,
                             ws.blockcnt, nb, first, n_total > 0 ? n_total : n, prep_params,
                             ws.wt, (prec == NBM_PREC_FP32) ? nullptr : ws.wtc, prec);
  // up to 2048 blocks the scatter blocks sum the earlier blocks' counts
  // themselves (at most 6 K integers each) and write the tile records;
  // beyond, one scan kernel, and the records come from k_gather_tiles
  const int scanned = tiles_in_scatter(n) ? 0 : 1;
  if (scanned) tiles = false;
  if (e == cudaSuccess && scanned)
    e = launch_pdl(k_scan_counts, dim3(1), dim3(1024), 0, st, ws.blockcnt, nb, ws.counters);
  if (e == cudaSuccess)
    e = launch_pdl(k_scatter, dim3(nb), dim3(kBlk), 0, st, P, (const uint8_t*)ws.cls, n,
                   (const int*)ws.blockcnt, nb, scanned, ws.list_minus, ws.list_plus,
                   ws.cut_pt, ws.counters, (const float*)ws.x, (const float*)ws.y,
                   (const float*)ws.z, tiles ? ws.rec : nullptr, ws.rec_cut, ws.cut_rpos);
  return e;
}

bool tiles_in_scatter(int64_t n) { return (n + kBlk - 1) / kBlk <= kScatterPrefixBlocks; }

cudaError_t launch_gather_tiles(const ProbDev& P, int64_t n, Workspace& ws, cudaStream_t st) {
  const int64_t worst = 2 * n + 32;  // both lists, padded
  return launch_pdl(k_gather_tiles, dim3((unsigned)((worst + 255) / 256)), dim3(256), 0, st, P,
                    (const int*)ws.counters, (const int*)ws.list_minus,
                    (const int*)ws.list_plus, (const int*)ws.cut_pt, (const float*)ws.x,
                    (const float*)ws.y, (const float*)ws.z, (const CutRec*)ws.cut, ws.rec,
                    ws.rec_cut);
}

cudaError_t launch_cut_geometry(const ProbDev& P, int64_t n, Workspace& ws, cudaStream_t st,
                                bool tiles) {
  if (!tiles_in_scatter(n)) tiles = false;
  // 8 lanes per cut cell, 16 cells per block; at most 8 blocks per SM, each
  // striding over the cut list
  const int64_t worst = (n + 15) / 16, cap = 8 * (int64_t)ws.grid;
  int nb = (int)(worst < cap ? worst : cap);
  return launch_pdl(P.fp64 ? k_cut_geometry<true> : k_cut_geometry<false>, dim3(nb), dim3(128), 0,
                    st, P, (const float*)ws.x, (const float*)ws.y, (const float*)ws.z,
                    (const int*)ws.cut_pt, (const int*)ws.counters, ws.cut,
                    tiles ? ws.rec : nullptr, ws.rec_cut, (const int2*)ws.cut_rpos);
}

// blocks of the cut-row kernel (grid-stride over the cut cells), i.e. the
// number of its loss partials
int cut_residual_blocks(int64_t n, const Workspace& ws) {
  const int64_t worst = (n + 31) / 32, cap = 8 * (int64_t)ws.grid;
  return (int)(worst < cap ? worst : cap);
}

cudaError_t launch_cut_residual(const ProbDev& P, int64_t n, float scale, bool want_seeds,
                                float* r2_out, Workspace& ws, cudaStream_t st) {
  int nb = cut_residual_blocks(n, ws);
  return launch_pdl(k_cut_residual, dim3(nb), dim3(32), 0, st, P, ws.x, ws.y, ws.z, ws.counters,
                    ws.cut, ws.cut_out, want_seeds ? ws.cut_seed : nullptr, scale, r2_out,
                    ws.cut_loss_part);
}

cudaError_t launch_prep_weights(const ProbDev& P, const float* params, int prec, Workspace& ws,
                                cudaStream_t st) {
  return launch_pdl(k_prep_weights, dim3(prep_weight_blocks(P)), dim3(256), 0, st, P, params, ws.wt,
                    (prec == NBM_PREC_FP32) ? nullptr : ws.wtc, prec);
}

cudaError_t launch_finish(const ProbDev& P, int64_t n, int grid, bool adam, bool want_grad,
                          float* params, float* m, float* v, float* grad_out, float lr, float b1,
                          float b2, float eps, float* loss_hist, int64_t hist_base, int prec,
                          Workspace& ws, cudaStream_t st, int level, int n_levels,
                          double loss_scale, int64_t adam_t) {
  const bool last = level == n_levels - 1;
  const float c1 = adam ? adam_correction(b1, adam_t) : 1.f;
  const float c2 = adam ? adam_correction(b2, adam_t) : 1.f;
  LossOut lo;
  lo.lp = ws.loss_part;
  lo.nlp = grid;
  lo.clp = ws.cut_loss_part;
  lo.nclp = cut_residual_blocks(n, ws);
  lo.scale = loss_scale > 0.0 ? loss_scale : 1.0 / (double)n;
  lo.loss = ws.loss;
  lo.step = adam ? ws.step : nullptr;
  lo.loss_hist = loss_hist;
  lo.hist_base = hist_base;
  lo.status = ws.status;
  lo.loss_acc = ws.loss_acc;
  lo.acc_in = (int)(level > 0);
  lo.last = (int)last;
  if (!(adam || want_grad)) return launch_pdl(k_loss, dim3(1), dim3(256), 0, st, lo);
  // the reduction kernel finishes the loss too
  const int nb_net = (int)((P.p_net + 127) / 128);
  cudaError_t e =
      launch_pdl(k_reduce_adam, dim3(2 * nb_net), dim3(256), 0, st, P, grid, nb_net, ws.gpart,
                 (const int*)ws.gpart_flag, grad_out, adam ? params : nullptr, m, v, lr, b1, b2,
                 eps, c1, c2, lo, ws.wt, (prec == NBM_PREC_FP32) ? nullptr : ws.wtc, prec,
                 (const float*)(level > 0 ? ws.gacc : nullptr), last ? nullptr : ws.gacc);
  return e;
}

}  // namespace nbm
