// nbm_device.cuh -- device-side building blocks of the NBM training step
// (arXiv 2210.14907, Sec. 2-3): problem constants, Philox4x32-10, level sets,
// manufactured data, the difference-form tanh layer and its adjoint, and the
// per-point balance/jump rows.  Shared by every kernel translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbm_host.h"

namespace nbm {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of a training step are
// launched with programmatic stream serialization (launch_pdl), so that a
// kernel's launch is processed while its predecessor in the stream finishes.
// Every such kernel begins with pdl_enter(), which waits until the
// predecessor grid has completed and its writes are visible.  No kernel
// signals an early launch of its successor (the implicit signal is at grid
// completion), and data that an earlier kernel of the step writes is read
// with ordinary loads (no __restrict__ / __ldg read-only path), so that no
// read of it can be scheduled before the wait.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Problem constants, passed by value to every kernel.
// ---------------------------------------------------------------------------
struct ProbDev {
  int geometry;  // nbm_geometry
  int H, L;      // width, number of tanh layers
  int fp64;      // residual combination in FP64
  double r0, amp, lt, lp;
  double mu[2], k[2];
  double h, lambda;
  double h_band;   // base spacing: band points are drawn within 4 h_band of Gamma
  int level;       // refinement level of this pass (0: base cell; > 0 accumulates r2_out)
  int solution;    // manufactured pair: 0 benchmark (constant mu), 1 Sec. 4.1 (variable mu)
  int activation;  // hidden-layer activation: 0 tanh, 1 sin
  int phi_n;              // NBM_GEOM_GRID: cells per axis of the level-set mesh
  const double* phi_grid; // NBM_GEOM_GRID: (phi_n+1)^3 node values, x fastest
  float hf, inv_hf, h2f, inv_h2f;  // h, 1/h, h^2, 1/h^2 in FP32
  float r0f, ampf, ltf, lpf;
  float muf[2], kf[2];
  double inv_h, inv_h2, inv_D[2];  // 1/h, 1/h^2, 1/(6 mu_s + h^2 k_s) of the uncut rows
  float inv_Df[2];
  int lt_i, lp_i;  // flower lobe counts when integers (else -1): Chebyshev evaluation
  int64_t p_net;  // parameters per network
  int64_t gstride;  // per-CTA partial-gradient slice stride (p_net rounded up to 4)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011).
// ---------------------------------------------------------------------------
__host__ __device__ inline void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
#ifdef __CUDA_ARCH__
    uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
#else
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

constexpr uint32_t kPointStream = 0x4E424D31u;  // 4th counter word of point draws

// ---------------------------------------------------------------------------
// Level sets (Sec. 3: the level set gives the cell/interface crossings).
// theta = atan2(rho, z) is the polar angle, psi = atan2(y, x) the azimuth.
// ---------------------------------------------------------------------------
// Level set stored on a coarse mesh (NBM_GEOM_GRID): the trilinear interpolant
// of the node values in the mesh cell containing x (index floor((x+1) n/2),
// clamped to the last cell on the upper faces), and its gradient in that cell.
template <typename T>
__device__ inline T grid_phi(const ProbDev& P, T x, T y, T z, T* g) {
  const int n = P.phi_n;
  const int64_t N1 = n + 1;
  const T sc = (T)0.5 * (T)n;
  const T t[3] = {(x + (T)1) * sc, (y + (T)1) * sc, (z + (T)1) * sc};
  int i[3];
  T f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int c = (int)floor(t[a]);
    c = c < 0 ? 0 : (c > n - 1 ? n - 1 : c);
    i[a] = c;
    f[a] = t[a] - (T)c;
  }
  const double* cg = P.phi_grid + i[0] + N1 * (i[1] + N1 * (int64_t)i[2]);
  const int64_t sy = N1, sz = N1 * N1;
  const T c000 = (T)cg[0], c100 = (T)cg[1], c010 = (T)cg[sy], c110 = (T)cg[sy + 1];
  const T c001 = (T)cg[sz], c101 = (T)cg[sz + 1], c011 = (T)cg[sz + sy], c111 = (T)cg[sz + sy + 1];
  const T c00 = c000 * ((T)1 - f[0]) + c100 * f[0], c10 = c010 * ((T)1 - f[0]) + c110 * f[0];
  const T c01 = c001 * ((T)1 - f[0]) + c101 * f[0], c11 = c011 * ((T)1 - f[0]) + c111 * f[0];
  const T c0 = c00 * ((T)1 - f[1]) + c10 * f[1], c1 = c01 * ((T)1 - f[1]) + c11 * f[1];
  if (g) {
    g[0] = sc * (((c100 - c000) * ((T)1 - f[1]) + (c110 - c010) * f[1]) * ((T)1 - f[2]) +
                 ((c101 - c001) * ((T)1 - f[1]) + (c111 - c011) * f[1]) * f[2]);
    g[1] = sc * ((c10 - c00) * ((T)1 - f[2]) + (c11 - c01) * f[2]);
    g[2] = sc * (c1 - c0);
  }
  return c0 * ((T)1 - f[2]) + c1 * f[2];
}

// Chebyshev recurrences: cos(n a) = T_n(c), sin(n a) = sin(a) U_{n-1}(c) for
// c = cos(a).  Returns T_n(c) and U_{n-1}(c) (n >= 0; U_{-1} = 0).
template <typename T>
__device__ inline void chebyshev_tu(int n, T c, T& Tn, T& Un1) {
  T t0 = T(1), t1 = c, u0 = T(0), u1 = T(1);
  for (int k = 1; k < n; ++k) {
    const T t2 = T(2) * c * t1 - t0, u2 = T(2) * c * u1 - u0;
    t0 = t1;
    t1 = t2;
    u0 = u1;
    u1 = u2;
  }
  Tn = n == 0 ? T(1) : t1;
  Un1 = n == 0 ? T(0) : u1;
}

// The flower's angular factors from cos/sin of the polar angle theta and the
// azimuth psi: sin(lt theta), cos(lt theta), cos(lp psi), sin(lp psi).  Integer
// lobe counts (the configurations here) take the Chebyshev recurrences and no
// transcendental function; other counts go through the angles.
template <typename T>
__device__ inline void flower_factors(const ProbDev& P, T cth, T sth, T cps, T sps, T& st, T& ct,
                                      T& cp, T& sp) {
  if (P.lt_i >= 0) {
    T Tn, Un;
    chebyshev_tu<T>(P.lt_i, cth, Tn, Un);
    ct = Tn;
    st = sth * Un;
  } else {
    const T a = (sizeof(T) == 4 ? (T)P.ltf : (T)P.lt) * atan2(sth, cth);
    st = sin(a);
    ct = cos(a);
  }
  if (P.lp_i >= 0) {
    T Tn, Un;
    chebyshev_tu<T>(P.lp_i, cps, Tn, Un);
    cp = Tn;
    sp = sps * Un;
  } else {
    const T a = (sizeof(T) == 4 ? (T)P.lpf : (T)P.lp) * atan2(sps, cps);
    sp = sin(a);
    cp = cos(a);
  }
}

// phi = r - r0 - amp sin(lt theta) cos(lp psi) (flower), r - r0 (sphere)
template <typename T>
__device__ inline T phi_t(const ProbDev& P, T x, T y, T z) {
  if (P.geometry == NBM_GEOM_GRID) return grid_phi<T>(P, x, y, z, nullptr);
  if (P.geometry == NBM_GEOM_ALL_PLUS) return T(1);
  if (P.geometry == NBM_GEOM_ALL_MINUS) return T(-1);
  const T r0 = sizeof(T) == 4 ? (T)P.r0f : (T)P.r0, amp = sizeof(T) == 4 ? (T)P.ampf : (T)P.amp;
  const T rho2 = x * x + y * y;
  const T r = sqrt(rho2 + z * z);
  if (P.geometry == NBM_GEOM_SPHERE) return r - r0;
  if (r == T(0)) return -r0;
  const T rho = sqrt(rho2);
  const T cps = rho > T(0) ? x / rho : T(1), sps = rho > T(0) ? y / rho : T(0);
  T st, ct, cp, sp;
  flower_factors<T>(P, z / r, rho / r, cps, sps, st, ct, cp, sp);
  return r - r0 - amp * st * cp;
}
__device__ inline float phi_f(const ProbDev& P, float x, float y, float z) {
  return phi_t<float>(P, x, y, z);
}
__device__ inline double phi_d(const ProbDev& P, double x, double y, double z) {
  return phi_t<double>(P, x, y, z);
}

// grad phi: x / r, plus for the flower the derivatives of the angular factor
// through theta and psi
template <typename T>
__device__ inline void grad_phi_t(const ProbDev& P, const T x[3], T g[3]) {
  if (P.geometry == NBM_GEOM_GRID) {
    grid_phi<T>(P, x[0], x[1], x[2], g);
    return;
  }
  g[0] = g[1] = g[2] = T(0);
  if (P.geometry == NBM_GEOM_ALL_PLUS || P.geometry == NBM_GEOM_ALL_MINUS) return;
  const T rho = sqrt(x[0] * x[0] + x[1] * x[1]);
  const T r = sqrt(rho * rho + x[2] * x[2]);
  if (r == T(0)) return;
  for (int i = 0; i < 3; ++i) g[i] = x[i] / r;
  if (P.geometry != NBM_GEOM_FLOWER || rho == T(0)) return;
  const T amp = sizeof(T) == 4 ? (T)P.ampf : (T)P.amp;
  const T lt = sizeof(T) == 4 ? (T)P.ltf : (T)P.lt, lp = sizeof(T) == 4 ? (T)P.lpf : (T)P.lp;
  T st, ct, cp, sp;
  flower_factors<T>(P, x[2] / r, rho / r, x[0] / rho, x[1] / rho, st, ct, cp, sp);
  const T r2 = r * r;
  const T dth[3] = {x[2] * x[0] / (r2 * rho), x[2] * x[1] / (r2 * rho), -rho / r2};
  const T dps[3] = {-x[1] / (rho * rho), x[0] / (rho * rho), T(0)};
  const T ga = -amp * lt * ct * cp;
  const T gb = amp * lp * st * sp;
  for (int i = 0; i < 3; ++i) g[i] += ga * dth[i] + gb * dps[i];
}
__device__ inline void grad_phi_d(const ProbDev& P, const double x[3], double g[3]) {
  grad_phi_t<double>(P, x, g);
}

// ---------------------------------------------------------------------------
// Manufactured pairs.  Solution 0 (the benchmark configurations), constant
// mu^s:  u- = e^x cos y sin z (Lap u- = -u-),  u+ = |x|^2 (Lap u+ = 6).
// Solution 1 (Sec. 4.1):  u- = e^z,  u+ = cos x sin y,  mu- = y^2 ln(x+2) + 4,
// mu+ = e^-z.  (The FP32 overloads call CUDA's float functions.)
// ---------------------------------------------------------------------------
__device__ inline double m_exp(double v) { return exp(v); }
__device__ inline float m_exp(float v) { return expf(v); }
__device__ inline double m_cos(double v) { return cos(v); }
__device__ inline float m_cos(float v) { return cosf(v); }
__device__ inline double m_sin(double v) { return sin(v); }
__device__ inline float m_sin(float v) { return sinf(v); }
__device__ inline double m_log(double v) { return log(v); }
__device__ inline float m_log(float v) { return logf(v); }

template <typename T>
__device__ inline T exact_u(const ProbDev& P, int s, T x, T y, T z) {
  if (P.solution == 1) return s == 0 ? m_exp(z) : m_cos(x) * m_sin(y);
  if (s == 0) return m_exp(x) * m_cos(y) * m_sin(z);
  return x * x + y * y + z * z;
}

// Problem constants in the working precision: the FP32 paths read the FP32
// copies (an FP64 operation is slow on this part and would sit on the
// critical path of the residual rows).
template <typename T>
__device__ __forceinline__ T pc_h(const ProbDev& P) {
  if constexpr (sizeof(T) == 4) return P.hf; else return P.h;
}
template <typename T>
__device__ __forceinline__ T pc_mu(const ProbDev& P, int s) {
  if constexpr (sizeof(T) == 4) return P.muf[s]; else return P.mu[s];
}
template <typename T>
__device__ __forceinline__ T pc_k(const ProbDev& P, int s) {
  if constexpr (sizeof(T) == 4) return P.kf[s]; else return P.k[s];
}

// diffusion coefficient mu^s(x)
template <typename T>
__device__ inline T mu_at(const ProbDev& P, int s, T x, T y, T z) {
  if (P.solution == 1) return s == 0 ? y * y * m_log(x + (T)2) + (T)4 : m_exp(-z);
  return pc_mu<T>(P, s);
}

// f^s = k^s u^s - div(mu^s grad u^s)
template <typename T>
__device__ inline T rhs_f(const ProbDev& P, int s, T x, T y, T z) {
  const T k = pc_k<T>(P, s);
  if (P.solution == 1) {
    if (s == 0) {
      // grad mu- = (y^2/(x+2), 2y ln(x+2), 0) is orthogonal to grad u- = (0, 0, e^z)
      const T u = m_exp(z);
      return k * u - mu_at<T>(P, 0, x, y, z) * u;
    }
    // grad mu+ = (0, 0, -e^-z) is orthogonal to grad u+ = (-sin x sin y, cos x cos y, 0)
    const T u = m_cos(x) * m_sin(y);
    return k * u + (T)2 * m_exp(-z) * u;
  }
  const T u = exact_u<T>(P, s, x, y, z);
  const T mu = pc_mu<T>(P, s);
  return s == 0 ? k * u + mu * u : k * u - (T)6 * mu;
}

template <typename T>
__device__ inline T dirichlet_g(const ProbDev& P, T x, T y, T z) {
  return exact_u<T>(P, P.geometry == NBM_GEOM_ALL_MINUS ? 0 : 1, x, y, z);
}

template <typename T>
__device__ inline void exact_grad_u(const ProbDev& P, int s, const T x[3], T g[3]) {
  if (P.solution == 1) {
    if (s == 0) {
      g[0] = g[1] = (T)0;
      g[2] = m_exp(x[2]);
    } else {
      g[0] = -m_sin(x[0]) * m_sin(x[1]);
      g[1] = m_cos(x[0]) * m_cos(x[1]);
      g[2] = (T)0;
    }
    return;
  }
  if (s == 0) {
    const T e = m_exp(x[0]);
    g[0] = e * m_cos(x[1]) * m_sin(x[2]);
    g[1] = -e * m_sin(x[1]) * m_sin(x[2]);
    g[2] = e * m_cos(x[1]) * m_cos(x[2]);
  } else {
    g[0] = (T)2 * x[0];
    g[1] = (T)2 * x[1];
    g[2] = (T)2 * x[2];
  }
}

__device__ inline double alpha_d(const ProbDev& P, const double x[3]) {
  return exact_u<double>(P, 1, x[0], x[1], x[2]) - exact_u<double>(P, 0, x[0], x[1], x[2]);
}

// FP32 versions of the level-set gradient, [u] and [mu d_n u] (the FP32 rows)
__device__ inline void grad_phi_f(const ProbDev& P, const float x[3], float g[3]) {
  grad_phi_t<float>(P, x, g);
}

__device__ inline float alpha_f(const ProbDev& P, const float x[3]) {
  return exact_u<float>(P, 1, x[0], x[1], x[2]) - exact_u<float>(P, 0, x[0], x[1], x[2]);
}

__device__ inline float beta_f(const ProbDev& P, const float x[3]) {
  float gm[3], gp[3], gf[3];
  exact_grad_u<float>(P, 0, x, gm);
  exact_grad_u<float>(P, 1, x, gp);
  grad_phi_f(P, x, gf);
  const float nn = sqrtf(gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2]);
  if (nn == 0.f) return 0.f;
  const float mp = mu_at<float>(P, 1, x[0], x[1], x[2]), mm = mu_at<float>(P, 0, x[0], x[1], x[2]);
  float b = 0.f;
  for (int i = 0; i < 3; ++i) b += (mp * gp[i] - mm * gm[i]) * gf[i] / nn;
  return b;
}

__device__ inline double beta_d(const ProbDev& P, const double x[3]) {
  double gp[3], gm[3], gf[3];
  exact_grad_u<double>(P, 1, x, gp);
  exact_grad_u<double>(P, 0, x, gm);
  grad_phi_d(P, x, gf);
  double nn = sqrt(gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2]);
  if (nn == 0.0) return 0.0;
  const double mp = mu_at<double>(P, 1, x[0], x[1], x[2]), mm = mu_at<double>(P, 0, x[0], x[1], x[2]);
  double b = 0.0;
  for (int i = 0; i < 3; ++i) b += (mp * gp[i] - mm * gm[i]) * gf[i] / nn;
  return b;
}

// ---------------------------------------------------------------------------
// tanh.  Accurate path: CUDA's tanhf.  Fast path: the SFU approximation
// (tanh.approx.f32), used only where the mixed-precision tolerance allows.
// ---------------------------------------------------------------------------
template <bool FAST>
__device__ __forceinline__ float act_tanh(float x) {
  if constexpr (FAST) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  } else {
    return tanhf(x);
  }
}
template <bool FAST>
__device__ __forceinline__ float rcp(float x) {
  if constexpr (FAST) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  } else {
    return 1.0f / x;
  }
}

// ---------------------------------------------------------------------------
// Difference-form tanh layer.  For one unit of one point the stencil values
// z(p), z(p +- h e_i) are carried as
//   z            centre pre-activation,
//   mu_i  = (z(p+h e_i) + z(p-h e_i))/2 - z(p)     (symmetric, O(h^2)),
//   del_i = (z(p+h e_i) - z(p-h e_i))/2            (antisymmetric, O(h)),
// scaled as mt = mu/h^2 and dt = del/h.  With t = tanh z the layer outputs
// the same three kinds of quantity for a = tanh(.), computed from tanh
// addition identities so that no O(1) values are subtracted:
//   tanh(z+mu) - tanh z          = Tm (1-t^2)/(1+t Tm),     Tm = tanh mu
//   [tanh(w+d) + tanh(w-d)]/2 - tanh w = -tw (1-tw^2) Td^2/(1-tw^2 Td^2)
//   [tanh(w+d) - tanh(w-d)]/2    = (1-tw^2) Td/(1-tw^2 Td^2),  Td = tanh d,
// with w = z + mu and tw = tanh w = (t+Tm)/(1+t Tm).
// Evaluating the network this way is exactly the same function as seven
// independent evaluations; it only changes the rounding.
// ---------------------------------------------------------------------------
//
// small_mu (every lane of the warp has |mu| below the path's threshold): the
// symmetric part from its Taylor series instead of the addition identity,
//   tanh(z+mu) - tanh z = (1-t^2) mu (1 - t mu + (t^2 - 1/3) mu^2) + R,
//   |R| <= (1-t^2) mu^4 / 2,
// i.e. a relative error below mu^3/2: 6.3e-5 at the SFU path's threshold
// kSmallMu (its outputs are rounded to 16 bits next), 3e-8 (below FP32
// rounding) at the accurate path's kSmallMuAccurate = 2^-8.  It saves the
// tanh of mu and a reciprocal per axis.
constexpr float kSmallMu = 0.05f;
constexpr float kSmallMuAccurate = 0.00390625f;

// small_de (accurate path only; every lane of the warp has |del| <= 2^-4): the
// antisymmetric part's tanh and reciprocal from their series,
//   tanh d = d (1 - d^2/3 + 2 d^4/15) + R,        |R| <= 17 |d|^7 / 315,
//   1 / (1 - x) = 1 + x + x^2 + x^3 + x^4/(1-x),  x = tw^2 Td^2 <= 2^-8,
// relative errors below 4e-9 and 2.4e-10 (FP32 rounding is 6e-8), in place of
// tanhf and an IEEE division.  The SFU path keeps tanh.approx and rcp.approx,
// which cost less than the series there.
constexpr float kSmallDelAccurate = 0.0625f;
__device__ __forceinline__ float tanh_small(float d) {
  const float d2 = d * d;
  return d * fmaf(d2, fmaf(d2, 2.0f / 15.0f, -1.0f / 3.0f), 1.0f);
}
__device__ __forceinline__ float rcp_one_minus_small(float x) {  // 1 / (1 - x), 0 <= x <= 2^-8
  return fmaf(x, fmaf(x, x + 1.0f, 1.0f), 1.0f);
}

template <bool FAST>
__device__ __forceinline__ void tanh_stencil_fwd(float t, float mt, float dt, float h, float h2,
                                                 float inv_h, float inv_h2, float& mo, float& dout,
                                                 bool small_mu = false, bool small_de = false) {
  float mu = mt * h2, de = dt * h;
  const bool sde = !FAST && small_de;
  float Td = sde ? tanh_small(de) : act_tanh<FAST>(de);
  float tw, dm;
  if (small_mu) {
    const float poly = fmaf(fmaf(t, t, -1.0f / 3.0f), mu * mu, fmaf(-t, mu, 1.0f));
    dm = fmaf(-t, t, 1.0f) * mu * poly;
    tw = t + dm;
  } else {
    float Tm = act_tanh<FAST>(mu);
    float q = rcp<FAST>(fmaf(t, Tm, 1.0f));
    tw = (t + Tm) * q;
    dm = Tm * fmaf(-t, t, 1.0f) * q;
  }
  float sw = fmaf(-tw, tw, 1.0f);
  float Td2 = Td * Td;
  float r2 = sde ? rcp_one_minus_small(tw * tw * Td2)
                 : rcp<FAST>(fmaf(sw - 1.0f, Td2, 1.0f));  // 1 / (1 - tw^2 Td^2)
  float k = sw * r2;
  float m = fmaf(-tw * Td2, k, dm);
  float d = k * Td;
  mo = m * inv_h2;
  dout = d * inv_h;
}

// The same for mu = 0 (the first layer, whose symmetric increments vanish):
// Tm = 0, tw = t, dm = 0.
template <bool FAST>
__device__ __forceinline__ void tanh_stencil_fwd0(float t, float dt, float h, float inv_h,
                                                  float inv_h2, float& mo, float& dout) {
  const float Td = act_tanh<FAST>(dt * h);
  const float sw = fmaf(-t, t, 1.0f);
  const float Td2 = Td * Td;
  const float r2 = rcp<FAST>(fmaf(-t * t, Td2, 1.0f));
  mo = (-t * sw * Td2 * r2) * inv_h2;
  dout = (sw * Td * r2) * inv_h;
}

// ---------------------------------------------------------------------------
// Difference-form sine layer (the sine-activated networks of Sec. 4.1).  Same
// column convention as the tanh layer (mt = mu/h^2, dt = del/h); with
// w = z + mu the outputs are
//   [sin(w+d) + sin(w-d)]/2 - sin z = [cos z sin mu - 2 sin z sin^2(mu/2)] cos d
//                                     - 2 sin z sin^2(d/2),
//   [sin(w+d) - sin(w-d)]/2         = cos w sin d,
// cos w = cos z (1 - 2 sin^2(mu/2)) - sin z sin mu: no O(1) values are
// subtracted.  sz, cz = sin z, cos z of the centre column.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sin_stencil_fwd(float sz, float cz, float mt, float dt, float h,
                                                float h2, float inv_h, float inv_h2, float& mo,
                                                float& dout) {
  float sh, ch, shd, chd;
  sincosf(0.5f * mt * h2, &sh, &ch);
  sincosf(0.5f * dt * h, &shd, &chd);
  const float sm = 2.f * sh * ch, sh2 = sh * sh;
  const float sd = 2.f * shd * chd, shd2 = shd * shd, cd = fmaf(-2.f, shd2, 1.f);
  const float dsw = fmaf(cz, sm, -2.f * sz * sh2);  // sin w - sin z
  const float cw = fmaf(cz, fmaf(-2.f, sh2, 1.f), -sz * sm);
  mo = fmaf(dsw, cd, -2.f * sz * shd2) * inv_h2;
  dout = cw * sd * inv_h;
}

// Adjoint of one axis of the sine layer: inputs z (via sz, cz), mt, dt and the
// upstream gradients with respect to the scaled outputs (Gm_s, Gd_s).  Writes
// the gradients with respect to the scaled inputs and returns the contribution
// to d/dz.  With M = sin w cos d - sin z and D = cos w sin d:
//   dM/dz = (cos w - cos z) cos d - cos z (1 - cos d), dM/dmu = cos w cos d,
//   dM/dd = dD/dz = dD/dmu = -sin w sin d, dD/dd = cos w cos d,
// cos w - cos z = -2 cos z sin^2(mu/2) - sin z sin mu.
__device__ __forceinline__ float sin_stencil_bwd(float sz, float cz, float mt, float dt,
                                                 float Gm_s, float Gd_s, float h, float h2,
                                                 float inv_h, float inv_h2, float& gmu_s,
                                                 float& gdel_s) {
  float sh, ch, shd, chd;
  sincosf(0.5f * mt * h2, &sh, &ch);
  sincosf(0.5f * dt * h, &shd, &chd);
  const float sm = 2.f * sh * ch, sh2 = sh * sh;
  const float sd = 2.f * shd * chd, shd2 = shd * shd, cd = fmaf(-2.f, shd2, 1.f);
  const float cmu = fmaf(-2.f, sh2, 1.f);
  const float cw = fmaf(cz, cmu, -sz * sm), sw = fmaf(sz, cmu, cz * sm);
  const float Gm = Gm_s * inv_h2, Gd = Gd_s * inv_h;
  const float dMdz = fmaf(fmaf(-2.f * cz, sh2, -sz * sm), cd, -2.f * cz * shd2);
  const float cc = cw * cd, ss = -sw * sd;
  gmu_s = fmaf(Gm, cc, Gd * ss) * h2;
  gdel_s = fmaf(Gm, ss, Gd * cc) * h;
  return fmaf(Gm, dMdz, Gd * ss);
}

// Adjoint of one stencil axis.  Inputs: forward outputs t (centre), mo, dout
// (scaled), upstream gradients with respect to the scaled outputs (Gm, Gd).
// Writes the gradients with respect to the scaled inputs (gmu, gdel) and
// returns the contribution to d/dz.  With s0 = 1-t^2, m = mo h^2, d = dout h:
//   P = -(2 t m + m^2 + d^2)  = (s+ + s- - 2 s0)/2,
//   Q = -2 d (t + m)          = (s+ - s-)/2,      s+- = 1 - tanh^2(z+mu+-del),
//   dm/dz = P, dm/dmu = s0+P, dm/ddel = Q, dd/dz = dd/dmu = Q, dd/ddel = s0+P.
__device__ __forceinline__ float tanh_stencil_bwd(float t, float s0, float mo, float dout,
                                                  float Gm_s, float Gd_s, float h, float h2,
                                                  float inv_h, float inv_h2, float& gmu_s,
                                                  float& gdel_s) {
  float m = mo * h2, d = dout * h;
  float Gm = Gm_s * inv_h2, Gd = Gd_s * inv_h;
  float P = -fmaf(2.f * t, m, fmaf(m, m, d * d));
  float Q = -2.f * d * (t + m);
  float S = s0 + P;
  gmu_s = fmaf(S, Gm, Q * Gd) * h2;
  gdel_s = fmaf(Q, Gm, S * Gd) * h;
  return fmaf(P, Gm, Q * Gd);
}

// ---------------------------------------------------------------------------
// Balance row of an uncut cell of phase s (Sec. 3 reading):
//   B/h^2 = k U(p) - f(p) - mu sum_{i,sigma} dU_{sigma i}/h^2,
//   dU_{+-i}/h^2 = Mt_i +- Dt_i/h   (interior neighbour)
//               = (g(q) - U(p))/h^2  (neighbour outside the cube: Dirichlet),
//   D = 6 mu + h^2 k,  r = B/D.
// out[8] = network outputs (U, Mt1..3, Dt1..3, unused); seeds[8] receives
// d(scale * r^2)/d(out).  Returns r^2.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline T uncut_residual(const ProbDev& P, int s, float px, float py, float pz,
                                   const float out[8], T scale, float seeds[8]) {
  const T h = pc_h<T>(P), h2 = h * h, mu = pc_mu<T>(P, s), k = pc_k<T>(P, s);
  const T U = (T)out[0];
  const T x[3] = {(T)px, (T)py, (T)pz};
  T Bt = k * U - rhs_f<T>(P, s, x[0], x[1], x[2]);
  T dU = k;
  T dM[3], dD[3];
  T D = h2 * k;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dM[i] = 0;
    dD[i] = 0;
#pragma unroll
    for (int sg = -1; sg <= 1; sg += 2) {
      T q[3] = {x[0], x[1], x[2]};
      q[i] += sg * h;
      // mu at the face centre (variable coefficients of Sec. 4.1)
      T mf = mu;
      if (P.solution == 1) {
        T c[3] = {x[0], x[1], x[2]};
        c[i] += (T)0.5 * (T)sg * h;
        mf = mu_at<T>(P, s, c[0], c[1], c[2]);
        D += mf;
      }
      bool bnd = fabs(q[i]) >= (T)1;
      if (bnd) {
        T g = dirichlet_g<T>(P, q[0], q[1], q[2]);
        Bt -= mf * (g - U) / h2;
        dU += mf / h2;
      } else {
        Bt -= mf * ((T)out[1 + i] + (T)sg * (T)out[4 + i] / h);
        dM[i] -= mf;
        dD[i] -= mf * (T)sg / h;
      }
    }
  }
  if (P.solution != 1) D = (T)6 * mu + h2 * k;
  T r = h2 * Bt / D;
  T c = scale * (T)2 * r * h2 / D;
  seeds[0] = (float)(c * dU);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    seeds[1 + i] = (float)(c * dM[i]);
    seeds[4 + i] = (float)(c * dD[i]);
  }
  seeds[7] = 0.f;
  return r * r;
}

// The same rows for one point in one thread of the tensor-core path.  fsrc =
// f^s(p), evaluated ahead (the tile records carry it); divisions by h, h^2
// and D are multiplications by the reciprocals in P.  out[8] = network
// outputs in the scaled convention (U, Mt1..3, Dt1..3, unused); sd[8]
// receives d(scale * r^2)/d(out).  Returns r^2.
template <typename T>
__device__ __forceinline__ T uncut_residual_pt(const ProbDev& P, int s, float px, float py,
                                               float pz, T fsrc, const float out[8], T scale,
                                               float sd[8]) {
  const T h = pc_h<T>(P), h2 = h * h, mu = pc_mu<T>(P, s), kk = pc_k<T>(P, s);
  T ih, ih2, iD;
  if constexpr (sizeof(T) == 4) {
    ih = P.inv_hf;
    ih2 = P.inv_h2f;
    iD = P.inv_Df[s];
  } else {
    ih = P.inv_h;
    ih2 = P.inv_h2;
    iD = P.inv_D[s];
  }
  const T U = (T)out[0];
  const T x[3] = {(T)px, (T)py, (T)pz};
  T Bt = kk * U - fsrc;
  T nbmu = 0;  // sum of mu over the Dirichlet faces
  T cM[3], cD[3];
  T Dv = h2 * kk;  // Jacobi diagonal accumulated over faces (variable mu only)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T Mt = (T)out[1 + i], Dt = (T)out[4 + i];
    T qm[3] = {x[0], x[1], x[2]}, qp[3] = {x[0], x[1], x[2]};
    qm[i] -= h;
    qp[i] += h;
    // mu at the two face centres (variable coefficients of Sec. 4.1)
    T mm = mu, mp = mu;
    if (P.solution == 1) {
      T cm[3] = {x[0], x[1], x[2]}, cp[3] = {x[0], x[1], x[2]};
      cm[i] -= (T)0.5 * h;
      cp[i] += (T)0.5 * h;
      mm = mu_at<T>(P, s, cm[0], cm[1], cm[2]);
      mp = mu_at<T>(P, s, cp[0], cp[1], cp[2]);
      Dv += mm + mp;
    }
    const bool bm = fabs(qm[i]) >= (T)1, bp = fabs(qp[i]) >= (T)1;
    if (bm) {
      Bt -= mm * (dirichlet_g<T>(P, qm[0], qm[1], qm[2]) - U) * ih2;
      nbmu += mm;
    } else {
      Bt -= mm * (Mt - Dt * ih);
    }
    if (bp) {
      Bt -= mp * (dirichlet_g<T>(P, qp[0], qp[1], qp[2]) - U) * ih2;
      nbmu += mp;
    } else {
      Bt -= mp * (Mt + Dt * ih);
    }
    cM[i] = -((bm ? (T)0 : mm) + (bp ? (T)0 : mp));
    cD[i] = -((bp ? (T)0 : mp) - (bm ? (T)0 : mm)) * ih;
  }
  if (P.solution == 1) iD = (T)1 / Dv;
  const T r = h2 * Bt * iD;
  const T c = scale * (T)2 * r * h2 * iD;
  sd[0] = (float)(c * (kk + nbmu * ih2));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sd[1 + i] = (float)(c * cM[i]);
    sd[4 + i] = (float)(c * cD[i]);
  }
  sd[7] = 0.f;
  return r * r;
}

// The row of uncut_residual_pt spread over the 8 lanes c = 0..7 of an aligned
// group of a warp (all 8 call it for the same point; `mask` covers the
// calling lanes).  Lane c < 6 takes face c (axis c/2, side c%2), lane 6 the
// reaction and source term; the balance row and the Dirichlet and face sums
// are added over the group by shuffles.  Every lane passes the point's U and
// the Mt, Dt columns of its face's axis (any value on lanes 6 and 7), returns
// r^2 and writes seed c.  The same terms as the one-thread row, added in a
// different order, with the dependency chain of one face per lane: a short
// chain for the FP32 rows, and for the FP64 rows each instruction of the
// narrow FP64 pipe carries 8 lanes instead of 1.
template <typename T>
__device__ __forceinline__ T uncut_residual_lanes(const ProbDev& P, int s, float px, float py,
                                                  float pz, T fsrc, float U_c, float Mt_c,
                                                  float Dt_c, T scale, int c, unsigned mask,
                                                  float& sd_c) {
  const T h = pc_h<T>(P), h2 = h * h, mu = pc_mu<T>(P, s), kk = pc_k<T>(P, s);
  T ih, ih2, iD;
  if constexpr (sizeof(T) == 4) {
    ih = P.inv_hf;
    ih2 = P.inv_h2f;
    iD = P.inv_Df[s];
  } else {
    ih = P.inv_h;
    ih2 = P.inv_h2;
    iD = P.inv_D[s];
  }
  const T U = (T)U_c;
  const T x[3] = {(T)px, (T)py, (T)pz};
  T term = (T)0, nb = (T)0, cm = (T)0, dv = (T)0;
  if (c < 6) {
    // (selects, not indexing: the coordinates stay in registers)
    const int i = c >> 1;
    const bool plus = c & 1;
    const T Mt = (T)Mt_c, Dt = (T)Dt_c;
    const T dq = plus ? h : -h;
    const T q0 = i == 0 ? x[0] + dq : x[0], q1 = i == 1 ? x[1] + dq : x[1],
            q2 = i == 2 ? x[2] + dq : x[2];
    T mf = mu;
    if (P.solution == 1) {
      const T dc = plus ? (T)0.5 * h : -(T)0.5 * h;
      mf = mu_at<T>(P, s, i == 0 ? x[0] + dc : x[0], i == 1 ? x[1] + dc : x[1],
                    i == 2 ? x[2] + dc : x[2]);
      dv = mf;
    }
    if (fabs(i == 0 ? q0 : i == 1 ? q1 : q2) >= (T)1) {
      term = -mf * (dirichlet_g<T>(P, q0, q1, q2) - U) * ih2;
      nb = mf;
    } else {
      term = -mf * (plus ? Mt + Dt * ih : Mt - Dt * ih);
      cm = mf;
    }
  } else if (c == 6) {
    term = kk * U - fsrc;
  }
  T Bt = term, nbmu = nb, Dv = dv;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    Bt += __shfl_xor_sync(mask, Bt, o, 8);
    nbmu += __shfl_xor_sync(mask, nbmu, o, 8);
    Dv += __shfl_xor_sync(mask, Dv, o, 8);
  }
  // the two faces of the axis of seed c (c = 1..3: symmetric, 4..6: antisymmetric)
  const int ax = c >= 4 ? c - 4 : c - 1;
  const int fa = ax < 0 || ax > 2 ? 0 : 2 * ax;
  const T cmm = __shfl_sync(mask, cm, fa, 8), cmp = __shfl_sync(mask, cm, fa + 1, 8);
  if (P.solution == 1) iD = (T)1 / (Dv + h2 * kk);
  const T r = h2 * Bt * iD;
  const T cf = scale * (T)2 * r * h2 * iD;
  T sd = (T)0;
  if (c == 0) sd = cf * (kk + nbmu * ih2);
  else if (c <= 3) sd = cf * -(cmm + cmp);
  else if (c <= 6) sd = cf * (-(cmp - cmm) * ih);
  sd_c = (float)sd;
  return r * r;
}

}  // namespace nbm
