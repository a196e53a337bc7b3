// Device math shared by the CUDA translation units of this library: scalar
// helpers per precision, the pinhole projection with R = Rz(gamma) Ry(beta)
// Rx(alpha) (Sec. 2.1, Eq. 1), the misfit losses, and the local solve of
// Eq. (9).  Included inside namespace dba { namespace { ... } } by each unit.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include <type_traits>

#include "dba_internal.h"

namespace dba {
namespace {

// ------------------------------------------------------------ scalar helpers
template <typename T> struct Num;
// FP32 path: single SFU instructions (PTX rcp/sqrt/rsqrt .approx, relative error of
// about one ulp; sin/cos with 2^-21 absolute error after reduction to [-pi, pi]).  Their
// error stays far below the pixel tolerance and inside the model_tol noise rule.
template <> struct Num<float> {
  using V2 = float2;
  static __device__ __forceinline__ void sc(float x, float* s, float* c) {
    // Cody-Waite reduction by 2 pi (two-term split of 2 pi), then the SFU sin/cos
    const float k = rintf(x * 0.15915494309189535f);
    float r = fmaf(-k, 6.28318548202514648f, x);
    r = fmaf(-k, -1.7484555314695172e-7f, r);
    __sincosf(r, s, c);
  }
  static __device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  static __device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  // p / sqrt(s) for s > 0
  static __device__ __forceinline__ float div_sqrt(float p, float s) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
    return p * r;
  }
  static __device__ __forceinline__ float tenth(float x) { return x * 0.1f; }
  static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
  static __device__ __forceinline__ float inf() { return CUDART_INF_F; }
  static constexpr float unit_roundoff = 5.9604644775390625e-08f;  // 2^-24
};
// FP64 path: correctly rounded operations, as the oracle uses.
template <> struct Num<double> {
  using V2 = double2;
  static __device__ __forceinline__ void sc(double x, double* s, double* c) { sincos(x, s, c); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double div_sqrt(double p, double s) { return p / sqrt(s); }
  static __device__ __forceinline__ double tenth(double x) { return x / 10.0; }
  static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
  static __device__ __forceinline__ double inf() { return CUDART_INF; }
  static constexpr double unit_roundoff = 1.1102230246251565e-16;  // 2^-53
};

// float <-> double by integer bit manipulation (IEEE-754 binary32/binary64 layouts), so the
// FP32 path spends none of GB300's scarce FP64 issue slots on conversions.  Exact for normal
// numbers; magnitudes below 2^-126 become signed zero; infinities stay infinite, NaNs stay
// NaN and float overflow becomes infinity.  The special cases are selected, not branched
// to, so the conversions compile to straight-line integer code.
__device__ __forceinline__ double widen(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int sign = b & 0x80000000u, mag = b & 0x7fffffffu;
  const bool special = mag >= 0x7f800000u, tiny = mag < 0x00800000u;
  unsigned int hi = sign | ((mag >> 3) + (896u << 20));
  hi = special ? (sign | 0x7ff00000u | ((mag >> 3) & 0xfffffu)) : hi;
  hi = tiny ? sign : hi;
  const unsigned int lo = tiny ? 0u : (mag << 29);
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float narrow(double d) {
  const unsigned int hi = (unsigned int)__double2hiint(d);
  const unsigned int lo = (unsigned int)__double2loint(d);
  const unsigned int sign = hi & 0x80000000u;
  const unsigned int e = (hi >> 20) & 0x7ffu;
  unsigned int f = ((e - 896u) << 23) + (((hi & 0xfffffu) << 3) | (lo >> 29));
  f += (lo >> 28) & 1u;  // round to nearest (halfway cases away from zero)
  const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
  f = e >= 1151u ? (nan ? 0x7fc00000u : 0x7f800000u) : f;
  f = e <= 896u ? 0u : f;
  return __uint_as_float(f | sign);
}
template <typename T> __device__ __forceinline__ double to_f64(T v);
template <> __device__ __forceinline__ double to_f64<float>(float v) { return widen(v); }
template <> __device__ __forceinline__ double to_f64<double>(double v) { return v; }
template <typename T> __device__ __forceinline__ T from_f64(double v);
template <> __device__ __forceinline__ float from_f64<float>(double v) { return narrow(v); }
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }

template <typename T>
struct Prm {
  T focal, cx, cy, lp, rho_x, rho_y, rho_a, lambda0, lambda_min, eps, model_tol;
  int loss, steps, solver;
  // penalty of coordinate c of (x, alpha, beta, gamma, t)
  __device__ __forceinline__ T rho(int c) const { return c < 3 ? rho_x : (c < 6 ? rho_a : rho_y); }
};

template <typename T>
__host__ __device__ Prm<T> make_prm(const Params& p) {
  Prm<T> q;
  q.focal = (T)p.focal; q.cx = (T)p.cx; q.cy = (T)p.cy; q.lp = (T)p.loss_param;
  q.rho_x = (T)p.rho_x; q.rho_y = (T)p.rho_y; q.rho_a = (T)p.rho_a; q.lambda0 = (T)p.lambda0;
  q.lambda_min = (T)p.lambda_min; q.eps = (T)p.eps_depth; q.model_tol = (T)p.model_tol;
  q.loss = p.loss; q.steps = p.inner_steps; q.solver = p.solver;
  return q;
}

// Misfit phi_m as a function of s = |e|^2 and its derivative (IRLS weight).
template <typename T>
__device__ __forceinline__ T misfit(int loss, T p, T s) {
  if (loss == 1) return s <= p * p ? s : T(2) * p * Num<T>::sqrt_(s) - p * p;
  if (loss == 2) return p * Num<T>::log1p_(Num<T>::div(s, p));
  return s;
}
template <typename T>
__device__ __forceinline__ T misfit_weight(int loss, T p, T s) {
  if (loss == 1) return s <= p * p ? T(1) : Num<T>::div_sqrt(p, s);
  if (loss == 2) return Num<T>::div(p, p + s);
  return T(1);
}

// Camera pose evaluated at v = (x, alpha, beta, gamma, t): R = Rz Ry Rx
// (Sec. 2.1), u = R x and p = u + t (camera frame).
template <typename T>
struct Pose {
  T R[9];
  T u[3];
  T p[3];
  T sg, cg;
  bool valid;
};

template <typename T>
__device__ __forceinline__ void pose_at(const T v[9], T eps, Pose<T>& P) {
  T sa, ca, sb, cb;
  Num<T>::sc(v[3], &sa, &ca);
  Num<T>::sc(v[4], &sb, &cb);
  Num<T>::sc(v[5], &P.sg, &P.cg);
  const T sg = P.sg, cg = P.cg;
  P.R[0] = cg * cb;
  P.R[1] = cg * sb * sa - sg * ca;
  P.R[2] = cg * sb * ca + sg * sa;
  P.R[3] = sg * cb;
  P.R[4] = sg * sb * sa + cg * ca;
  P.R[5] = sg * sb * ca - cg * sa;
  P.R[6] = -sb;
  P.R[7] = cb * sa;
  P.R[8] = cb * ca;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    P.u[r] = P.R[3 * r] * v[0] + P.R[3 * r + 1] * v[1] + P.R[3 * r + 2] * v[2];
    P.p[r] = P.u[r] + v[6 + r];
  }
  P.valid = P.p[2] > eps;
}

// Eq. (9) in offset form: with d = v - vbar and a = dual / rho,
// r^T d + rho/2 |d|^2 = rho (a.d + d.d/2).  +inf behind the camera.
template <typename T>
__device__ __forceinline__ T local_objective(const T d[9], const T a[9], const Pose<T>& P,
                                             T z0, T z1, const Prm<T>& q) {
  if (!P.valid) return Num<T>::inf();
  const T iz = Num<T>::rcp(P.p[2]);
  const T e0 = z0 - (q.focal * P.p[0] * iz + q.cx);
  const T e1 = z1 - (q.focal * P.p[1] * iz + q.cy);
  T px = 0, pa = 0, pt = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) px += d[c] * (a[c] + T(0.5) * d[c]);
#pragma unroll
  for (int c = 3; c < 6; ++c) pa += d[c] * (a[c] + T(0.5) * d[c]);
#pragma unroll
  for (int c = 6; c < 9; ++c) pt += d[c] * (a[c] + T(0.5) * d[c]);
  return misfit<T>(q.loss, q.lp, e0 * e0 + e1 * e1) + q.rho_x * px + q.rho_a * pa + q.rho_y * pt;
}

// Eq. (9): inner_steps damped Gauss-Newton steps with IRLS weights.  The
// damped normal matrix 2w J^T J + diag(rho) + lambda I is diagonal plus rank
// 2 (one observation has two residuals), so each step solves it exactly
// through its 2x2 capacitance matrix (Sherman-Morrison-Woodbury) instead of a
// 9x9 factorisation.  Accept/reject and the damping schedule follow the
// Levenberg rule: accept iff the trial is in front of the camera and lowers
// Eq. (9).  A step whose predicted decrease is below the objective's rounding
// noise is accepted without the comparison (model_tol).  d (offset from vbar)
// is updated in place.
// Linearisation of the pixel model at pose P: residual e = z - f(v), IRLS
// weight w = phi'(|e|^2), and the 2x9 Jacobian rows J0, J1 (d p/d v columns:
// x_k -> R[:,k]; alpha -> R[:,0] x u; beta -> (-sin g, cos g, 0) x u;
// gamma -> e_z x u; t_k -> e_k; row r of J = f/p_3 (dp_r - z_r dp_3)).
template <typename T>
__device__ __forceinline__ void linearize(const Pose<T>& P, T z0, T z1, const Prm<T>& q, T J0[9], T J1[9], T& e0,
                                          T& e1, T& w) {
  const T iz = Num<T>::rcp(P.p[2]);
  const T zx = P.p[0] * iz, zy = P.p[1] * iz;
  e0 = z0 - (q.focal * zx + q.cx);
  e1 = z1 - (q.focal * zy + q.cy);
  w = misfit_weight<T>(q.loss, q.lp, e0 * e0 + e1 * e1);
  const T fi = q.focal * iz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    J0[k] = fi * (P.R[k] - zx * P.R[6 + k]);
    J1[k] = fi * (P.R[3 + k] - zy * P.R[6 + k]);
  }
  {
    const T c0 = P.R[0], c1 = P.R[3], c2 = P.R[6];
    const T d0 = c1 * P.u[2] - c2 * P.u[1];
    const T d1 = c2 * P.u[0] - c0 * P.u[2];
    const T d2 = c0 * P.u[1] - c1 * P.u[0];
    J0[3] = fi * (d0 - zx * d2);
    J1[3] = fi * (d1 - zy * d2);
  }
  {
    const T b0 = -P.sg, b1 = P.cg;
    const T d0 = b1 * P.u[2];
    const T d1 = -b0 * P.u[2];
    const T d2 = b0 * P.u[1] - b1 * P.u[0];
    J0[4] = fi * (d0 - zx * d2);
    J1[4] = fi * (d1 - zy * d2);
  }
  J0[5] = fi * (-P.u[1]);
  J1[5] = fi * (P.u[0]);
  J0[6] = fi;
  J1[6] = 0;
  J0[7] = 0;
  J1[7] = fi;
  J0[8] = -fi * zx;
  J1[8] = -fi * zy;
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// One Gauss-Newton step's linear algebra in FP32 on pairs of adjacent components
// (packed FP32x2 multiply/add/FMA of the sm_100 family; component 8 alone): gradient
// g = -2w J^T e + rho (a + d), the first damping from the trace of H, the step
// s = -D^-1 g + 2w D^-1 J^T y with D = diag(rho) + lambda I and the 2x2 capacitance
// solve for y, and the model decrease (lambda |s|^2 - g.s) / 2.  Same formulas as the
// scalar path, summed in two lanes.
__device__ __forceinline__ void gn_step_f32(const float J0[9], const float J1[9], float e0, float e1, float tw,
                                            const float a[9], const float d[9], const Prm<float>& q,
                                            float& lambda, float stp[9], float& pred, float& gs_out) {
  const float2 rp[4] = {f2(q.rho_x, q.rho_x), f2(q.rho_x, q.rho_a), f2(q.rho_a, q.rho_a), f2(q.rho_y, q.rho_y)};
  const float2 ntw = f2(-tw, -tw), E0 = f2(e0, e0), E1 = f2(e1, e1);
  float2 g2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 j0 = f2(J0[2 * k], J0[2 * k + 1]), j1 = f2(J1[2 * k], J1[2 * k + 1]);
    const float2 m = __ffma2_rn(j1, E1, __fmul2_rn(j0, E0));
    g2[k] = __ffma2_rn(rp[k], __fadd2_rn(f2(a[2 * k], a[2 * k + 1]), f2(d[2 * k], d[2 * k + 1])), __fmul2_rn(ntw, m));
  }
  const float g8 = -tw * (J0[8] * e0 + J1[8] * e1) + q.rho_y * (a[8] + d[8]);
  if (lambda < 0.f) {
    float2 tr2 = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 j0 = f2(J0[2 * k], J0[2 * k + 1]), j1 = f2(J1[2 * k], J1[2 * k + 1]);
      tr2 = __ffma2_rn(j1, j1, __ffma2_rn(j0, j0, tr2));
    }
    const float tr = 3.f * (q.rho_x + q.rho_a + q.rho_y) + tw * (tr2.x + tr2.y + J0[8] * J0[8] + J1[8] * J1[8]);
    lambda = q.lambda0 * tr / 9.f;
  }
  const float iDx = Num<float>::rcp(q.rho_x + lambda), iDa = Num<float>::rcp(q.rho_a + lambda),
              iDy = Num<float>::rcp(q.rho_y + lambda);
  const float2 niD[4] = {f2(-iDx, -iDx), f2(-iDx, -iDa), f2(-iDa, -iDa), f2(-iDy, -iDy)};
  // nq = -D^-1 g; G = J D^-1 J^T; T = J nq = -J D^-1 g
  float2 nq[4], G00 = f2(0.f, 0.f), G01 = f2(0.f, 0.f), G11 = f2(0.f, 0.f), T0 = f2(0.f, 0.f), T1 = f2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 j0 = f2(J0[2 * k], J0[2 * k + 1]), j1 = f2(J1[2 * k], J1[2 * k + 1]);
    nq[k] = __fmul2_rn(g2[k], niD[k]);
    const float2 a0 = __fmul2_rn(j0, niD[k]), a1 = __fmul2_rn(j1, niD[k]);  // -J D^-1
    G00 = __ffma2_rn(a0, j0, G00);
    G01 = __ffma2_rn(a0, j1, G01);
    G11 = __ffma2_rn(a1, j1, G11);
    T0 = __ffma2_rn(j0, nq[k], T0);
    T1 = __ffma2_rn(j1, nq[k], T1);
  }
  const float nq8 = -g8 * iDy;
  const float g00 = -(G00.x + G00.y) + J0[8] * J0[8] * iDy, g01 = -(G01.x + G01.y) + J0[8] * J1[8] * iDy,
              g11 = -(G11.x + G11.y) + J1[8] * J1[8] * iDy;
  const float t0 = -(T0.x + T0.y + J0[8] * nq8), t1 = -(T1.x + T1.y + J1[8] * nq8);
  const float S00 = 1.f + tw * g00, S01 = tw * g01, S11 = 1.f + tw * g11;
  const float idet = Num<float>::rcp(S00 * S11 - S01 * S01);
  const float y0 = (S11 * t0 - S01 * t1) * idet;
  const float y1 = (S00 * t1 - S01 * t0) * idet;
  const float2 Y0 = f2(y0, y0), Y1 = f2(y1, y1);
  float2 GS = f2(0.f, 0.f), SS = f2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 j0 = f2(J0[2 * k], J0[2 * k + 1]), j1 = f2(J1[2 * k], J1[2 * k + 1]);
    const float2 u = __ffma2_rn(j1, Y1, __fmul2_rn(j0, Y0));
    const float2 ntwiD = __fmul2_rn(ntw, niD[k]);  // 2w D^-1
    const float2 s2 = __ffma2_rn(ntwiD, u, nq[k]);
    GS = __ffma2_rn(g2[k], s2, GS);
    SS = __ffma2_rn(s2, s2, SS);
    stp[2 * k] = s2.x;
    stp[2 * k + 1] = s2.y;
  }
  stp[8] = nq8 + tw * iDy * (J0[8] * y0 + J1[8] * y1);
  const float gs = GS.x + GS.y + g8 * stp[8], ss = SS.x + SS.y + stp[8] * stp[8];
  pred = 0.5f * (lambda * ss - gs);
  gs_out = gs;
}

// Eq. (9): inner_steps damped Gauss-Newton steps with IRLS weights.  The
// damped normal matrix 2w J^T J + diag(rho) + lambda I is diagonal plus rank
// 2 (one observation has two residuals), so each step solves it exactly
// through its 2x2 capacitance matrix (Sherman-Morrison-Woodbury) instead of a
// 9x9 factorisation.  Accept/reject and the damping schedule follow the
// Levenberg rule: accept iff the trial is in front of the camera and lowers
// Eq. (9).  A step whose predicted decrease is below the objective's rounding
// noise is accepted without the comparison (model_tol); an accepted step keeps
// Eq. (9) evaluated at its new point.  d (offset from vbar) is updated in place.
// With kAlt, `alt` is a second candidate start (a learned warm start): the
// solve starts from whichever of d and alt has the lower Eq. (9).
template <typename T, bool kAlt = false>
__device__ __forceinline__ void local_solve(T z0, T z1, const T vbar[9], const T a[9], T d[9],
                                            const Prm<T>& q, const T* alt = nullptr) {
  T v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = vbar[c] + d[c];
  Pose<T> P;
  pose_at(v, q.eps, P);
  T L = local_objective(d, a, P, z0, z1, q);
  if constexpr (kAlt) {
    T da[9], va[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      da[c] = alt[c];
      va[c] = vbar[c] + da[c];
    }
    Pose<T> Pa;
    pose_at(va, q.eps, Pa);
    const T La = local_objective(da, a, Pa, z0, z1, q);
    if (La < L) {  // the plain start stays unless the candidate lowers Eq. (9) (the fallback)
#pragma unroll
      for (int c = 0; c < 9; ++c) d[c] = da[c];
      P = Pa;
      L = La;
    }
  }
  T lambda = T(-1);
  for (int step = 0; step < q.steps; ++step) {
    T J0[9], J1[9];
    T w = 0, e0 = 0, e1 = 0;
    if (P.valid) {
      linearize(P, z0, z1, q, J0, J1, e0, e1, w);
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) J0[k] = J1[k] = 0;
    }
    const T tw = T(2) * w;
    T stp[9], pred, gs;
    if constexpr (std::is_same<T, float>::value) {
      gn_step_f32(J0, J1, e0, e1, tw, a, d, q, lambda, stp, pred, gs);
    } else {
      T g[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = -tw * (J0[c] * e0 + J1[c] * e1) + q.rho(c) * (a[c] + d[c]);
      if (lambda < T(0)) {
        T tr = T(3) * (q.rho_x + q.rho_a + q.rho_y);
#pragma unroll
        for (int c = 0; c < 9; ++c) tr += tw * (J0[c] * J0[c] + J1[c] * J1[c]);
        lambda = q.lambda0 * tr / T(9);
      }
      const T iDx = Num<T>::rcp(q.rho_x + lambda), iDa = Num<T>::rcp(q.rho_a + lambda),
              iDy = Num<T>::rcp(q.rho_y + lambda);
      T G00 = 0, G01 = 0, G11 = 0, t0 = 0, t1 = 0;
      T qv[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const T iD = c < 3 ? iDx : (c < 6 ? iDa : iDy);
        qv[c] = g[c] * iD;
        G00 += J0[c] * J0[c] * iD;
        G01 += J0[c] * J1[c] * iD;
        G11 += J1[c] * J1[c] * iD;
        t0 += J0[c] * qv[c];
        t1 += J1[c] * qv[c];
      }
      const T S00 = T(1) + tw * G00, S01 = tw * G01, S11 = T(1) + tw * G11;
      const T idet = Num<T>::rcp(S00 * S11 - S01 * S01);
      const T y0 = (S11 * t0 - S01 * t1) * idet;
      const T y1 = (S00 * t1 - S01 * t0) * idet;
      T ss = 0;
      gs = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const T iD = c < 3 ? iDx : (c < 6 ? iDa : iDy);
        stp[c] = -qv[c] + tw * iD * (J0[c] * y0 + J1[c] * y1);
        gs += g[c] * stp[c];
        ss += stp[c] * stp[c];
      }
      // decrease of the Gauss-Newton model; with (H + lambda I) s = -g it is (lambda s.s - g.s) / 2
      pred = T(0.5) * (lambda * ss - gs);
    }
    bool trust = false;
    if (P.valid && q.model_tol > T(0)) {
      // below the rounding noise of L the objective comparison is arbitrary: trust the model
      const T noise = q.model_tol * Num<T>::unit_roundoff *
                      (fabs(L) + T(2) * w * Num<T>::sqrt_(e0 * e0 + e1 * e1) * (fabs(z0) + fabs(z1)));
      trust = pred <= noise;
    }
    T dt[9], vt[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      dt[c] = d[c] + stp[c];
      vt[c] = vbar[c] + dt[c];
    }
    // the trial pose replaces the current one; a rejected step recomputes the kept copy's
    // pose (the same arithmetic on the same input, so bit-identical to the pose it had)
    pose_at(vt, q.eps, P);
    // Eq. (9) at the trial point: compared with L, and kept as L once the step is accepted.
    // Only a trusted last step needs neither (L is not read after the last step), so a warp
    // whose lanes all trust their last step skips it.
    T Lt = L;
    if (__any_sync(__activemask(), !trust || step + 1 < q.steps)) Lt = local_objective(dt, a, P, z0, z1, q);
    const bool accept = P.valid && (trust || Lt < L);
    if (accept) {
#pragma unroll
      for (int c = 0; c < 9; ++c) d[c] = dt[c];
      L = Lt;
      const T lr = Num<T>::tenth(lambda);
      lambda = lr > q.lambda_min ? lr : q.lambda_min;
    } else {
      lambda *= T(10);
    }
    if (__any_sync(__activemask(), !accept) && !accept) {
#pragma unroll
      for (int c = 0; c < 9; ++c) v[c] = vbar[c] + d[c];
      pose_at(v, q.eps, P);
    }
  }
}

// Gradient of Eq. (9) in offset form at pose P (v = vbar + d): -2 w J^T e + rho (a + d), no
// misfit term behind the camera; noise = 2 w |e| (|z1| + |z2|), the objective's rounding scale.
template <typename T>
__device__ __forceinline__ void local_gradient(const Pose<T>& P, T z0, T z1, const T a[9], const T d[9],
                                               const Prm<T>& q, T g[9], T& noise) {
  T J0[9], J1[9], e0 = 0, e1 = 0, w = 0;
  if (P.valid) {
    linearize(P, z0, z1, q, J0, J1, e0, e1, w);
  } else {
#pragma unroll
    for (int c = 0; c < 9; ++c) J0[c] = J1[c] = 0;
  }
  const T tw = T(2) * w;
#pragma unroll
  for (int c = 0; c < 9; ++c) g[c] = -tw * (J0[c] * e0 + J1[c] * e1) + q.rho(c) * (a[c] + d[c]);
  noise = tw * Num<T>::sqrt_(e0 * e0 + e1 * e1) * (fabs(z0) + fabs(z1));
}

constexpr int kLbfgsMemory = 4;
constexpr int kLbfgsHalvings = 10;

// Eq. (9) by L-BFGS (Sec. 3.1 names it for the Huber loss; Nocedal and Wright, Ch. 7):
// inner_steps iterations in the coordinates u = r d, r_c = sqrt(rho_c), where the penalty has
// unit curvature.  Direction -H g_u by the two-loop recursion over the last kLbfgsMemory
// pairs, H0 = (s.y / y.y) I (I before the first pair); backtracking Armijo line search from
// step 1 (c1 = 1e-4, at most kLbfgsHalvings halvings), accepting without the comparison a
// decrease below the objective's rounding noise; a pair is kept when s.y > 0; a failed line
// search ends the solve.  With kAlt, starts from the better of d and alt.  d in place.
template <typename T, bool kAlt = false>
__device__ __forceinline__ void local_solve_lbfgs(T z0, T z1, const T vbar[9], const T a[9], T d[9],
                                                  const Prm<T>& q, const T* alt = nullptr) {
  constexpr int M = kLbfgsMemory;
  T r[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) r[c] = Num<T>::sqrt_(q.rho(c));
  T v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = vbar[c] + d[c];
  Pose<T> P;
  pose_at(v, q.eps, P);
  T L = local_objective(d, a, P, z0, z1, q);
  if constexpr (kAlt) {
    T da[9], va[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      da[c] = alt[c];
      va[c] = vbar[c] + da[c];
    }
    Pose<T> Pa;
    pose_at(va, q.eps, Pa);
    const T La = local_objective(da, a, Pa, z0, z1, q);
    if (La < L) {
#pragma unroll
      for (int c = 0; c < 9; ++c) d[c] = da[c];
      P = Pa;
      L = La;
    }
  }
  T gu[9], noise;
  {
    T g[9];
    local_gradient(P, z0, z1, a, d, q, g, noise);
#pragma unroll
    for (int c = 0; c < 9; ++c) gu[c] = Num<T>::div(g[c], r[c]);
  }
  T S[M][9], Y[M][9], rh[M];
  int nh = 0, newest = -1;
  for (int it = 0; it < q.steps; ++it) {
    T qv[9], al[M];
#pragma unroll
    for (int c = 0; c < 9; ++c) qv[c] = gu[c];
    for (int h = 0; h < nh; ++h) {
      const int k = (newest - h + M) % M;
      T sq = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) sq += S[k][c] * qv[c];
      al[k] = rh[k] * sq;
#pragma unroll
      for (int c = 0; c < 9; ++c) qv[c] -= al[k] * Y[k][c];
    }
    T gamma = 1;
    if (nh > 0) {
      T sy = 0, yy = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        sy += S[newest][c] * Y[newest][c];
        yy += Y[newest][c] * Y[newest][c];
      }
      gamma = Num<T>::div(sy, yy);
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) qv[c] *= gamma;
    for (int h = nh - 1; h >= 0; --h) {
      const int k = (newest - h + M) % M;
      T yq = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) yq += Y[k][c] * qv[c];
      const T beta = rh[k] * yq;
#pragma unroll
      for (int c = 0; c < 9; ++c) qv[c] += S[k][c] * (al[k] - beta);
    }
    T p[9], gp = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      p[c] = -qv[c];
      gp += gu[c] * p[c];
    }
    if (!(gp < T(0))) {  // not a descent direction: steepest descent
      gp = 0;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        p[c] = -gu[c];
        gp -= gu[c] * gu[c];
      }
    }
    T t = 1, dt[9], Lt = Num<T>::inf();
    Pose<T> Pt;
    bool accepted = false;
    for (int hv = 0; hv <= kLbfgsHalvings; ++hv, t *= T(0.5)) {
      T vt[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        dt[c] = d[c] + Num<T>::div(t * p[c], r[c]);
        vt[c] = vbar[c] + dt[c];
      }
      pose_at(vt, q.eps, Pt);
      Lt = local_objective(dt, a, Pt, z0, z1, q);
      if (!(Lt < Num<T>::inf())) continue;
      const bool trust = isfinite(L) && q.model_tol > T(0) &&
                         -t * gp <= q.model_tol * Num<T>::unit_roundoff * (fabs(L) + noise);
      if (trust || Lt <= L + T(1e-4) * t * gp) {
        accepted = true;
        break;
      }
    }
    if (!accepted) break;
    T gt[9], noise_t, sv[9], yv[9], sy = 0;
    local_gradient(Pt, z0, z1, a, dt, q, gt, noise_t);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const T gut = Num<T>::div(gt[c], r[c]);
      sv[c] = t * p[c];
      yv[c] = gut - gu[c];
      sy += sv[c] * yv[c];
      gu[c] = gut;
    }
    if (sy > T(0)) {
      newest = (newest + 1) % M;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        S[newest][c] = sv[c];
        Y[newest][c] = yv[c];
      }
      rh[newest] = Num<T>::rcp(sy);
      if (nh < M) nh += 1;
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) d[c] = dt[c];
    L = Lt;
    noise = noise_t;
  }
}

// ---------------------------------------------------- learned warm start
// Features of one local problem (Eq. 9) for the warm-start network, in
// coordinates scaled by r_c = sqrt(rho_c) so that the consensus penalty reads
// |r (d + a)|^2 / 2 for every scene: residual at the start (2), sqrt of the
// IRLS weight (1), Jacobian / r (18), r (d0 + a) (9), two zeros.  Returns false
// (features zero) when the start is behind the camera.
constexpr int kMlpIn = 32, kMlpHidden = 64, kMlpOut = 16, kMlpUsedOut = 9;

template <typename T>
__device__ __forceinline__ bool warm_features(T z0, T z1, const T vbar[9], const T a[9], const T d0[9],
                                              const Prm<T>& q, float feat[kMlpIn], T r[9]) {
#pragma unroll
  for (int c = 0; c < 9; ++c) r[c] = Num<T>::sqrt_(q.rho(c));
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) feat[k] = 0.f;
  T v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = vbar[c] + d0[c];
  Pose<T> P;
  pose_at(v, q.eps, P);
  if (!P.valid) return false;
  T J0[9], J1[9], e0, e1, w;
  linearize(P, z0, z1, q, J0, J1, e0, e1, w);
  feat[0] = (float)e0;
  feat[1] = (float)e1;
  feat[2] = (float)Num<T>::sqrt_(w);
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const T ir = Num<T>::rcp(r[c]);
    feat[3 + c] = (float)(J0[c] * ir);
    feat[12 + c] = (float)(J1[c] * ir);
    feat[21 + c] = (float)(r[c] * (d0[c] + a[c]));
  }
  return true;
}

}  // namespace
}  // namespace dba
