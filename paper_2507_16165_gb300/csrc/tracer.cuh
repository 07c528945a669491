// Device-side ray tracer for the Schwarzschild renderer (sm_103a).
//
// One thread owns one ray.  The ray is reduced to its orbital plane through
// the hole (basis e1 toward the observer, e2 completing the plane), the
// photon-orbit equation u'' = 3Mu^2 - u (Eq. 1 of Naddell & Ponce, PEARC '25,
// with the sign fixed by the first integral) is integrated in the azimuth
// with Dormand-Prince 5(4), events are located on the quintic Hermite
// interpolant of each accepted step, and the result is mapped back to 3-D and
// shaded.  Everything is templated on the arithmetic type R (float or double).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bh_types.cuh"

namespace bhk {

// ---------------------------------------------------------------------------
// Precision-overloaded math.
// ---------------------------------------------------------------------------
// Square root.  sqrt_approx is the single-instruction hardware
// approximation (relative error about 2^-23, far inside the FP32 passes'
// 1e-4 rad budget; 0 gives 0, a negative argument NaN), used in the FP32
// arccos, the sphere windows and the warp's sphere cull; m_sqrt keeps the
// correctly rounded routine (in the mixed tile pass the approximation there
// measured 5% slower: the pass sits at its register limit and the changed
// code spilled more).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double m_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double m_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float m_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double m_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ double m_acos(double x) { return acos(x); }
__device__ __forceinline__ double m_asin(double x) { return asin(x); }
// sin and cos for the map-back: Cody & Waite argument reduction by 2 pi with
// a two-term split of 2 pi (float(2 pi) and its residual), then the hardware
// approximation on [-pi, pi] (absolute error below 4e-7).  The FP64
// overload is the accurate library routine.
__device__ __forceinline__ void m_sincos_mapback(float x, float* s, float* c) {
  const float k = rintf(x * 0.15915494309189535f);
  const float r = fmaf(k, 1.7484555e-7f, fmaf(-k, 6.28318548202514648f, x));
  __sincosf(r, s, c);
}
__device__ __forceinline__ void m_sincos_mapback(double x, double* s, double* c) { sincos(x, s, c); }
// sin and cos inside the FP32 event searches (sphere entry): the same
// reduction and hardware approximation; a 4e-7 error in g moves a located
// entry by far less than the FP32 passes' 1e-4 rad budget.  FP64 keeps the
// accurate routine.
__device__ __forceinline__ void m_sincos_evt(float x, float* s, float* c) { m_sincos_mapback(x, s, c); }
__device__ __forceinline__ void m_sincos_evt(double x, double* s, double* c) { sincos(x, s, c); }
// Single special-function-unit instructions (PTX approximate forms with
// denormals flushed to zero): reciprocal, reciprocal square root, base-2
// logarithm and exponential, each within a few ulp.  Their operands here are
// normal numbers or the limits 0 and infinity, whose results (infinity,
// -infinity, 0) the callers handle.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Programmatic dependent launch: a kernel lets the next kernel of its
// stream (launched with programmatic stream serialization) start once all
// of its blocks have called pdl_launch_dependents; the dependent's
// pdl_wait_primary returns when the first kernel has completed and its
// memory operations are visible.  Both are no-ops without such a launch.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_primary() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Quotient and reciprocal square root: the hardware approximations in FP32
// (a few ulp, far inside the FP32 passes' error budget), correctly rounded
// in FP64.
__device__ __forceinline__ float m_div(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
// Quotient of the event location (interpolant scaling, root iterations,
// sphere prefilter), which needs about 1e-14 relative in FP64, not a
// correctly rounded result: the FP32 reciprocal refined by one FP64 Newton
// step, y = y0 + y0 (1 - b y0) (relative error about 2^-46), three
// operations on the FP64 pipe and two conversions instead of a division's
// ten or so.  b = 0 or outside FP32's range gives NaN, which the root
// search treats as a step outside its bracket.
__device__ __forceinline__ float m_quot(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double m_quot(double a, double b) {
  const double y0 = (double)rcp_approx((float)b);
  return a * fma(y0, fma(-b, y0, 1.0), y0);
}
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrt_approx(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return 1.0 / sqrt(x); }

// Inverse trigonometric functions for the FP32 paths from the polynomial
// approximations of Abramowitz & Stegun: 4.4.49 for arctan on [-1, 1]
// (error below 2e-8) and 4.4.46 for arccos on [0, 1] (below 2e-8), with
// octant and sign reduction; FP32 evaluation adds about 1e-7.  The FP64
// overloads are the accurate library routines.
__device__ __forceinline__ float atan_unit(float t) {  // arctan, |t| <= 1
  const float t2 = t * t;
  float p = fmaf(t2, 0.0028662257f, -0.0161657367f);
  p = fmaf(t2, p, 0.0429096138f);
  p = fmaf(t2, p, -0.0752896400f);
  p = fmaf(t2, p, 0.1065626393f);
  p = fmaf(t2, p, -0.1420889944f);
  p = fmaf(t2, p, 0.1999355085f);
  p = fmaf(t2, p, -0.3333314528f);
  return fmaf(t * t2, p, t);
}
__device__ __forceinline__ float m_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  float a = mx > 0.0f ? atan_unit(mn * rcp_approx(mx)) : 0.0f;
  if (ay > ax) a = 1.57079632679489662f - a;
  if (x < 0.0f) a = 3.14159265358979324f - a;
  return copysignf(a, y);
}
__device__ __forceinline__ float m_acos(float x) {
  const float a = fminf(1.0f, fabsf(x));
  float p = fmaf(a, -0.0012624911f, 0.0066700901f);
  p = fmaf(a, p, -0.0170881256f);
  p = fmaf(a, p, 0.0308918810f);
  p = fmaf(a, p, -0.0501743046f);
  p = fmaf(a, p, 0.0889789874f);
  p = fmaf(a, p, -0.2145988016f);
  p = fmaf(a, p, 1.5707963050f);
  const float r = sqrt_approx(1.0f - a) * p;
  return x < 0.0f ? 3.14159265358979324f - r : r;
}
__device__ __forceinline__ float m_asin(float x) {
  return 1.57079632679489662f - m_acos(x);
}
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
__device__ __forceinline__ float m_ceil(float x) { return ceilf(x); }
__device__ __forceinline__ double m_ceil(double x) { return ceil(x); }
// Reciprocals of the error-norm scales only: the hardware approximation (a
// few ulp), as a relative error of 1e-6 in err^2 cannot change an accept
// decision except within 1e-6 of the threshold.  The double overload goes
// through single precision for the same reason.
__device__ __forceinline__ float m_rcp(float x) { return rcp_approx(x); }
__device__ __forceinline__ double m_rcp(double x) { return (double)rcp_approx((float)x); }

template <typename R> struct Num;
template <> struct Num<float> {
  static constexpr float pi = 3.14159265358979323846f;
  static constexpr float two_pi = 6.28318530717958647692f;
  static constexpr float tie = 1e-6f;          // event tie window (rad)
  static constexpr float radial = 1e-6f;       // |P x d| / |P| below: radial
  static constexpr int root_iters = 24;        // root iterations (bisection-safe)
  static constexpr int golden_iters = 32;
  
};
template <> struct Num<double> {
  static constexpr double pi = 3.14159265358979323846;
  static constexpr double two_pi = 6.28318530717958647692;
  static constexpr double tie = 1e-12;
  static constexpr double radial = 1e-12;
  static constexpr int root_iters = 60;
  static constexpr int golden_iters = 70;
};

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4) (Dormand & Prince 1980) for y = (u, v = u'),
// y' = (v, F(u)), F(u) = 3Mu^2 - u.  The published tableau a_sj, weights
// b_j and error weights E_j = b_j - bhat_j, stage s evaluated at
// U_s = u + h sum_j a_sj V_j with V_j = v + h sum_k a_jk F_k, F_1 = F(u),
// F_s = F(U_s) and the 7th stage the fifth-order solution (first same as
// last).  Because F does not depend on v, substituting V_j gives the same
// method in second-order (Nystrom) form, which never forms the V_s:
//   U_s   = u + c_s h v + h^2 sum_k abar_sk F_k,   abar_sk = sum_j a_sj a_jk
//   u_new = u + h v + h^2 sum_k bbar_k F_k,         bbar_k  = sum_j b_j a_jk
//   v_new = v + h sum_k b_k F_k
//   e_u   = h^2 sum_k ehat_k F_k,                   ehat_k  = sum_j E_j a_jk
//   e_v   = h sum_j E_j F_j
// (e_u has no h v term since the E_j sum to zero).  The derived
// coefficients below are those sums in exact rational arithmetic; zeros
// (abar_{s,s-1}, bbar_2, bbar_6, ehat_2) are left out.  In exact arithmetic
// every quantity equals the first-order form's; this form takes 57
// floating-point operations per attempted step instead of about 80.
// ---------------------------------------------------------------------------
#define DP_C2 (1.0 / 5.0)
#define DP_C3 (3.0 / 10.0)
#define DP_C4 (4.0 / 5.0)
#define DP_C5 (8.0 / 9.0)
#define DP_AB31 (9.0 / 200.0)
#define DP_AB41 (-12.0 / 25.0)
#define DP_AB42 (4.0 / 5.0)
#define DP_AB51 (-12248.0 / 6561.0)
#define DP_AB52 (7208.0 / 2187.0)
#define DP_AB53 (-6784.0 / 6561.0)
#define DP_AB61 (-533.0 / 264.0)
#define DP_AB62 (91.0 / 22.0)
#define DP_AB63 (-56.0 / 33.0)
#define DP_AB64 (7.0 / 88.0)
#define DP_BB1 (35.0 / 384.0)
#define DP_BB3 (50.0 / 159.0)
#define DP_BB4 (25.0 / 192.0)
#define DP_BB5 (-243.0 / 6784.0)
#define DP_B1 (35.0 / 384.0)
#define DP_B3 (500.0 / 1113.0)
#define DP_B4 (125.0 / 192.0)
#define DP_B5 (-2187.0 / 6784.0)
#define DP_B6 (11.0 / 84.0)
#define DP_EH1 (611.0 / 230400.0)
#define DP_EH3 (-514.0 / 83475.0)
#define DP_EH4 (391.0 / 38400.0)
#define DP_EH5 (-4617.0 / 1356800.0)
#define DP_EH6 (-11.0 / 3360.0)
#define DP_E1 (71.0 / 57600.0)
#define DP_E3 (-71.0 / 16695.0)
#define DP_E4 (71.0 / 1920.0)
#define DP_E5 (-17253.0 / 339200.0)
#define DP_E6 (22.0 / 525.0)
#define DP_E7 (-1.0 / 40.0)

template <typename R>
__device__ __forceinline__ R accel(R M3, R u) {
  return u * m_fma(M3, u, R(-1));  // 3Mu^2 - u
}

// One attempted step.  Returns the fifth-order state (un, vn), the FSAL
// derivative fn = accel(un), and the squared Hairer error norm
// err2 = ((eu/su)^2 + (ev/sv)^2) / 2 with su = atol + rtol max(|u|, |un|).
// The error estimate (eu, ev) is formed in the working precision (it is a
// small difference of stage sums); its normalisation and err2 are FP32 for
// both types: err2 only steers the step size, which the FP32 step factor
// already perturbs at 1e-7 relative, and decides acceptance, which a 1e-7
// relative change of err2 can flip only within 1e-7 of err2 = 1.  In FP64
// that takes the norm from 14 operations on the FP64 pipe to 6 conversions.
template <typename R>
__device__ __forceinline__ void dp5_attempt(R M3, R u, R v, R f1, R h, R rtol, R atol,
                                            R& un, R& vn, R& fn, float& err2) {
  const R hv = h * v, h2 = h * h;
  const R F2 = accel(M3, m_fma(R(DP_C2), hv, u));
  const R F3 = accel(M3, m_fma(h2, R(DP_AB31) * f1, m_fma(R(DP_C3), hv, u)));
  const R F4 = accel(M3, m_fma(h2, m_fma(R(DP_AB42), F2, R(DP_AB41) * f1), m_fma(R(DP_C4), hv, u)));
  const R F5 = accel(M3, m_fma(h2, m_fma(R(DP_AB53), F3, m_fma(R(DP_AB52), F2, R(DP_AB51) * f1)),
                               m_fma(R(DP_C5), hv, u)));
  const R uhv = u + hv;
  const R F6 = accel(M3, m_fma(h2, m_fma(R(DP_AB64), F4, m_fma(R(DP_AB63), F3,
                                     m_fma(R(DP_AB62), F2, R(DP_AB61) * f1))), uhv));
  un = m_fma(h2, m_fma(R(DP_BB5), F5, m_fma(R(DP_BB4), F4, m_fma(R(DP_BB3), F3, R(DP_BB1) * f1))), uhv);
  vn = m_fma(h, m_fma(R(DP_B6), F6, m_fma(R(DP_B5), F5, m_fma(R(DP_B4), F4,
                m_fma(R(DP_B3), F3, R(DP_B1) * f1)))), v);
  fn = accel(M3, un);
  // embedded error (fifth minus fourth order)
  const R eu = h2 * m_fma(R(DP_EH6), F6, m_fma(R(DP_EH5), F5, m_fma(R(DP_EH4), F4,
                m_fma(R(DP_EH3), F3, R(DP_EH1) * f1))));
  const R ev = h * m_fma(R(DP_E7), fn, m_fma(R(DP_E6), F6, m_fma(R(DP_E5), F5,
                m_fma(R(DP_E4), F4, m_fma(R(DP_E3), F3, R(DP_E1) * f1)))));
  const float rt = (float)rtol, at = (float)atol;
  const float su = fmaf(rt, fmaxf(fabsf((float)u), fabsf((float)un)), at);
  const float sv = fmaf(rt, fmaxf(fabsf((float)v), fabsf((float)vn)), at);
  const float ru = (float)eu * rcp_approx(su), rv = (float)ev * rcp_approx(sv);
  err2 = 0.5f * fmaf(ru, ru, rv * rv);
}

// Step-size factor 0.9 err^(-1/5) clamped to [0.2, 10], from err2 = err^2.
// Computed in single precision for both arithmetic types: it only steers the
// step size (a relative change of 1e-7 in h moves the solution by far less
// than the tolerance); acceptance uses err2 <= 1 in the working precision.
// Without branches: err2 = 0 gives log2 = -inf and a factor clamped to 10;
// NaN propagates to fmaxf, which returns 0.2.  The 0.9 is folded into the
// exponent as log2(0.9).
template <typename R>
__device__ __forceinline__ R step_factor(float err2) {
  const float e2 = err2;
  const float fac = ex2_approx(fmaf(-0.1f, lg2_approx(e2), -0.15200309344504997f));
  return R(fminf(10.0f, fmaxf(0.2f, fac)));
}

// Starting step (Hairer, Norsett & Wanner, Solving ODEs I, II.4), capped at
// cap rad.
template <typename R>
__device__ R initial_step(R M3, R u, R v, R rtol, R atol, R cap) {
  const R scu = m_fma(rtol, m_abs(u), atol), scv = m_fma(rtol, m_abs(v), atol);
  const R fu = v, fv = accel(M3, u);
  const R iu = R(1) / scu, iv = R(1) / scv;
  const R d0 = m_sqrt(R(0.5) * ((u * iu) * (u * iu) + (v * iv) * (v * iv)));
  const R d1 = m_sqrt(R(0.5) * ((fu * iu) * (fu * iu) + (fv * iv) * (fv * iv)));
  const R h0 = (d0 < R(1e-5) || d1 < R(1e-5)) ? R(1e-6) : R(0.01) * d0 / d1;
  const R u1 = m_fma(h0, fu, u), v1 = m_fma(h0, fv, v);
  const R gu = v1 - fu, gv = accel(M3, u1) - fv;
  const R d2 = m_sqrt(R(0.5) * ((gu * iu) * (gu * iu) + (gv * iv) * (gv * iv))) / h0;
  const R dm = m_max(d1, d2);
  R h1;
  if (dm <= R(1e-15)) {
    h1 = m_max(R(1e-6), h0 * R(1e-3));
  } else {
    h1 = R(exp2f(0.2f * __log2f((float)(R(0.01) / dm))));
  }
  return m_min(m_min(R(100) * h0, h1), cap);
}

// ---------------------------------------------------------------------------
// Quintic Hermite interpolant of u on [pa, pa + h] from u, h u', h^2 u''
// at both ends, held in the power basis of the normalised t in [0, 1]:
//   p(t) = c0 + c1 t + c2 t^2 + c3 t^3 + c4 t^4 + c5 t^5,
// c0 = u_a, c1 = h v_a, c2 = h^2 f_a / 2, and with the end mismatches
// A = u_b - (c0 + c1 + c2), B = h v_b - (c1 + 2 c2), C = h^2 f_b - 2 c2,
// c3 = 10A - 4B + C/2, c4 = -15A + 7B - C, c5 = 6A - 3B + C/2 (the unique
// solution of the three end conditions).  Values and slopes are then 5 and 4
// fused multiply-adds.
// ---------------------------------------------------------------------------
template <typename R>
struct Hermite {
  R pa, h, ih;
  R c0, c1, c2, c3, c4, c5;
  __device__ __forceinline__ void make(R pa_, R h_, R ua, R va, R fa, R ub, R vb, R fb) {
    pa = pa_;
    h = h_;
    ih = m_quot(R(1), h_);
    const R hh = h_ * h_;
    c0 = ua;
    c1 = h_ * va;
    c2 = R(0.5) * hh * fa;
    const R A = ub - (c0 + c1 + c2);
    const R B = m_fma(h_, vb, -m_fma(R(2), c2, c1));
    const R C = m_fma(hh, fb, R(-2) * c2);
    c3 = m_fma(R(10), A, m_fma(R(-4), B, R(0.5) * C));
    c4 = m_fma(R(-15), A, m_fma(R(7), B, -C));
    c5 = m_fma(R(6), A, m_fma(R(-3), B, R(0.5) * C));
  }
  // value at normalised t
  __device__ __forceinline__ R val_t(R t) const {
    return m_fma(t, m_fma(t, m_fma(t, m_fma(t, m_fma(t, c5, c4), c3), c2), c1), c0);
  }
  // d/dt of the interpolant
  __device__ __forceinline__ R dval_t(R t) const {
    return m_fma(t, m_fma(t, m_fma(t, m_fma(t, R(5) * c5, R(4) * c4), R(3) * c3), R(2) * c2), c1);
  }
  __device__ __forceinline__ R t_of(R phi) const { return (phi - pa) * ih; }
  __device__ __forceinline__ R u_at(R phi) const { return val_t(t_of(phi)); }
  __device__ __forceinline__ R v_at(R phi) const { return dval_t(t_of(phi)) * ih; }
  // end values in the scaled form: h u' at t = 0 and t = 1
  __device__ __forceinline__ R d_start() const { return c1; }
  __device__ __forceinline__ R d_end() const { return dval_t(R(1)); }
};

// Root t in [lo, hi] of val_t(t) - target, given a sign change, by Newton
// steps kept inside a shrinking bracket (bisection when Newton leaves it).
// Convergence is tested on the Newton step before the bracket test: at the
// root the sign of the residual is rounding noise, and a step that lands a
// hair outside the bracket must end the search, not restart it from the
// bracket's midpoint.
template <typename R>
__device__ R hermite_root(const Hermite<R>& H, R target, R lo, R hi) {
  R flo = H.val_t(lo) - target;
  R t = lo + (hi - lo) * m_quot(flo, flo - (H.val_t(hi) - target));
  if (!(t > lo && t < hi)) t = R(0.5) * (lo + hi);
  for (int it = 0; it < Num<R>::root_iters; ++it) {
    const R f = H.val_t(t) - target;
    if (f == R(0)) return t;
    if ((f > R(0)) == (flo > R(0))) {
      lo = t;
      flo = f;
    } else {
      hi = t;
    }
    const R df = H.dval_t(t);
    R tn = t - m_quot(f, df);
    if (m_abs(tn - t) * H.h < R(sizeof(R) == 8 ? 1e-15 : 1e-7)) return m_min(hi, m_max(lo, tn));
    if (!(tn > lo && tn < hi)) tn = R(0.5) * (lo + hi);
    t = tn;
  }
  return t;
}

// ---------------------------------------------------------------------------
// Per-ray state.
// ---------------------------------------------------------------------------
// Angular windows of the spheres that a ray's plane cuts (centre and
// half-width, rad, from the set-up).  They are indexed by sphere and so live
// in local memory; they are kept apart from the Ray so that the Ray itself
// stays in registers (an indexed array inside it kept the whole struct in
// local memory, with its fields stored at every step).
struct SphWin {
  float c[kMaxSph];
  float d[kMaxSph];
};

template <typename R>
struct Ray {
  R u, v, f, phi, h;     // state, FSAL derivative, azimuth, next step
  R e1x, e1y, e1z, e2x, e2y, e2z;  // plane basis
  R phi_node;            // next disk node angle (> phi), or +inf
  R phi_sph;             // next sphere-window start, or +inf
  R phi_evt;             // min(phi_node, phi_sph, phi_max): steps ending
                         // before it need no event search
  R es;                  // scale of the squared error norm: the ray's tolerance
                         // tier (1, (rtol/rtol_far)^2 or (rtol/rtol_near)^2)
  R hc;                  // step-size cap of the ray's tier (h_max or h_max_far)
  R up;                  // periastron u of the orbit (MIXED reset), NaN if none
  R tp;                  // MIXED: 0 while the turning-point reset is pending, else -inf
  unsigned sph_mask;     // spheres whose in-plane circle is non-empty
  SphWin* win;           // angular window of each such sphere
  int steps;             // attempted steps
  int out;               // output pixel index
  unsigned aux;          // BAND / FP64 provenance bits, periastron-done bit
};

constexpr unsigned kAuxPeriDone = 1u << 16;
constexpr unsigned kAuxFar = 1u << 17;  // ray takes the relaxed step cap h_far
constexpr unsigned kAuxNear = 1u << 18; // FP32 form: ray held to rtol_near

// Event produced when a ray terminates.
template <typename R>
struct Hit {
  unsigned flags;  // low byte BH_FLAG_*, high byte sphere id
  R phi;           // event angle
  R u, v;          // state at the event
};

// Camera ray through the image point (px + ox, py + oy), by default the
// centre of pixel (px, py); row 0 is at the top.
template <typename R>
__device__ __forceinline__ void camera_ray(const CamK& c, int px, int py, R P[3], R d[3],
                                           R ox = R(0.5), R oy = R(0.5)) {
  const CamR<R>& C = CR<R>(c);
  const R sx = m_fma(R(px) + ox, C.px_scale, -C.sx);
  const R sy = m_fma(-(R(py) + oy), C.py_scale, C.sy);
  R dd[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    P[k] = C.pos[k];
    dd[k] = C.fwd[k] + sx * C.right[k] + sy * C.up[k];
  }
  const R inv = m_rsqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = dd[k] * inv;
}

// Angular window [phi_c - dphi, phi_c + dphi] of sphere k in the ray's
// plane: the directions from the hole that meet the sphere's in-plane
// circle.  (cx, cy): the sphere centre in the plane's basis.  Evaluated once
// per ray in single precision for both arithmetic types (it only gates the
// exact test) and widened by 1e-4 rad.
template <typename R>
__device__ __forceinline__ void sphere_window_setup(const SceneK& s, Ray<R>& r, int k, float cx,
                                                    float cy) {
  const float rho2 = cx * cx + cy * cy;
  const float rp2 = fmaxf(0.0f, s.f.rad[k] * s.f.rad[k] - (s.f.c2[k] - rho2));
  float pc = m_atan2(cy, cx);
  if (pc < 0.0f) pc += 6.28318530717958647692f;
  r.win->c[k] = pc;
  r.win->d[k] = m_asin(fminf(1.0f, sqrt_approx(rp2 * rcp_approx(rho2)))) + 1e-4f;
}

// The first window of sphere k whose end lies at or after phi_from:
// returns its start, *we its end.
template <typename R>
__device__ __forceinline__ float sphere_window(const Ray<R>& r, int k, float phi_from, float* we) {
  const float pc = r.win->c[k], dp = r.win->d[k];
  const float m = ceilf((phi_from - pc - dp) * 0.15915494309189535f);
  *we = pc + dp + 6.28318530717958647692f * m;
  return pc - dp + 6.28318530717958647692f * m;
}

template <typename R>
__device__ __forceinline__ R next_sphere_window(const Ray<R>& r, R phi_from) {
  float best = INFINITY;
  unsigned m = r.sph_mask;
  while (m) {
    const int k = __ffs(m) - 1;
    m &= m - 1;
    float we;
    best = fminf(best, sphere_window(r, k, (float)phi_from, &we));
  }
  return R(best);
}

// Spheres whose circle the orbital plane of some ray of this warp's 32 rays
// may cut (all lanes call it; the rays share one camera).  With the plane's
// normal n = (sx up - sy right) / rho, sphere k is cut when
// g(sx, sy) = |sx (up . c_k) - sy (right . c_k)| - R_k rho < 0.  g changes by
// at most (|c_k| + R_k) per unit distance in the image plane, so when it is
// positive by more than that times the distance from lane 0's point to the
// farthest point of the group (plus a pixel diagonal, for sub-pixel samples)
// no ray of the group cuts the sphere.  The exact test per ray follows for
// the spheres that remain.
template <typename R>
__device__ __forceinline__ unsigned warp_sphere_candidates(const SceneK& s, const CamK& cam, R sx,
                                                           R sy) {
  const unsigned full = 0xFFFFFFFFu;
  const float fx = (float)sx, fy = (float)sy;
  const float x0 = __shfl_sync(full, fx, 0), y0 = __shfl_sync(full, fy, 0);
  const float dx = fx - x0, dy = fy - y0;
  const float d2 = fmaf(dx, dx, dy * dy);
  const float dmax = sqrt_approx(__uint_as_float(__reduce_max_sync(full, __float_as_uint(d2))));
  const float reach = fmaf(dmax + cam.f.pdiag, 1.0001f, 1e-5f);
  const int k = threadIdx.x & 31;
  bool maybe = false;
  if (k < s.n_sph) {
    const float rho0 = sqrt_approx(fmaf(x0, x0, y0 * y0));
    const float g = fabsf(fmaf(x0, cam.f.uc[k], -y0 * cam.f.rc[k])) - s.f.rad[k] * rho0;
    maybe = g <= (s.f.cnorm[k] + s.f.rad[k]) * reach;
  }
  return __ballot_sync(full, maybe);
}

// Orbital-plane set-up of the ray through image-plane point (sx, sy) of
// camera cam.  Returns 0 for a ray to integrate, 1 for a radial ray (handled
// by the caller with straight-line geometry).  cand: the spheres to test
// for a cut of the plane (warp_sphere_candidates, or all of them).  WIN:
// the angular windows of the cut spheres too; without them (the surrogate
// pass, which hands every ray whose plane cuts a sphere to the integrator)
// sph_mask holds the first cut sphere only.
template <typename R, bool WIN = true>
__device__ int plane_setup(const SceneK& s, const CamK& cam, R sx, R sy, unsigned cand, Ray<R>& r,
                           R* b_out, R* cos_a_out) {
  const CamR<R>& C = CR<R>(cam);
  r.e1x = -C.fwd[0];
  r.e1y = -C.fwd[1];
  r.e1z = -C.fwd[2];
  const R rho2 = m_fma(sx, sx, sy * sy);
  // |P x d| / |P| = sin(alpha) = rho / sqrt(1 + rho^2); cos(alpha) = d . e1
  const R iL = m_rsqrt(R(1) + rho2);
  *cos_a_out = -iL;
  if (rho2 < R(Num<R>::radial) * R(Num<R>::radial)) {
    *b_out = R(0);
    return 1;
  }
  const R irho = m_rsqrt(rho2);
  r.e2x = m_fma(sx, C.right[0], sy * C.up[0]) * irho;
  r.e2y = m_fma(sx, C.right[1], sy * C.up[1]) * irho;
  r.e2z = m_fma(sx, C.right[2], sy * C.up[2]) * irho;
  const R sin_a = rho2 * irho * iL;
  const SceneR<R>& S = SR<R>(s);
  const R M = S.M;
  const R u0 = C.ir;
  R b;
  if (s.ic == 0) {
    b = C.kb * sin_a;
  } else {
    b = C.r_obs * sin_a * m_rsqrt(R(1) - R(2) * M * sin_a * sin_a * u0);
  }
  // u'0 = -u0 cot(alpha) sqrt(1 - 2M u0) (static) or -u0 cot(alpha), with
  // cot(alpha) = -1 / rho
  r.v = C.kv * irho;
  *b_out = b;
  r.u = u0;
  r.f = accel(S.M3, u0);
  r.phi = R(0);
  // disk nodes: z(phi) ~ cos(phi) e1z + sin(phi) e2z
  r.phi_node = R(INFINITY);
  if (s.disk_on) {
    const R a = r.e1z, c = r.e2z;
    if (a * a + c * c >= R(sizeof(R) == 8 ? 1e-24 : 1e-12)) {
      R p0 = m_atan2(-a, c);
      if (p0 < R(0)) p0 += Num<R>::pi;
      if (p0 >= Num<R>::pi) p0 -= Num<R>::pi;
      r.phi_node = (p0 > R(0)) ? p0 : Num<R>::pi;
    }
  }
  // spheres cut by the plane (|n . c_k| < R_k) and not wholly inside the
  // orbit's periastron (SceneR::cull_b); their windows from the centre's
  // coordinates in the plane, c . e1 (per camera) and c . e2
  unsigned mask = 0;
  r.phi_sph = R(INFINITY);
  while (cand) {
    const int k = __ffs(cand) - 1;
    cand &= cand - 1;
    const R nc = m_fma(sx, C.uc[k], -sy * C.rc[k]);
    if (m_abs(nc) < S.rad[k] * rho2 * irho && b <= S.cull_b[k]) {
      mask |= 1u << k;
      if (!WIN) break;
      sphere_window_setup(s, r, k, (float)C.ec[k], (float)(m_fma(sx, C.rc[k], sy * C.uc[k]) * irho));
    }
  }
  r.sph_mask = mask;
  if (WIN && mask) r.phi_sph = next_sphere_window(r, R(0));
  return 0;
}

// g(phi) < 0 inside sphere k's in-plane circle (u^2 (|p - c'|^2 - R'^2)).
template <typename R>
__device__ __forceinline__ R sphere_g(R cx, R cy, R K, R phi, R u) {
  R sp, cp;
  m_sincos_evt(phi, &sp, &cp);
  return m_fma(K * u, u, m_fma(R(-2) * u, m_fma(cx, cp, cy * sp), R(1)));
}

// First entry into sphere k during the accepted step [pa, pb] (u at the
// ends ua, ub from the interpolant H).  A step's arc never leaves the
// straight chord between its end points by more than 3M q^2 h^2 / 8 in
// radius (the deviation w from the chord obeys w'' + w = 3Mu^2 with zero end
// values; q = u_max / u_min on the step), so steps whose chord passes farther
// than R' + that margin from the circle are rejected without a search.
//
// The search runs in the event type R, which may be narrower than the ray's
// stepping type T (the FP64 band pass of the MIXED mode locates its events
// in FP32); pa, pb and the result are then angles relative to a multiple
// of 2 pi, which leaves the sphere windows unchanged.
template <typename R, typename T>
__device__ bool sphere_entry(const SceneK& s, const Ray<T>& r, int k, const Hermite<R>& H,
                             R pa, R pb, R* phi_hit) {
  float wef;
  const float wsf = sphere_window(r, k, (float)pa, &wef);
  if (R(wsf) > pb || R(wef) < pa) return false;
  R lo = m_max(pa, R(wsf)), hi = m_min(pb, R(wef));
  if (!(hi > lo)) return false;
  const SceneR<R>& S = SR<R>(s);
  const R c0 = S.c[k][0], c1 = S.c[k][1], c2 = S.c[k][2];
  const R cx = c0 * R(r.e1x) + c1 * R(r.e1y) + c2 * R(r.e1z);
  const R cy = c0 * R(r.e2x) + c1 * R(r.e2y) + c2 * R(r.e2z);
  const R K = S.K[k];
  const R rp2 = S.rad[k] * S.rad[k] - (S.c2[k] - (cx * cx + cy * cy));
  if (!(rp2 > R(0))) return false;
  const R ulo = H.u_at(lo), uhi = H.u_at(hi);
  if (ulo > R(0) && uhi > R(0)) {
    R sa, ca, sb, cb;
    m_sincos_evt(lo, &sa, &ca);
    m_sincos_evt(hi, &sb, &cb);
    const R ia = m_quot(R(1), ulo), ib = m_quot(R(1), uhi);
    const R ax = ca * ia, ay = sa * ia;
    const R bx = cb * ib - ax, by = sb * ib - ay;
    const R qx = cx - ax, qy = cy - ay;
    const R bb = m_fma(bx, bx, by * by);
    R t = bb > R(0) ? m_quot(m_fma(qx, bx, qy * by), bb) : R(0);
    t = m_min(R(1), m_max(R(0), t));
    const R dx = qx - t * bx, dy = qy - t * by;
    const R q = m_quot(m_max(ulo, uhi), m_min(ulo, uhi));
    const R hh = hi - lo;
    const R margin = R(0.47) * S.M3 * q * q * hh * hh + R(1e-6);
    const R reach = m_sqrt(rp2) + margin;
    if (m_fma(dx, dx, dy * dy) > reach * reach) return false;
  }
  // careful search on the interpolant
  const R glo = sphere_g(cx, cy, K, lo, ulo);
  if (!(glo > R(0))) {
    *phi_hit = lo;
    return true;
  }
  R a_lo = lo, a_hi, g_lo = glo, g_hi;
  const R ghi = sphere_g(cx, cy, K, hi, uhi);
  if (ghi <= R(0)) {
    a_hi = hi;
    g_hi = ghi;
  } else {
    // golden-section search for the minimum of g on [lo, hi]
    R x0 = lo, x3 = hi, g0 = glo;
    const R gr = R(0.6180339887498949);
    R x1 = x3 - gr * (x3 - x0), x2 = x0 + gr * (x3 - x0);
    R g1 = sphere_g(cx, cy, K, x1, H.u_at(x1));
    R g2 = sphere_g(cx, cy, K, x2, H.u_at(x2));
    bool found = false;
    for (int it = 0; it < Num<R>::golden_iters; ++it) {
      if (g1 <= R(0) || g2 <= R(0)) {
        found = true;
        break;
      }
      if (g1 < g2) {
        x3 = x2;
        x2 = x1;
        g2 = g1;
        x1 = x3 - gr * (x3 - x0);
        g1 = sphere_g(cx, cy, K, x1, H.u_at(x1));
      } else {
        x0 = x1;
        g0 = g1;
        x1 = x2;
        g1 = g2;
        x2 = x0 + gr * (x3 - x0);
        g2 = sphere_g(cx, cy, K, x2, H.u_at(x2));
      }
      if (x3 - x0 < R(sizeof(R) == 8 ? 1e-13 : 1e-6)) break;
    }
    if (!found) return false;
    a_hi = (g1 <= R(0)) ? x1 : x2;
    g_hi = (g1 <= R(0)) ? g1 : g2;
    a_lo = x0;
    g_lo = g0;
  }
  // the entry: g(a_lo) > 0 >= g(a_hi), by regula falsi with the Illinois
  // modification (the value kept at an end that stays twice is halved), so
  // the bracket shrinks from both sides; a point outside the open bracket
  // falls back to the midpoint.  The bracket holds the entry throughout, as
  // bisection's does, and converges superlinearly instead of linearly.
  int side = 0;
  for (int it = 0; it < Num<R>::root_iters; ++it) {
    R mid = a_lo + (a_hi - a_lo) * m_quot(g_lo, g_lo - g_hi);
    if (!(mid > a_lo && mid < a_hi)) mid = R(0.5) * (a_lo + a_hi);
    if (!(mid > a_lo && mid < a_hi)) break;
    const R gm = sphere_g(cx, cy, K, mid, H.u_at(mid));
    if (gm > R(0)) {
      a_lo = mid;
      g_lo = gm;
      if (side == 1) g_hi *= R(0.5);
      side = 1;
    } else {
      a_hi = mid;
      g_hi = gm;
      if (side == -1) g_lo *= R(0.5);
      side = -1;
    }
    if (a_hi - a_lo < R(sizeof(R) == 8 ? 1e-14 : 1e-7)) break;
  }
  *phi_hit = a_hi;
  return true;
}

// ---------------------------------------------------------------------------
// Shading and stores.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned quant8(float c) {
  float q = floorf(fmaf(255.0f, c, 0.5f));
  q = fminf(255.0f, fmaxf(0.0f, q));
  return (unsigned)q;
}

__device__ __forceinline__ unsigned pack_rgba(float r, float g, float b) {
  return quant8(r) | (quant8(g) << 8) | (quant8(b) << 16) | (255u << 24);
}

// Sky image: bilinear in linear colour between the four texel centres
// around (theta, phi), wrapping in phi, clamped at the first and last rows.
template <typename R>
__device__ __noinline__ void sky_image_rgb(const SceneK& s, R theta, R phi, float rgb[3]) {
  const int W = s.sky_w, H = s.sky_h;
  const R x = phi * R(W * 0.15915494309189535) - R(0.5);
  const R y = theta * R(H * 0.31830988618379067) - R(0.5);
  const R x0 = m_floor(x), y0 = m_floor(y);
  const float fx = (float)(x - x0), fy = (float)(y - y0);
  const int i0 = (int)x0, j0 = (int)y0;
  const int ia = ((i0 % W) + W) % W, ib = (((i0 + 1) % W) + W) % W;
  const int ja = min(H - 1, max(0, j0)), jb = min(H - 1, max(0, j0 + 1));
  const uint32_t t00 = __ldg(&s.sky_tex[(size_t)ja * W + ia]), t10 = __ldg(&s.sky_tex[(size_t)ja * W + ib]);
  const uint32_t t01 = __ldg(&s.sky_tex[(size_t)jb * W + ia]), t11 = __ldg(&s.sky_tex[(size_t)jb * W + ib]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float c00 = (float)((t00 >> (8 * c)) & 255u), c10 = (float)((t10 >> (8 * c)) & 255u);
    const float c01 = (float)((t01 >> (8 * c)) & 255u), c11 = (float)((t11 >> (8 * c)) & 255u);
    const float top = fmaf(fx, c10 - c00, c00), bot = fmaf(fx, c11 - c01, c01);
    rgb[c] = fmaf(fy, bot - top, top) * (1.0f / 255.0f);
  }
}

// Colour of sky cell (i, j): parity picks the base colour, a splitmix64
// hash of the seed and the cell tints each channel.
__device__ __forceinline__ void sky_cell_rgb(unsigned long long seed, int i, int j, float rgb[3]) {
  const bool light = ((i + j) & 1) == 0;
  const unsigned long long hsh = splitmix64(seed * 2654435761ull + (unsigned long long)(32 * i + j));
  const float base[3] = {light ? 0.9f : 0.1f, light ? 0.9f : 0.1f, light ? 0.9f : 0.25f};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float slice = (float)((hsh >> (16 * c)) & 0xFFFFFFull);
    // (0.75 + 0.25 slice / 2^24), evaluated in double-free single precision
    rgb[c] = base[c] * (0.75f + 0.25f * (slice * (1.0f / 16777216.0f)));
  }
}

// Checkerboard sky: the 16 x 32 cells in (theta, phi); the cell colours come
// from the scene's table of the 512 cell colours (made by sky_cell_rgb when
// the scene is created), or are computed when the scene has none.
template <typename R>
__device__ __forceinline__ void sky_rgb(const SceneK& s, R theta, R phi, float rgb[3]) {
  int i = (int)m_floor(theta * R(5.09295817894065074));   // 16 / pi
  int j = (int)m_floor(phi * R(5.09295817894065074));     // 32 / (2 pi)
  i = min(15, max(0, i));
  j = min(31, max(0, j));
  if (s.sky_lut) {
    const float4 t = __ldg(&s.sky_lut[32 * i + j]);
    rgb[0] = t.x;
    rgb[1] = t.y;
    rgb[2] = t.z;
  } else {
    sky_cell_rgb(s.seed, i, j, rgb);
  }
}

// Colour accumulator of one pixel rendered with several samples: the
// stratified samples add their linear colour; the extra ray through the
// pixel centre stores the pixel's direction and flags.
struct SppAcc {
  float c[3];
  bool centre;
};

template <typename R>
__device__ __forceinline__ void dir_angles(R x, R y, R z, R* th, R* ph) {
  z = m_min(R(1), m_max(R(-1), z));
  *th = m_acos(z);
  R p = m_atan2(y, x);
  if (p < R(0)) p += Num<R>::two_pi;
  *ph = p;
}

// Store one finished ray.  OutR is the element type of out_dirs.
template <typename OutR>
__device__ __forceinline__ void store_ray(const Params& p, int out, OutR th, OutR ph, unsigned flags,
                                          unsigned rgba) {
  if (p.dirs) {
    OutR* d = reinterpret_cast<OutR*>(p.dirs);
    d[out] = th;
    d[(long long)p.n_rays + out] = ph;
  }
  if (p.flags) p.flags[out] = (uint16_t)flags;
  if (p.rgba) p.rgba[out] = rgba;
}

// Frequency ratio camera / gas of a disk hit for gas on prograde Keplerian
// orbits about +z: with Omega = sqrt(M/r^3) and lambda = b n_z, the traced
// ray's angular momentum about z per unit energy (the photon's is -lambda),
//   g = sqrt(1 - 3M/r) / (sqrt(1 - 2M/r_obs) (1 + Omega lambda));
// b from the first integral at the hit, 1/b^2 = u'^2 + u^2 (1 - 2Mu), and
// r_obs from the camera the output pixel belongs to.  No circular orbit
// inside 3M: g = 0.
template <typename R>
__device__ float disk_shift(const Params& p, const Ray<R>& r, float u, float v) {
  const float M = p.s.f.M;
  const float a = fmaf(-3.0f * M, u, 1.0f);
  if (!(a > 0.0f)) return 0.0f;
  int lo = 0, hi = p.n_cams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.cams[mid].out_off <= r.out)
      lo = mid;
    else
      hi = mid - 1;
  }
  const float u0 = p.cams[lo].f.ir;
  const float b = rsqrt_approx(fmaf(v, v, u * u * fmaf(-2.0f * M, u, 1.0f)));
  const float nz = (float)(r.e1x * r.e2y - r.e1y * r.e2x);
  const float omega = sqrtf(M * u * u * u);
  return sqrtf(a) * rsqrt_approx(fmaf(-2.0f * M, u0, 1.0f)) * rcp_approx(fmaf(omega * b, nz, 1.0f));
}

// Hand a finished ray's outputs over: stored directly, or with several
// samples per pixel (SPP) added to the pixel's colour (stratified samples)
// or stored without colour (the centre ray).
template <typename OutR, bool SPP>
__device__ __forceinline__ void emit_ray(const Params& p, int out, OutR th, OutR ph, unsigned flags,
                                         const float c[3], SppAcc* acc) {
  if (!SPP) {
    store_ray<OutR>(p, out, th, ph, flags, pack_rgba(c[0], c[1], c[2]));
  } else if (acc->centre) {
    if (p.dirs) {
      OutR* d = reinterpret_cast<OutR*>(p.dirs);
      d[out] = th;
      d[(long long)p.n_rays + out] = ph;
    }
    if (p.flags) p.flags[out] = (uint16_t)flags;
  } else {
    acc->c[0] += c[0];
    acc->c[1] += c[1];
    acc->c[2] += c[2];
  }
}

// Map a terminated ray back to 3-D, shade it and store it.  The map-back
// and shading run in the output precision OutR: an FP64 ray of the MIXED
// band is reduced to phi mod 2 pi in FP64 and finished in FP32, as its
// directions are stored in FP32.
template <typename R, typename OutR, bool SPP = false>
__device__ void finish_ray(const Params& p, const Ray<R>& r, const Hit<R>& hit,
                           SppAcc* acc = nullptr) {
  using T = OutR;
  const SceneK& s = p.s;
  const unsigned fl = hit.flags & 0xFFu;
  const unsigned flags = hit.flags | (r.aux & 0xFFu);
  float c[3] = {0.0f, 0.0f, 0.0f};
  if (fl == BH_FLAG_CAPT || fl == BH_FLAG_STEP_LIMIT) {
    emit_ray<OutR, SPP>(p, r.out, OutR(NAN), OutR(NAN), flags, c, acc);
    return;
  }
  R phr = hit.phi;
  if (sizeof(T) < sizeof(R)) phr -= Num<R>::two_pi * m_floor(phr * R(0.15915494309189535));
  T sp, cp;
  m_sincos_mapback(T(phr), &sp, &cp);
  const T e1x = T(r.e1x), e1y = T(r.e1y), e1z = T(r.e1z);
  const T e2x = T(r.e2x), e2y = T(r.e2y), e2z = T(r.e2z);
  const T dx = cp * e1x + sp * e2x;
  const T dy = cp * e1y + sp * e2y;
  const T dz = cp * e1z + sp * e2z;
  T th, ph;
  dir_angles(dx, dy, dz, &th, &ph);
  if (fl == BH_FLAG_ESC) {
    if (s.sky_tex)
      sky_image_rgb<T>(s, th, ph, c);
    else
      sky_rgb<T>(s, th, ph, c);
  } else if (fl == BH_FLAG_DISK) {
    const float rr = (float)m_quot(R(1), hit.u);
    float t = ex2_approx(0.75f * lg2_approx(s.f.r_in * rcp_approx(rr)));
    float bright = 1.0f;
    if (p.doppler) {
      const float g = disk_shift(p, r, (float)hit.u, (float)hit.v);
      t *= g;
      bright = g * g * g;
    }
    const float k = fmaf(0.7f, t, 0.3f) * bright;
    c[0] = k;
    c[1] = fmaf(0.65f, t, 0.35f) * k;
    c[2] = fmaf(0.9f * t, t, 0.1f) * k;
  } else {  // sphere
    const int id = (int)(hit.flags >> 8);
    const T u = T(hit.u), v = T(hit.v);
    const T iu = T(1) / u;
    // tangent d x/d phi scaled by u^2
    const T T0 = u * (-sp * e1x + cp * e2x) - v * dx, T1 = u * (-sp * e1y + cp * e2y) - v * dy,
            T2 = u * (-sp * e1z + cp * e2z) - v * dz;
    const T it = T(1) / m_sqrt(T0 * T0 + T1 * T1 + T2 * T2);
    const SceneR<T>& S = SR<T>(s);
    const T iR = T(1) / S.rad[id];
    const T N0 = (dx * iu - S.c[id][0]) * iR, N1 = (dy * iu - S.c[id][1]) * iR,
            N2 = (dz * iu - S.c[id][2]) * iR;
    const float ndt = (float)(-(N0 * T0 + N1 * T1 + N2 * T2) * it);
    const float lam = 0.25f + 0.75f * fmaxf(0.0f, ndt);
    c[0] = s.alb[id][0] * lam;
    c[1] = s.alb[id][1] * lam;
    c[2] = s.alb[id][2] * lam;
  }
  emit_ray<OutR, SPP>(p, r.out, th, ph, flags, c, acc);
}

}  // namespace bhk
