/*
 * dg_device.cuh -- device helpers shared by the forward and adjoint kernels:
 * compile-time sizes of a discretisation, the Euler flux in reference form, the
 * local Lax-Friedrichs flux and the transposed Jacobian products used by the
 * discrete adjoint.
 */
#pragma once

#include <cuda_runtime.h>

#include "dg_internal.h"
#include "dg_tcgen05.cuh"

namespace dg {

__device__ __forceinline__ float f64_to_f32_dev(double x) { return tc::f64_to_f32(x); }
__device__ __forceinline__ double f32_to_f64_dev(float f) { return tc::f32_to_f64(f); }

template <int P, int NE>
struct Cfg {
  static constexpr int NP = (P + 1) * (P + 2) / 2;
  static constexpr int ND = P + 1;
  static constexpr int NQ = ND * ND;
  static constexpr int NF = 3 * NE;
  static constexpr int EB = P <= 1 ? 64 : (P <= 3 ? 32 : 16);   // elements per tile
  static constexpr int TAB = NP * NQ * 3 + NF * NP * 2;          // direct tables, doubles
};

constexpr int kThreads = 256;

// 1/x for a positive normal x: Newton-Raphson refinement r <- r + r (1 - x r) of
// the hardware's approximate float64 reciprocal (rcp.approx.ftz.f64); each step
// doubles the number of correct bits, two steps reach double precision
// (checked against 1/x by dg_self_test).
__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}


// Local Lax-Friedrichs flux, scaled: out = h (F(Ul).n + F(Ur).n - alpha (Ur - Ul)),
// alpha = max(|v_l.n| + c_l, |v_r.n| + c_r).  With h = l/2 this is l F_hat.
// FAST_ALPHA (mixed-precision modes only): alpha, a dissipation coefficient, is
// formed in float32 from the float64 pressure, density and normal velocity; the
// flux itself stays float64.
// x > 0 and finite, tested on the bit pattern with integer instructions (a float64
// compare would take a slot of the narrow float64 pipe)
__device__ __forceinline__ bool positive_finite(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  return hi < 0x7FF00000u && (hi | lo) != 0u;      // sign clear, exponent not all ones, not zero
}

// Returns false if either trace is non-physical (rho <= 0 or p <= 0, or NaN).
template <bool FAST_ALPHA = false>
__device__ __forceinline__ bool lax_friedrichs_scaled(const double ul[M], const double ur[M], double nx,
                                                      double ny, double gamma, double h, double out[M]) {
  const double il = recip(ul[0]), ir = recip(ur[0]);
  const double uL = ul[1] * il, vL = ul[2] * il, uR = ur[1] * ir, vR = ur[2] * ir;
  const double pL = (gamma - 1.0) * (ul[3] - 0.5 * (ul[1] * uL + ul[2] * vL));
  const double pR = (gamma - 1.0) * (ur[3] - 0.5 * (ur[1] * uR + ur[2] * vR));
  const double vnL = uL * nx + vL * ny, vnR = uR * nx + vR * ny;
  double a;
  if (FAST_ALPHA) {
    const float g = (float)gamma;
    const float sL = fabsf(f64_to_f32_dev(vnL)) + sqrtf(g * f64_to_f32_dev(pL) * f64_to_f32_dev(il));
    const float sR = fabsf(f64_to_f32_dev(vnR)) + sqrtf(g * f64_to_f32_dev(pR) * f64_to_f32_dev(ir));
    a = f32_to_f64_dev(fmaxf(sL, sR));
  } else {
    const double sL = fabs(vnL) + sqrt(gamma * pL * il);
    const double sR = fabs(vnR) + sqrt(gamma * pR * ir);
    a = fmax(sL, sR);
  }
  double fL[M], fR[M];
  fL[0] = ul[0] * vnL;              fR[0] = ur[0] * vnR;
  fL[1] = ul[1] * vnL + pL * nx;    fR[1] = ur[1] * vnR + pR * nx;
  fL[2] = ul[2] * vnL + pL * ny;    fR[2] = ur[2] * vnR + pR * ny;
  fL[3] = (ul[3] + pL) * vnL;       fR[3] = (ur[3] + pR) * vnR;
#pragma unroll
  for (int m = 0; m < M; ++m) out[m] = h * fma(-a, ur[m] - ul[m], fL[m] + fR[m]);
  return positive_finite(ul[0]) & positive_finite(ur[0]) & positive_finite(pL) & positive_finite(pR);
}

// device error flag bits (read by dg_device_status)
constexpr int kErrTimeout = 1;      // a bounded tensor-core wait expired
constexpr int kErrNonPhysical = 2;  // rho <= 0 or p <= 0 met at a quadrature point

// out = (d(F(U).n)/dU)^T b for the Euler flux F.n = (rho vn, mx vn + p nx,
// my vn + p ny, (E+p) vn), using d vn/dU = (-vn, nx, ny, 0)/rho and
// dp/dU = (gamma-1) (|v|^2/2, -u, -v, 1).
__device__ __forceinline__ void flux_jac_t(const double U[M], double nx, double ny, double gamma,
                                           const double b[M], double out[M]) {
  const double inv = recip(U[0]);
  const double u = U[1] * inv, v = U[2] * inv;
  const double q2 = u * u + v * v;
  const double p = (gamma - 1.0) * (U[3] - 0.5 * U[0] * q2);
  const double vn = u * nx + v * ny;
  const double sig = (b[1] * U[1] + b[2] * U[2] + b[3] * (U[3] + p)) * inv;
  const double tau = (gamma - 1.0) * (b[1] * nx + b[2] * ny + b[3] * vn);
  out[0] = -sig * vn + 0.5 * tau * q2;
  out[1] = b[0] * nx + b[1] * vn + sig * nx - tau * u;
  out[2] = b[0] * ny + b[2] * vn + sig * ny - tau * v;
  out[3] = b[3] * vn + tau;
}

// Wave speed s = |v.n| + c and its gradient (d|x|/dx = sign(x), sign(0) = 0).
__device__ __forceinline__ double wave_speed_grad(const double U[M], double nx, double ny,
                                                  double gamma, double ds[M]) {
  const double inv = recip(U[0]);
  const double u = U[1] * inv, v = U[2] * inv;
  const double q2 = u * u + v * v;
  const double p = (gamma - 1.0) * (U[3] - 0.5 * U[0] * q2);
  const double vn = u * nx + v * ny;
  const double c = sqrt(gamma * p * inv);
  const double sg = vn > 0.0 ? 1.0 : (vn < 0.0 ? -1.0 : 0.0);
  const double k = gamma / (2.0 * c) * inv;          // dc = k (dp - p/rho drho)
  const double g1 = gamma - 1.0;
  ds[0] = sg * (-vn * inv) + k * (g1 * 0.5 * q2 - p * inv);
  ds[1] = sg * (nx * inv) + k * (-g1 * u);
  ds[2] = sg * (ny * inv) + k * (-g1 * v);
  ds[3] = k * g1;
  return fabs(vn) + c;
}

// Transposed Lax-Friedrichs Jacobians applied to a cotangent fb:
//   gl = (dF_hat/dUl)^T fb,  gr = (dF_hat/dUr)^T fb,
// dF_hat/dUl = A(Ul)/2 + alpha/2 I - (Ur-Ul)/2 (x) d alpha/dUl, and alike for Ur;
// d alpha follows the larger wave speed, the left one at a tie.
__device__ __forceinline__ void lax_friedrichs_vjp(const double ul[M], const double ur[M], double nx,
                                                   double ny, double gamma, const double fb[M],
                                                   double gl[M], double gr[M]) {
  double dsl[M], dsr[M], jl[M], jr[M];
  const double sl = wave_speed_grad(ul, nx, ny, gamma, dsl);
  const double sr = wave_speed_grad(ur, nx, ny, gamma, dsr);
  const bool left = sl >= sr;
  const double a = left ? sl : sr;
  double jump = 0.0;
#pragma unroll
  for (int m = 0; m < M; ++m) jump += (ur[m] - ul[m]) * fb[m];
  flux_jac_t(ul, nx, ny, gamma, fb, jl);
  flux_jac_t(ur, nx, ny, gamma, fb, jr);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    gl[m] = 0.5 * jl[m] + 0.5 * a * fb[m] - (left ? 0.5 * jump * dsl[m] : 0.0);
    gr[m] = 0.5 * jr[m] - 0.5 * a * fb[m] - (left ? 0.0 : 0.5 * jump * dsr[m]);
  }
}

}  // namespace dg
