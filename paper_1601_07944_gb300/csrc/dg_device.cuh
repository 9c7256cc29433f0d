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

// points of the fully symmetric volume rule of degree 2p (p = 1..5)
__host__ __device__ constexpr int sym_points(int p) {
  return p == 1 ? 3 : p == 2 ? 6 : p == 3 ? 12 : p == 4 ? 16 : 25;
}

// Q = 0: the collapsed (p+1)^2 grid; Q > 0: a rule of Q points (the symmetric one)
template <int P, int NE, int Q = 0>
struct Cfg {
  static constexpr int NP = (P + 1) * (P + 2) / 2;
  static constexpr int ND = P + 1;
  static constexpr int NQ = Q > 0 ? Q : ND * ND;
  static constexpr int NF = 3 * NE;
  static constexpr int EB = P <= 1 ? 64 : (P <= 3 ? 32 : 16);   // elements per tile
  static constexpr int TAB = NP * NQ * 3 + NF * NP * 2;          // direct tables, doubles
};

constexpr int kThreads = 256;

// Edge traces of one variable at edge point k of the three reference faces,
// factorised on the collapsed coordinates (face 0: alpha = xi, beta = -1;
// face 1: alpha = 1, beta = xi; face 2: alpha = -1, beta = -xi):
//   t0 = T0_k = sum_a P_a(xi_k) Z_a,  Z_a = sum_b chi_ab(-1) c_ab,
//   t1 = T1_k = sum_a Y_a(xi_k),  t2 = T2_{NE-1-k} = sum_a (-1)^a Y_a(xi_k),
//   Y_a(xi) = sum_b chi_ab(xi) c_ab,
// with t1 = E + O and t2 = E - O formed from the sums over the modes of even and
// of odd first index, E = sum_{a even} Y_a and O = sum_{a odd} Y_a (one FMA per
// mode into one of two accumulators, then two additions).
// face0_z forms the Z_a of a coefficient set (they do not depend on k);
// edge_traces_sf takes them with cj, the N_p coefficients; ePa = P_a(xi_k)
// [ND][NE], eChi = chi_j(xi_k) [N_p][NE], eChiM1 = chi_j(-1) [N_p].  Every kernel
// that writes traces goes through these two (or through face_sums and
// edge_traces_unit below, which give the same values), in this order of
// operations, so traces of the same state agree bit for bit whichever kernel
// wrote them.
template <int P>
__device__ __forceinline__ void face0_z(const double *cj, const double *eChiM1, double z[P + 1]) {
#pragma unroll
  for (int a = 0; a <= P; ++a) z[a] = 0.0;
#pragma unroll
  for (int d = 0; d <= P; ++d)
#pragma unroll
    for (int b = 0; b <= d; ++b) {
      const int j = d * (d + 1) / 2 + b;
      z[d - b] = fma(eChiM1[j], cj[j], z[d - b]);
    }
}

template <int P, int NE>
__device__ __forceinline__ void edge_traces_sf(const double *cj, const double *z, const double *ePa,
                                               const double *eChi, int k, double &t0, double &t1, double &t2) {
  double ev = 0.0, od = 0.0;
  t0 = 0.0;
#pragma unroll
  for (int a = 0; a <= P; ++a) t0 = fma(ePa[a * NE + k], z[a], t0);
#pragma unroll
  for (int d = 0; d <= P; ++d)
#pragma unroll
    for (int b = 0; b <= d; ++b) {
      const int j = d * (d + 1) / 2 + b;
      const double cv = cj[j];
      if ((d - b) & 1) od = fma(eChi[j * NE + k], cv, od);
      else ev = fma(eChi[j * NE + k], cv, ev);
    }
  t1 = ev + od;
  t2 = ev - od;
}

// The same traces from the unweighted tables, in 2 n_e - 1 fewer float64
// operations per (element, variable): P_0 = 1, so T0_k starts from Z_0; and
// chi_00 does not depend on the edge point, so the constant mode's term
// chi_00 c_00 of faces 1 and 2 is formed once (face_sums puts it in z[P+1]).
// The values are those of edge_traces_sf on the same tables: fma(1, Z_0, 0) is
// Z_0, and chi_00 c_00 is the same rounded product.  (The weighted tables of the
// adjoint's transposed lift have neither property: edge_traces_sf serves them.)
template <int P>
__device__ __forceinline__ void face_sums(const double *cj, const double *eChiM1, double chi00, double z[P + 2]) {
  face0_z<P>(cj, eChiM1, z);
  z[P + 1] = chi00 * cj[0];
}

template <int P, int NE>
__device__ __forceinline__ void edge_traces_unit(const double *cj, const double *z, const double *ePa,
                                                 const double *eChi, int k, double &t0, double &t1, double &t2) {
  double ev = z[P + 1], od = 0.0;
  t0 = z[0];
#pragma unroll
  for (int a = 1; a <= P; ++a) t0 = fma(ePa[a * NE + k], z[a], t0);
#pragma unroll
  for (int d = 1; d <= P; ++d)
#pragma unroll
    for (int b = 0; b <= d; ++b) {
      const int j = d * (d + 1) / 2 + b;
      const double cv = cj[j];
      if ((d - b) & 1) od = fma(eChi[j * NE + k], cv, od);
      else ev = fma(eChi[j * NE + k], cv, ev);
    }
  t1 = ev + od;
  t2 = ev - od;
}

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

// x > 0 and finite, tested on the bit pattern with integer instructions (a float64
// compare would take a slot of the narrow float64 pipe)
__device__ __forceinline__ bool positive_finite(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  return hi < 0x7FF00000u && (hi | lo) != 0u;      // sign clear, exponent not all ones, not zero
}

// sqrt(x) for a finite x >= 0 in float64 by Newton-Raphson (Heron) refinement of
// a float32 estimate r of 1/sqrt(x) (rsqrt.approx.ftz.f32 on x rounded to
// float32): y = x r, then twice y <- y + (x - y^2) r / 2.  The estimate is good to
// about 2^-22; the first step leaves a relative error of about 1.5 (2^-22)^2, the
// second one of about its cube, below float64 rounding (dg_self_test checks the
// result against the correctly rounded square root: at most 1 ulp apart).  Five
// float64 operations.  x below the float32 normal range gives 0; x < 0 gives NaN.
__device__ __forceinline__ double sqrt_nr(double x) {
  const float xf = f64_to_f32_dev(x);
  float rf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  if (xf == 0.0f) rf = 0.0f;
  const double r = f32_to_f64_dev(rf), hr = f32_to_f64_dev(0.5f * rf);
  double y = x * r;
  y = fma(fma(-y, y, x), hr, y);
  return fma(fma(-y, y, x), hr, y);
}

// max(a, b) of two non-negative float64 values on their bit patterns (integer
// order equals numeric order there); a NaN with the sign bit clear wins.
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}

// Local Lax-Friedrichs flux times the edge's half length l (Eq. len), at one edge
// point, float64 throughout:
//   out = l F_hat = h (F(Ul).n + F(Ur).n - alpha (Ur - Ul)),  h = l / 2,
//   alpha = max(|v_l.n| + c_l, |v_r.n| + c_r),  c = sqrt(gamma p / rho).
// The scaled normal s = h n of the face record is folded into the physical
// fluxes: with w = s.(rho u) / rho = h v.n and P = E - |rho u|^2 / (2 rho) =
// p / (gamma - 1),
//   h F(U).n = (rho w, mx w + P (gamma-1) s_x, my w + P (gamma-1) s_y, (E + (gamma-1) P) w),
//   h alpha = max(|w_l| + h c_l, |w_r| + h c_r),  h c = sqrt(hk P / rho).
// The dissipation term moves into the normal velocities, wa = w_l + h alpha and
// wb = w_r - h alpha, so that
//   l F_hat = (rho_l wa + rho_r wb,
//              mx_l wa + mx_r wb + (P_l + P_r) (gamma-1) s_x,
//              my_l wa + my_r wb + (P_l + P_r) (gamma-1) s_y,
//              E_l wa + E_r wb + (gamma-1) (P_l w_l + P_r w_r))
// (about 56 float64 operations per point).  The square roots of the sound speeds
// are sqrt_nr; the larger wave speed is picked on the bit patterns.
// Returns false if either side is non-physical (rho <= 0 or p <= 0, or NaN).
__device__ __forceinline__ bool lax_friedrichs_edge(const double ul[M], const double ur[M], const FaceGeo &g,
                                                    double gamma, double out[M]) {
  const double g1 = gamma - 1.0;
  const double il = recip(ul[0]), ir = recip(ur[0]);
  const double wL = fma(ul[1], g.sx, ul[2] * g.sy) * il, wR = fma(ur[1], g.sx, ur[2] * g.sy) * ir;
  const double PL = fma(-0.5 * fma(ul[1], ul[1], ul[2] * ul[2]), il, ul[3]);
  const double PR = fma(-0.5 * fma(ur[1], ur[1], ur[2] * ur[2]), ir, ur[3]);
  const double aL = fabs(wL) + sqrt_nr(g.hk * PL * il);
  const double aR = fabs(wR) + sqrt_nr(g.hk * PR * ir);
  const double la = max_nonneg(aL, aR);
  const double wa = wL + la, wb = wR - la, Ps = PL + PR;
  out[0] = fma(ul[0], wa, ur[0] * wb);
  out[1] = fma(ul[1], wa, fma(ur[1], wb, Ps * g.gsx));
  out[2] = fma(ul[2], wa, fma(ur[2], wb, Ps * g.gsy));
  out[3] = fma(ul[3], wa, fma(ur[3], wb, g1 * fma(PL, wL, PR * wR)));
  return positive_finite(ul[0]) & positive_finite(ur[0]) & positive_finite(PL) & positive_finite(PR);
}

// lax_friedrichs_edge for two float32 traces (an interior face of the mixed
// modes: the values widen exactly), with two float64 operations fewer per point:
// one reciprocal serves both sides (1/rho_l = rho_r / (rho_l rho_r), the product
// of two float32 values being exact in float64), and |rho u|^2 / 2 is formed
// from the momenta halved in float32 (exact) instead of a multiply by 1/2.
__device__ __forceinline__ bool lax_friedrichs_edge_f32(const float4 a, const float4 b, const FaceGeo &g,
                                                        double gamma, double out[M]) {
  const double g1 = gamma - 1.0;
  const double ul[M] = {f32_to_f64_dev(a.x), f32_to_f64_dev(a.y), f32_to_f64_dev(a.z), f32_to_f64_dev(a.w)};
  const double ur[M] = {f32_to_f64_dev(b.x), f32_to_f64_dev(b.y), f32_to_f64_dev(b.z), f32_to_f64_dev(b.w)};
  const double hxL = f32_to_f64_dev(0.5f * a.y), hyL = f32_to_f64_dev(0.5f * a.z);
  const double hxR = f32_to_f64_dev(0.5f * b.y), hyR = f32_to_f64_dev(0.5f * b.z);
  const double ilr = recip(ul[0] * ur[0]);
  const double il = ur[0] * ilr, ir = ul[0] * ilr;
  const double wL = fma(ul[1], g.sx, ul[2] * g.sy) * il, wR = fma(ur[1], g.sx, ur[2] * g.sy) * ir;
  const double PL = fma(-fma(hxL, ul[1], hyL * ul[2]), il, ul[3]);
  const double PR = fma(-fma(hxR, ur[1], hyR * ur[2]), ir, ur[3]);
  const double aL = fabs(wL) + sqrt_nr(g.hk * PL * il);
  const double aR = fabs(wR) + sqrt_nr(g.hk * PR * ir);
  const double la = max_nonneg(aL, aR);
  const double wa = wL + la, wb = wR - la, Ps = PL + PR;
  out[0] = fma(ul[0], wa, ur[0] * wb);
  out[1] = fma(ul[1], wa, fma(ur[1], wb, Ps * g.gsx));
  out[2] = fma(ul[2], wa, fma(ur[2], wb, Ps * g.gsy));
  out[3] = fma(ul[3], wa, fma(ur[3], wb, g1 * fma(PL, wL, PR * wR)));
  return positive_finite(ul[0]) & positive_finite(ur[0]) & positive_finite(PL) & positive_finite(PR);
}

// Ghost state at a point of a boundary face (Algorithm 2: it takes the right
// trace's place in the numerical flux).  A solid wall (DG_BC_WALL) mirrors the
// momentum in the wall, U_g = (rho, m - 2 (m.n) n, E), with n the unit outward
// normal; a prescribed boundary (DG_BC_STATE) takes the caller's state ub there.
__device__ __forceinline__ void ghost_state(int code, const double ul[M], double nx, double ny,
                                            const double *ub, double ug[M]) {
  if (code == DG_BC_WALL) {
    const double mn2 = 2.0 * fma(ul[1], nx, ul[2] * ny);
    ug[0] = ul[0];
    ug[1] = fma(-mn2, nx, ul[1]);
    ug[2] = fma(-mn2, ny, ul[2]);
    ug[3] = ul[3];
  } else {
#pragma unroll
    for (int m = 0; m < M; ++m) ug[m] = ub[m];
  }
}

// The edge flux of one stage, float64: fhat[f][k][m] = l_f F_hat(U_l(r_{L,k}),
// U_r(r_{R,NE-1-k}), n_f) for every (edge, point) item; block `block` of
// `nblocks` takes the block-th equal slice of the items, so that a grid of what
// is resident at once gives every SM the same share (k_face, and the edge phase
// of the fused small-mesh stepper).
template <int NE>
__device__ __forceinline__ void face_flux_points(const double *__restrict__ trace, double *__restrict__ fhat,
                                                 const FaceConn *__restrict__ conn, const FaceGeo *__restrict__ fg,
                                                 const double *__restrict__ bstate, int64_t N, int64_t F,
                                                 double gamma, int *err, int block, int nblocks);

// device error flag bits (read by dg_device_status)
constexpr int kErrTimeout = 1;      // a bounded tensor-core wait expired
constexpr int kErrNonPhysical = 2;  // rho <= 0 or p <= 0 met at a quadrature point
constexpr int kErrIndex = 4;        // (DG_DEBUG builds) a connectivity index was out of range

// An index read from the mesh's connectivity (an element, a face, a local face).
// DG_DEBUG builds check it against [0, n) before it is used: outside, the flag
// kErrIndex is set and 0 is returned, so the access stays in bounds (a stand-in
// for a memory checker).  Other builds return i unchanged.
__device__ __forceinline__ int64_t checked(int64_t i, int64_t n, int *err) {
#ifdef DG_DEBUG
  if (i < 0 || i >= n) {
    atomicOr(err, kErrIndex);
    return 0;
  }
#else
  (void)n; (void)err;
#endif
  return i;
}

template <int NE>
__device__ __forceinline__ void face_flux_points(const double *__restrict__ trace, double *__restrict__ fhat,
                                                 const FaceConn *__restrict__ conn, const FaceGeo *__restrict__ fg,
                                                 const double *__restrict__ bstate, int64_t N, int64_t F,
                                                 double gamma, int *err, int block, int nblocks) {
  constexpr int NF = 3 * NE;
  bool ok = true;
  const int64_t n = F * NE;
  const int64_t lo = n * block / nblocks, hi = n * (block + 1) / nblocks;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int64_t f = i / NE;
    const int k = (int)(i - f * NE);
    const FaceConn cn = conn[f];
    const FaceGeo g = fg[f];
    const double *pl = trace + ((size_t)checked(cn.l, N, err) * NF + checked(cn.L, 3, err) * NE + k) * M;
    double ul[M], ur[M], Fh[M];
#pragma unroll
    for (int m = 0; m < M; ++m) ul[m] = pl[m];
    if (cn.r < 0) {
      // boundary face (the first faces of the list): the ghost state at the same point
      ghost_state(cn.r, ul, g.nx, g.ny, bstate + ((size_t)f * NE + k) * M, ur);
    } else {
      const double *pr =
          trace + ((size_t)checked(cn.r, N, err) * NF + checked(cn.R, 3, err) * NE + (NE - 1 - k)) * M;
#pragma unroll
      for (int m = 0; m < M; ++m) ur[m] = pr[m];
    }
    // l * F_hat = (l/2) (F(Ul).n + F(Ur).n - alpha (Ur - Ul))
    ok &= lax_friedrichs_edge(ul, ur, g, gamma, Fh);
    double *dst = fhat + (size_t)i * M;
#pragma unroll
    for (int m = 0; m < M; ++m) dst[m] = Fh[m];
  }
  if (!ok) atomicOr(err, kErrNonPhysical);
}

// 1/sqrt(x) for a finite x > 0 in float64: Newton-Raphson refinement of a float32
// estimate r (rsqrt.approx.ftz.f32 on x rounded to float32), twice
// r <- r + r (1/2 - (x/2) r^2); the estimate is good to about 2^-22 and each step
// squares the relative error (dg_self_test checks the result against
// 1 / sqrt(x): at most 1 ulp apart).  Seven float64 operations.
__device__ __forceinline__ double rsqrt_nr(double x) {
  const float xf = f64_to_f32_dev(x);
  float rf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  double r = f32_to_f64_dev(rf);
  const double h = 0.5 * x;
  r = fma(r, fma(-h * r, r, 0.5), r);
  return fma(r, fma(-h * r, r, 0.5), r);
}

// x with the sign of s applied, and 0 where s is zero (d|s|/ds times x with
// sign(0) = 0), on the bit patterns
__device__ __forceinline__ double sign_times(double s, double x) {
  const int hi = __double2hiint(s), lo = __double2loint(s);
  const bool zero = ((hi & 0x7FFFFFFF) | lo) == 0;
  const double y = __hiloint2double(__double2hiint(x) ^ (hi & (int)0x80000000), __double2loint(x));
  return zero ? 0.0 : y;
}

// The quantities of one Euler state that the transposed flux and wave-speed
// Jacobians share: 1/rho, velocity (u, v), |v|^2, pressure p, E + p, v.n.
struct EulerSide {
  double inv, u, v, q2, p, H, vn;
};
__device__ __forceinline__ EulerSide euler_side(const double U[M], double nx, double ny, double g1) {
  EulerSide s;
  s.inv = recip(U[0]);
  s.u = U[1] * s.inv;
  s.v = U[2] * s.inv;
  s.q2 = fma(s.u, s.u, s.v * s.v);
  s.p = g1 * fma(-0.5 * U[0], s.q2, U[3]);
  s.H = U[3] + s.p;
  s.vn = fma(s.u, nx, s.v * ny);
  return s;
}

// out = (d(F(U).n)/dU)^T b for the Euler flux F.n = (rho vn, mx vn + p nx,
// my vn + p ny, (E+p) vn), using d vn/dU = (-vn, nx, ny, 0)/rho and
// dp/dU = (gamma-1) (|v|^2/2, -u, -v, 1):
//   sig = (b1 mx + b2 my + b3 (E+p)) / rho,  tau = (gamma-1) (b1 nx + b2 ny + b3 vn),
//   out = (-sig vn + tau |v|^2 / 2, b0 nx + b1 vn + sig nx - tau u,
//          b0 ny + b2 vn + sig ny - tau v, b3 vn + tau).
__device__ __forceinline__ void flux_jac_t(const double U[M], const EulerSide &s, double nx, double ny, double g1,
                                           const double b[M], double out[M]) {
  const double sig = fma(b[1], U[1], fma(b[2], U[2], b[3] * s.H)) * s.inv;
  const double tau = g1 * fma(b[1], nx, fma(b[2], ny, b[3] * s.vn));
  out[0] = fma(0.5 * tau, s.q2, -sig * s.vn);
  out[1] = fma(b[0], nx, fma(b[1], s.vn, fma(sig, nx, -tau * s.u)));
  out[2] = fma(b[0], ny, fma(b[2], s.vn, fma(sig, ny, -tau * s.v)));
  out[3] = fma(b[3], s.vn, tau);
}

// The volume term's pull-back at a point: out = A_x(U)^T bx + A_y(U)^T by for the
// Jacobians A_x, A_y of the two Euler fluxes (flux_jac_t with n = (1, 0) and
// (0, 1), the shared terms formed once):
//   out = (T |v|^2/2 - sx u - sy v, bx0 + sx + (bx1 - T) u + by1 v,
//          by0 + sy + bx2 u + (by2 - T) v, bx3 u + by3 v + T)
// with sx = bx1 u + bx2 v + bx3 h, sy alike with by, h = (E+p) / rho the
// enthalpy, T = (gamma-1) (bx1 + bx3 u + by2 + by3 v).
__device__ __forceinline__ void flux_jac_t_xy(const double U[M], double gamma, const double bx[M],
                                              const double by[M], double out[M]) {
  const double g1 = gamma - 1.0;
  const double inv = recip(U[0]);
  const double u = U[1] * inv, v = U[2] * inv;
  const double q2 = fma(u, u, v * v);
  const double h = fma(g1, fma(-0.5 * U[0], q2, U[3]), U[3]) * inv;
  const double sx = fma(bx[1], u, fma(bx[2], v, bx[3] * h));
  const double sy = fma(by[1], u, fma(by[2], v, by[3] * h));
  const double T = g1 * (fma(bx[3], u, bx[1]) + fma(by[3], v, by[2]));
  out[0] = fma(0.5 * T, q2, -fma(sx, u, sy * v));
  out[1] = fma(bx[1] - T, u, fma(by[1], v, bx[0] + sx));
  out[2] = fma(by[2] - T, v, fma(bx[2], u, by[0] + sy));
  out[3] = fma(bx[3], u, fma(by[3], v, T));
}

// Wave speed s = |v.n| + c of a state and, when ds is not null, its gradient
// (d|x|/dx = sign(x), sign(0) = 0):  dc = k (dp - p/rho drho), k = gamma / (2 c rho).
__device__ __forceinline__ double wave_speed(const EulerSide &s, double gamma, double &rc) {
  const double x = gamma * s.p * s.inv;          // c^2
  rc = rsqrt_nr(x);                              // 1/c
  return fabs(s.vn) + x * rc;
}
__device__ __forceinline__ void wave_speed_grad(const EulerSide &s, double rc, double nx, double ny, double gamma,
                                                double ds[M]) {
  const double g1 = gamma - 1.0;
  const double k = (0.5 * gamma) * s.inv * rc;
  const double kg = k * g1;
  ds[0] = sign_times(s.vn, -s.vn * s.inv) + k * fma(0.5 * g1, s.q2, -s.p * s.inv);
  ds[1] = fma(-kg, s.u, sign_times(s.vn, nx * s.inv));
  ds[2] = fma(-kg, s.v, sign_times(s.vn, ny * s.inv));
  ds[3] = kg;
}

// Transposed Lax-Friedrichs Jacobians applied to a cotangent fb:
//   gl = (dF_hat/dUl)^T fb,  gr = (dF_hat/dUr)^T fb,
// dF_hat/dUl = A(Ul)/2 + alpha/2 I - (Ur-Ul)/2 (x) d alpha/dUl, and alike for Ur;
// d alpha follows the larger wave speed, the left one at a tie (the speeds are
// compared on their bit patterns: both are >= 0).
__device__ __forceinline__ void lax_friedrichs_vjp(const double ul[M], const double ur[M], double nx,
                                                   double ny, double gamma, const double fb[M],
                                                   double gl[M], double gr[M]) {
  const double g1 = gamma - 1.0;
  const EulerSide Sl = euler_side(ul, nx, ny, g1), Sr = euler_side(ur, nx, ny, g1);
  double rcl, rcr;
  const double sl = wave_speed(Sl, gamma, rcl), sr = wave_speed(Sr, gamma, rcr);
  const bool left = __double_as_longlong(sl) >= __double_as_longlong(sr);
  const double a = left ? sl : sr;
  double ds[M];
  wave_speed_grad(left ? Sl : Sr, left ? rcl : rcr, nx, ny, gamma, ds);
  double jump = (ur[0] - ul[0]) * fb[0];
#pragma unroll
  for (int m = 1; m < M; ++m) jump = fma(ur[m] - ul[m], fb[m], jump);
  double jl[M], jr[M];
  flux_jac_t(ul, Sl, nx, ny, g1, fb, jl);
  flux_jac_t(ur, Sr, nx, ny, g1, fb, jr);
  const double ha = 0.5 * a, hj = 0.5 * jump;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const double t = hj * ds[m];
    gl[m] = fma(0.5, jl[m], fma(ha, fb[m], left ? -t : 0.0));
    gr[m] = fma(0.5, jr[m], fma(-ha, fb[m], left ? 0.0 : -t));
  }
}

}  // namespace dg
