/*
 * dg_adjoint.cu -- float64 discrete adjoint of the DG right-hand side on
 * sm_103a: out = (dR/du)^T lam, combined with the transposed SSP-RK3 stage
 * weights.  The forward stage (dg_kernels.cu) is
 *     traces T = B_f u,   edge flux fhat = l F_hat(T_l, T_r, n),
 *     R = (V(u) + L fhat) / det J,
 * so its transpose runs backwards through the same three pieces:
 *
 *   k_adj_element   per element: lam_bar = lam / det J;  the cotangent of the
 *                   reference flux at each volume point (transposed projection),
 *                   pulled back through J^tau and the Euler flux Jacobians and
 *                   interpolated back to modes (transposed interpolation);  the
 *                   cotangent of the lifted edge fluxes (transposed lift);  and
 *                   the traces of u that the edge pass linearises about.
 *   k_adj_face      per edge point: gathers the cotangent of fhat from the two
 *                   elements (with the same signs and reversed right-side order
 *                   as the forward gather) and applies the transposed
 *                   Lax-Friedrichs Jacobians, writing one trace cotangent per
 *                   element face point (each slot has exactly one writer); on a
 *                   boundary face through the ghost state (a wall's reflection).
 *   k_adj_combine   per element: transposed trace interpolation, plus the linear
 *                   combination of the Runge-Kutta adjoint
 *                   out = x0 X + x1 Y + x2 Z + s (dR/du)^T lam.
 *
 * On the collapsed volume grid (the default rule) the element pieces are
 * sum-factorised as the forward kernel is (k_adj_element_sf, k_adj_combine_sf):
 * every contraction with a basis table is the transpose, in reverse order, of a
 * factorised forward contraction with the same table (the collapsed grid is a
 * tensor grid and phi_j(alpha, beta) = P_a(alpha) chi_j(beta)).  The direct
 * kernels above serve the symmetric rules.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

template <int P, int NE, int Q>
struct AdjCfg {
  using C = Cfg<P, NE, Q>;
  static constexpr int TILE = C::EB * (2 * M * C::NP + C::NQ * M);
  static constexpr int SMEM = (C::TAB + TILE) * 8;
};

template <int P, int NE, int Q>
__global__ void __launch_bounds__(kThreads)
k_adj_element(const double *__restrict__ u, const double *__restrict__ lam, double *__restrict__ uvol,
              double *__restrict__ G, double *__restrict__ T, const double *__restrict__ geo,
              DevTables tab, int N, double gamma) {
  using C = Cfg<P, NE, Q>;
  constexpr int NP = C::NP, NQ = C::NQ, NF = C::NF, EB = C::EB;
  extern __shared__ double smem[];
  double *sBvT = smem;                 // [NP][NQ]
  double *sDr = sBvT + NP * NQ;        // [NQ][NP]
  double *sDs = sDr + NQ * NP;         // [NQ][NP]
  double *sLf = sDs + NQ * NP;         // [NF][NP]
  double *sBfT = sLf + NF * NP;        // [NP][NF]
  double *sC = sBfT + NP * NF;         // [EB][M][NP]  u
  double *sL = sC + EB * M * NP;       // [EB][M][NP]  lam / det J
  double *sU = sL + EB * M * NP;       // [EB][NQ][M]  cotangent of U at volume points

  for (int i = threadIdx.x; i < NP * NQ; i += blockDim.x) {
    sBvT[i] = tab.BvT[i];
    sDr[i] = tab.Dr[i];
    sDs[i] = tab.Ds[i];
  }
  for (int i = threadIdx.x; i < NF * NP; i += blockDim.x) {
    sLf[i] = tab.Lf[i];
    sBfT[i] = tab.BfT[i];
  }
  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *su = u + (size_t)e0 * M * NP;
    const double *sl = lam + (size_t)e0 * M * NP;
    for (int i = threadIdx.x; i < EB * M * NP; i += blockDim.x) {
      const bool in = i < ecount * M * NP;
      const int el = i / (M * NP);
      sC[i] = in ? su[i] : 0.0;
      sL[i] = in ? sl[i] * geo[(size_t)(e0 + el) * GEO + 4] : 0.0;
    }
    __syncthreads();

    // volume points: U, the projection transposes a_r, a_s, then J^tau^T and
    // the flux Jacobians transposed
    for (int i = threadIdx.x; i < EB * NQ; i += blockDim.x) {
      const int el = i / NQ, k = i - el * NQ;
      double U[M] = {0.0, 0.0, 0.0, 0.0}, ar[M] = {0.0, 0.0, 0.0, 0.0}, as[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const double b = sBvT[j * NQ + k], dr = sDr[k * NP + j], ds = sDs[k * NP + j];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          U[m] += sC[(el * M + m) * NP + j] * b;
          ar[m] += sL[(el * M + m) * NP + j] * dr;
          as[m] += sL[(el * M + m) * NP + j] * ds;
        }
      }
      double ub[M] = {0.0, 0.0, 0.0, 0.0};
      if (el < ecount) {
        const double *g = geo + (size_t)(e0 + el) * GEO;
        double b1[M], b2[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          b1[m] = fma(ar[m], g[0], as[m] * g[2]);
          b2[m] = fma(ar[m], g[1], as[m] * g[3]);
        }
        flux_jac_t_xy(U, gamma, b1, b2, ub);
      }
#pragma unroll
      for (int m = 0; m < M; ++m) sU[i * M + m] = ub[m];
    }
    __syncthreads();

    // modes: transposed interpolation
    for (int i = threadIdx.x; i < ecount * NP; i += blockDim.x) {
      const int el = i / NP, j = i - el * NP;
      double acc[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
      for (int k = 0; k < NQ; ++k) {
        const double b = sBvT[j * NQ + k];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] += sU[(el * NQ + k) * M + m] * b;
      }
#pragma unroll
      for (int m = 0; m < M; ++m) uvol[((size_t)(e0 + el) * M + m) * NP + j] = acc[m];
    }

    // edge points: cotangent of the lifted fluxes and the traces of u
    for (int i = threadIdx.x; i < ecount * NF; i += blockDim.x) {
      const int el = i / NF, qk = i - el * NF;
      double g[M] = {0.0, 0.0, 0.0, 0.0}, t[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const double l = sLf[qk * NP + j], b = sBfT[j * NF + qk];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          g[m] += sL[(el * M + m) * NP + j] * l;
          t[m] += sC[(el * M + m) * NP + j] * b;
        }
      }
      const size_t o = ((size_t)(e0 + el) * NF + qk) * M;
#pragma unroll
      for (int m = 0; m < M; ++m) { G[o + m] = g[m]; T[o + m] = t[m]; }
    }
  }
}

template <int NE>
__global__ void __launch_bounds__(kThreads)
k_adj_face(const double *__restrict__ T, const double *__restrict__ G, double *__restrict__ TB,
           const FaceConn *__restrict__ conn, const FaceGeo *__restrict__ fg, const double *__restrict__ bstate,
           int64_t N, int64_t F, double gamma, int *err) {
  constexpr int NF = 3 * NE;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F * NE) return;
  const int64_t f = i / NE;
  const int k = (int)(i - f * NE);
  const FaceConn cn = conn[f];
  const FaceGeo g = fg[f];
  const size_t ol = ((size_t)checked(cn.l, N, err) * NF + checked(cn.L, 3, err) * NE + k) * M;
  double ul[M], ur[M], fb[M], gl[M], gr[M];
  if (cn.r < 0) {
    // boundary face: F_hat(U_l, U_g(U_l)).  A wall's ghost is the reflection
    // U_g = Rf U_l, Rf = diag(1, I - 2 n n^T, 1) (symmetric), so the trace's
    // cotangent is gl + Rf gr; a prescribed ghost does not depend on U_l.  Only
    // the left element lifts the flux (with -1).
#pragma unroll
    for (int m = 0; m < M; ++m) ul[m] = T[ol + m];
    ghost_state(cn.r, ul, g.nx, g.ny, bstate + ((size_t)f * NE + k) * M, ur);
#pragma unroll
    for (int m = 0; m < M; ++m) fb[m] = -g.hl * G[ol + m];
    lax_friedrichs_vjp(ul, ur, g.nx, g.ny, gamma, fb, gl, gr);
    if (cn.r == DG_BC_WALL) {
      const double gn2 = 2.0 * fma(gr[1], g.nx, gr[2] * g.ny);
      gl[0] += gr[0];
      gl[1] += fma(-gn2, g.nx, gr[1]);
      gl[2] += fma(-gn2, g.ny, gr[2]);
      gl[3] += gr[3];
    }
#pragma unroll
    for (int m = 0; m < M; ++m) TB[ol + m] = gl[m];
    return;
  }
  const size_t orr = ((size_t)checked(cn.r, N, err) * NF + checked(cn.R, 3, err) * NE + (NE - 1 - k)) * M;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    ul[m] = T[ol + m];
    ur[m] = T[orr + m];
    // fhat enters the left element with -1 and the right element with +1;
    // fhat = l * F_hat
    fb[m] = g.hl * (G[orr + m] - G[ol + m]);
  }
  lax_friedrichs_vjp(ul, ur, g.nx, g.ny, gamma, fb, gl, gr);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    TB[ol + m] = gl[m];
    TB[orr + m] = gr[m];
  }
}

template <int P, int NE>
__global__ void __launch_bounds__(kThreads)
k_adj_combine(const double *__restrict__ uvol, const double *__restrict__ TB, const double *__restrict__ BfT,
              const double *X, const double *Y, const double *Z, double x0, double x1, double x2,
              double s, double *out, int N) {
  using C = Cfg<P, NE>;
  constexpr int NP = C::NP, NF = C::NF, EB = C::EB;
  __shared__ double sB[NP * NF];
  __shared__ double sT[EB * NF * M];
  for (int i = threadIdx.x; i < NP * NF; i += blockDim.x) sB[i] = BfT[i];
  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *src = TB + (size_t)e0 * NF * M;
    for (int i = threadIdx.x; i < EB * NF * M; i += blockDim.x) sT[i] = i < ecount * NF * M ? src[i] : 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < ecount * NP; i += blockDim.x) {
      const int el = i / NP, j = i - el * NP;
      double acc[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int qk = 0; qk < NF; ++qk) {
        const double b = sB[j * NF + qk];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] += sT[(el * NF + qk) * M + m] * b;
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const size_t idx = ((size_t)(e0 + el) * M + m) * NP + j;
        double v = s * (uvol[idx] + acc[m]);
        if (X) v += x0 * X[idx];
        if (Y) v += x1 * Y[idx];
        if (Z) v += x2 * Z[idx];
        out[idx] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// sum-factorised transpose on the collapsed grid
//
// Forward (k_element_sf), per variable: W(a,ib) = sum_{j: a(j)=a} chi_j(ib) c_j,
// U(ia,ib) = sum_a P_a(ia) W(a,ib); at the points Ha = G_r + half(ia) G_s,
// Hb = G_s; Xa(a,ib) = sum_ia wa P_a'(ia) Ha, Xb(a,ib) = sum_ia wa P_a(ia) Hb;
// V_j = sum_ib chiA_j(ib) Xa(a_j,ib) + dchiB_j(ib) Xb(a_j,ib).  For a cotangent
// lb = lam / det J of V the transpose is, per variable,
//   Xa~(a,ib) = sum_{j: a(j)=a} chiA_j(ib) lb_j,   Xb~(a,ib) = sum_{j: a(j)=a} dchiB_j(ib) lb_j,
//   Ha~(ia,ib) = sum_a wa P_a'(ia) Xa~(a,ib),      Hb~(ia,ib) = sum_a wa P_a(ia) Xb~(a,ib),
//   G_r~ = Ha~,  G_s~ = half(ia) Ha~ + Hb~   (the cotangents of G_r, G_s at the point),
// then through J^tau and the Euler flux Jacobians at U to ub (flux_jac_t_xy), and
// back to modes by the transposed interpolation
//   U~(a,ib) = sum_ia P_a(ia) ub(ia,ib),   uvol_j = sum_ib chi_j(ib) U~(a_j,ib).
// The edge pieces: the transposed lift is the traces of lb weighted by the edge
// weights (Lf[qk][j] = omega_k phi_j(r_qk)), formed by edge_traces_sf with the
// weighted tables; the transposed trace interpolation is the forward lift with
// the unweighted ones.
// ---------------------------------------------------------------------------
template <int P, int NE>
struct AdjSf {
  static constexpr int NP = (P + 1) * (P + 2) / 2, ND = P + 1, NQ = ND * ND, NF = 3 * NE;
  static constexpr int EB = P <= 1 ? 64 : (P <= 3 ? 32 : 16);
  static constexpr int TAB = 3 * ND * ND + 3 * NP * ND + ND + 2 * NP * NE + 2 * ND * NE + NP;
  // per element: u, lb [M][NP] each; the factorisation buffer [ND][ND][12]
  // (W, Xa~, Xb~ at (a, ib), later U~ with stride 4); ub at the points [NQ][4];
  // Z_a of u and of lb [M][ND] each
  static constexpr int XS = 12 * ND * ND;
  // p >= 2: the volume points in mirror pairs of the Gauss-Legendre nodes, the
  // transpose of the forward kernel's folding (at p = 1 it saves nothing)
  static constexpr bool PAIRS = P >= 2;
  static constexpr int TILE = EB * (2 * M * NP + XS + 4 * NQ + 2 * M * ND);
  static constexpr int SMEM = (TAB + TILE) * 8;
};

template <int P, int NE>
__global__ void __launch_bounds__(kThreads, 2)
k_adj_element_sf(const double *__restrict__ u, const double *__restrict__ lam, double *__restrict__ uvol,
                 double *__restrict__ G, double *__restrict__ T, const double *__restrict__ geo, DevTables tab, int N,
                 double gamma) {
  using A = AdjSf<P, NE>;
  constexpr int NP = A::NP, ND = A::ND, NQ = A::NQ, NF = A::NF, EB = A::EB;
  extern __shared__ double smem[];
  double *sPa = smem;                  // [ND][ND]   P_a(alpha_ia)
  double *sPaW = sPa + ND * ND;        // [ND][ND]   wa P_a
  double *sdPaW = sPaW + ND * ND;      // [ND][ND]   wa P_a'
  double *sChi = sdPaW + ND * ND;      // [NP][ND]   chi_j(beta_ib)
  double *sChiA = sChi + NP * ND;      // [NP][ND]   chi_j wb / (4 (1-s))
  double *sdChiB = sChiA + NP * ND;    // [NP][ND]   chi_j' wb / 4
  double *sHalf = sdChiB + NP * ND;    // [ND]       (1 + alpha_ia) / 2
  double *sEChi = sHalf + ND;          // [NP][NE]   chi_j(xi_k)
  double *sEWChi = sEChi + NP * NE;    // [NP][NE]   omega_k chi_j(xi_k)
  double *sEWPa = sEWChi + NP * NE;    // [ND][NE]   omega_k P_a(xi_k)
  double *sEPa = sEWPa + ND * NE;      // [ND][NE]   P_a(xi_k)
  double *sEChiM1 = sEPa + ND * NE;    // [NP]       chi_j(-1)
  double *sC = sEChiM1 + NP;           // [EB][M][NP]      u
  double *sL = sC + EB * M * NP;       // [EB][M][NP]      lam / det J
  double *sX = sL + EB * M * NP;       // [EB][ND][ND][12] W, Xa~, Xb~; then U~ [EB][ND][ND][4]
  double *sB = sX + EB * A::XS;        // [EB][NQ][4]      ub
  double *sZ = sB + EB * NQ * 4;       // [EB][M][2][ND]   Z_a of u, of lb

  for (int i = threadIdx.x; i < ND * ND; i += blockDim.x) {
    sPa[i] = tab.SPa[i]; sPaW[i] = tab.SPaW[i]; sdPaW[i] = tab.SdPaW[i];
  }
  for (int i = threadIdx.x; i < NP * ND; i += blockDim.x) {
    sChi[i] = tab.SChi[i]; sChiA[i] = tab.SChiA[i]; sdChiB[i] = tab.SdChiB[i];
  }
  for (int i = threadIdx.x; i < ND; i += blockDim.x) sHalf[i] = tab.SHalf[i];
  for (int i = threadIdx.x; i < NP * NE; i += blockDim.x) { sEChi[i] = tab.EChi[i]; sEWChi[i] = tab.EWChi[i]; }
  for (int i = threadIdx.x; i < ND * NE; i += blockDim.x) { sEWPa[i] = tab.EWPa[i]; sEPa[i] = tab.EPa[i]; }
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sEChiM1[i] = tab.EChiM1[i];

  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *su = u + (size_t)e0 * M * NP;
    const double *sl = lam + (size_t)e0 * M * NP;
    for (int i = threadIdx.x; i < EB * M * NP; i += blockDim.x) {
      const bool in = i < ecount * M * NP;
      const int el = i / (M * NP);
      sC[i] = in ? su[i] : 0.0;
      sL[i] = in ? sl[i] * geo[(size_t)(e0 + el) * GEO + 4] : 0.0;
    }
    __syncthreads();

    // W, Xa~, Xb~ at (a, ib); one item per (element, ib, variable) over all modes
    // (Xa~(0, .) is not formed: wa P_0' = 0 takes it out of Ha~)
    for (int i = threadIdx.x; i < EB * ND * M; i += blockDim.x) {
      const int el = i / (ND * M), ib = (i / M) % ND, m = i % M;
      const double *cm = sC + (el * M + m) * NP, *lm = sL + (el * M + m) * NP;
      double w[ND], xa[ND], xb[ND];
#pragma unroll
      for (int a = 0; a < ND; ++a) { w[a] = 0.0; xa[a] = 0.0; xb[a] = 0.0; }
#pragma unroll
      for (int d = 0; d <= P; ++d)
#pragma unroll
        for (int b = 0; b <= d; ++b) {
          const int j = d * (d + 1) / 2 + b, a = d - b;
          w[a] = fma(sChi[j * ND + ib], cm[j], w[a]);
          if (a > 0) xa[a] = fma(sChiA[j * ND + ib], lm[j], xa[a]);
          xb[a] = fma(sdChiB[j * ND + ib], lm[j], xb[a]);
        }
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        double *x = sX + ((el * ND + a) * ND + ib) * 12;
        x[m] = w[a];
        x[4 + m] = xa[a];
        x[8 + m] = xb[a];
      }
    }
    __syncthreads();

    // points: U, the cotangents of G_r and G_s, through J^tau and the flux
    // Jacobians to ub; one item per (element, point), or (PAIRS) one per
    // (element, ib, mirror pair ia, ia' = ND-1-ia) and then one per (element, ib)
    // for the middle node of an odd p + 1.  With P_a(-x) = (-1)^a P_a(x),
    // P_a'(-x) = (-1)^(a+1) P_a'(x) and equal weights, each of U, ha, hb at the
    // pair is S +/- A from its sums over the terms that keep (S) and flip (A)
    // their sign; the pair's slots get ub + ub' (ia) and ub - ub' (ia'), which
    // the transposed interpolation below takes.
    if constexpr (A::PAIRS) {
      constexpr int NH = ND / 2, NPAIR = EB * ND * NH, NMID = (ND & 1) ? EB * ND : 0, MID = ND / 2;
      for (int i = threadIdx.x; i < NPAIR + NMID; i += blockDim.x) {
        const bool mid = (ND & 1) && i >= NPAIR;
        const int el = mid ? (i - NPAIR) / ND : i / (ND * NH);
        const int ib = mid ? (i - NPAIR) - el * ND : (i - el * (ND * NH)) / NH;
        const int ia = mid ? MID : (i - el * (ND * NH)) - ib * NH, ia2 = ND - 1 - ia;
        const double *x0 = sX + ((el * ND) * ND + ib) * 12;
        const double pw0 = sPaW[ia];
        // S: the terms of the same sign at ia and ia' (U, hb: even a; ha: odd a)
        double SU[M], AU[M], Sa[M], Aa[M], Sb[M], Ab[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          SU[m] = x0[m];                                // P_0 = 1
          Sb[m] = pw0 * x0[8 + m];
          AU[m] = 0.0; Sa[m] = 0.0; Aa[m] = 0.0; Ab[m] = 0.0;
        }
#pragma unroll
        for (int a = 1; a < ND; ++a) {
          if (mid && (a & 1)) {
            // at alpha = 0 only the terms of P_a' (odd a) remain
            const double dpw = sdPaW[a * ND + ia];
            const double *x = sX + ((el * ND + a) * ND + ib) * 12;
#pragma unroll
            for (int m = 0; m < M; ++m) Sa[m] = a == 1 ? dpw * x[4 + m] : fma(dpw, x[4 + m], Sa[m]);
            continue;
          }
          const double pa = sPa[a * ND + ia], dpw = sdPaW[a * ND + ia], pw = sPaW[a * ND + ia];
          const double *x = sX + ((el * ND + a) * ND + ib) * 12;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            if (a & 1) {
              AU[m] = a == 1 ? pa * x[m] : fma(pa, x[m], AU[m]);
              Sa[m] = a == 1 ? dpw * x[4 + m] : fma(dpw, x[4 + m], Sa[m]);
              Ab[m] = a == 1 ? pw * x[8 + m] : fma(pw, x[8 + m], Ab[m]);
            } else {
              SU[m] = fma(pa, x[m], SU[m]);
              if (!mid) Aa[m] = a == 2 ? dpw * x[4 + m] : fma(dpw, x[4 + m], Aa[m]);
              Sb[m] = fma(pw, x[8 + m], Sb[m]);
            }
          }
        }
        double ub1[M] = {0.0, 0.0, 0.0, 0.0}, ub2[M] = {0.0, 0.0, 0.0, 0.0};
        if (el < ecount) {
          const double *g = geo + (size_t)(e0 + el) * GEO;
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            if (mid && side == 1) break;
            const double sg = side ? -1.0 : 1.0;
            double U[M], bx[M], by[M];
            // the cotangents of G_r = ha and G_s = half ha + hb pulled back
            // through J^tau, as for a single point
            const double half = sHalf[side ? ia2 : ia];
            const double dax = fma(half, g[2], g[0]), day = fma(half, g[3], g[1]);
#pragma unroll
            for (int m = 0; m < M; ++m) {
              U[m] = mid ? SU[m] : fma(sg, AU[m], SU[m]);
              const double ha = mid ? Sa[m] : fma(sg, Aa[m], Sa[m]);
              const double hb = mid ? Sb[m] : fma(sg, Ab[m], Sb[m]);
              bx[m] = fma(dax, ha, g[2] * hb);
              by[m] = fma(day, ha, g[3] * hb);
            }
            flux_jac_t_xy(U, gamma, bx, by, side ? ub2 : ub1);
          }
        }
        double *b1 = sB + ((size_t)el * NQ + ib * ND + ia) * 4;
        if (mid) {
#pragma unroll
          for (int m = 0; m < M; ++m) b1[m] = ub1[m];
        } else {
          double *b2 = sB + ((size_t)el * NQ + ib * ND + ia2) * 4;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            b1[m] = ub1[m] + ub2[m];
            b2[m] = ub1[m] - ub2[m];
          }
        }
      }
    } else {
      for (int i = threadIdx.x; i < EB * NQ; i += blockDim.x) {
        const int el = i / NQ, k = i - el * NQ, ib = k / ND, ia = k - ib * ND;
        const double *x0 = sX + ((el * ND) * ND + ib) * 12;
        double U[M], ha[M], hb[M];
        const double pw0 = sPaW[ia];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          U[m] = x0[m];                                   // P_0 = 1
          ha[m] = 0.0;
          hb[m] = pw0 * x0[8 + m];
        }
#pragma unroll
        for (int a = 1; a < ND; ++a) {
          const double pa = sPa[a * ND + ia], dpw = sdPaW[a * ND + ia], pw = sPaW[a * ND + ia];
          const double *x = sX + ((el * ND + a) * ND + ib) * 12;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            U[m] = fma(pa, x[m], U[m]);
            ha[m] = fma(dpw, x[4 + m], ha[m]);
            hb[m] = fma(pw, x[8 + m], hb[m]);
          }
        }
        double ub[M] = {0.0, 0.0, 0.0, 0.0};
        if (el < ecount) {
          // the cotangents of G_r = ha and G_s = half ha + hb pulled back through
          // J^tau: bx = g0 ha + g2 (half ha + hb) = (g0 + half g2) ha + g2 hb, by alike
          const double *g = geo + (size_t)(e0 + el) * GEO;
          const double half = sHalf[ia];
          const double dax = fma(half, g[2], g[0]), day = fma(half, g[3], g[1]);
          double bx[M], by[M];
#pragma unroll
          for (int m = 0; m < M; ++m) {
            bx[m] = fma(dax, ha[m], g[2] * hb[m]);
            by[m] = fma(day, ha[m], g[3] * hb[m]);
          }
          flux_jac_t_xy(U, gamma, bx, by, ub);
        }
        double *b = sB + (size_t)i * 4;
#pragma unroll
        for (int m = 0; m < M; ++m) b[m] = ub[m];
      }
    }
    __syncthreads();

    // U~(a, ib) = sum_ia P_a(ia) ub(ia, ib); one item per (element, ib, variable).
    // PAIRS: over the pairs' sums (even a) and differences (odd a), and the
    // middle node (even a only; P_0 = 1 makes the a = 0 sum additions)
    for (int i = threadIdx.x; i < EB * ND * M; i += blockDim.x) {
      const int el = i / (ND * M), ib = (i / M) % ND, m = i % M;
      double ut[ND];
      const double *brow = sB + ((el * NQ) + ib * ND) * 4 + m;
      if constexpr (A::PAIRS) {
        constexpr int NH = ND / 2, MID = ND / 2;
#pragma unroll
        for (int a = 0; a < ND; ++a) {
          double t = ((ND & 1) && !(a & 1)) ? (a == 0 ? brow[MID * 4] : sPa[a * ND + MID] * brow[MID * 4]) : 0.0;
#pragma unroll
          for (int ia = 0; ia < NH; ++ia) {
            const double v = brow[((a & 1) ? ND - 1 - ia : ia) * 4];
            t = a == 0 ? t + v : fma(sPa[a * ND + ia], v, t);
          }
          ut[a] = t;
        }
      } else {
#pragma unroll
        for (int a = 0; a < ND; ++a) ut[a] = 0.0;
#pragma unroll
        for (int ia = 0; ia < ND; ++ia) {
          const double b = brow[ia * 4];
          ut[0] += b;
#pragma unroll
          for (int a = 1; a < ND; ++a) ut[a] = fma(sPa[a * ND + ia], b, ut[a]);
        }
      }
#pragma unroll
      for (int a = 0; a < ND; ++a) sX[((el * ND + a) * ND + ib) * 4 + m] = ut[a];
    }
    // Z_a of u and of lb (face 0 lies on beta = -1), one item per (element, variable)
    for (int i = threadIdx.x; i < EB * M; i += blockDim.x) {
      double z[ND];
      face0_z<P>(sC + i * NP, sEChiM1, z);
#pragma unroll
      for (int a = 0; a < ND; ++a) sZ[i * 2 * ND + a] = z[a];
      face0_z<P>(sL + i * NP, sEChiM1, z);
#pragma unroll
      for (int a = 0; a < ND; ++a) sZ[i * 2 * ND + ND + a] = z[a];
    }
    __syncthreads();

    // modes: uvol_j = sum_ib chi_j(ib) U~(a_j, ib)
    for (int i = threadIdx.x; i < ecount * NP; i += blockDim.x) {
      const int el = i / NP, j = i - el * NP;
      int d = 0;
      while ((d + 1) * (d + 2) / 2 <= j) ++d;
      const int a = d - (j - d * (d + 1) / 2);
      double acc[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int ib = 0; ib < ND; ++ib) {
        const double ch = sChi[j * ND + ib];
        const double *x = sX + ((el * ND + a) * ND + ib) * 4;
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] = fma(ch, x[m], acc[m]);
      }
#pragma unroll
      for (int m = 0; m < M; ++m) uvol[((size_t)(e0 + el) * M + m) * NP + j] = acc[m];
    }
    // edges: traces of u (T) and the weighted traces of lb (G, the transposed
    // lift); one item per (element, variable, edge point k)
    for (int i = threadIdx.x; i < ecount * M * NE; i += blockDim.x) {
      const int el = i / (M * NE), m = (i / NE) % M, k = i % NE;
      const int em = el * M + m;
      const size_t o = (size_t)(e0 + el) * NF * M + m;
      double t0, t1, t2;
      edge_traces_sf<P, NE>(sC + em * NP, sZ + em * 2 * ND, sEPa, sEChi, k, t0, t1, t2);
      T[o + k * M] = t0;
      T[o + (NE + k) * M] = t1;
      T[o + (3 * NE - 1 - k) * M] = t2;
      edge_traces_sf<P, NE>(sL + em * NP, sZ + em * 2 * ND + ND, sEWPa, sEWChi, k, t0, t1, t2);
      G[o + k * M] = t0;
      G[o + (NE + k) * M] = t1;
      G[o + (3 * NE - 1 - k) * M] = t2;
    }
  }
}

// Transposed trace interpolation, sum-factorised (the forward lift of
// k_element_sf with the unweighted edge tables), and the Runge-Kutta adjoint's
// combination out = x0 X + x1 Y + x2 Z + s (uvol + B_f^T TB).
template <int P, int NE>
__global__ void __launch_bounds__(kThreads)
k_adj_combine_sf(const double *__restrict__ uvol, const double *__restrict__ TB, DevTables tab, const double *X,
                 const double *Y, const double *Z, double x0, double x1, double x2, double s, double *out, int N) {
  constexpr int NP = (P + 1) * (P + 2) / 2, ND = P + 1, NF = 3 * NE;
  constexpr int EB = P <= 1 ? 64 : (P <= 3 ? 32 : 16);
  constexpr int LW = ND + 2 * NE;                  // Q_a, then G_even,k, G_odd,k
  __shared__ double sEPa[ND * NE], sEChi[NP * NE], sEChiM1[NP];
  __shared__ double sW[EB * M * LW];
  for (int i = threadIdx.x; i < ND * NE; i += blockDim.x) sEPa[i] = tab.EPa[i];
  for (int i = threadIdx.x; i < NP * NE; i += blockDim.x) sEChi[i] = tab.EChi[i];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sEChiM1[i] = tab.EChiM1[i];
  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    // per (element, variable): Q_a = sum_k P_a(xi_k) TB0_k, G_even/odd,k = TB1_k +/- TB2_{NE-1-k}
    for (int i = threadIdx.x; i < ecount * M; i += blockDim.x) {
      const int el = i / M, m = i % M;
      const double *tb = TB + (size_t)(e0 + el) * NF * M + m;
      double f[NF];
#pragma unroll
      for (int x = 0; x < NF; ++x) f[x] = tb[x * M];
      double *w = sW + i * LW;
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < NE; ++k) q = fma(sEPa[a * NE + k], f[k], q);
        w[a] = q;
      }
#pragma unroll
      for (int k = 0; k < NE; ++k) {
        w[ND + k] = f[NE + k] + f[3 * NE - 1 - k];
        w[ND + NE + k] = f[NE + k] - f[3 * NE - 1 - k];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ecount * M * NP; i += blockDim.x) {
      const int em = i / NP, j = i - em * NP;
      int d = 0;
      while ((d + 1) * (d + 2) / 2 <= j) ++d;
      const int a = d - (j - d * (d + 1) / 2);
      const double *w = sW + em * LW;
      double acc = sEChiM1[j] * w[a];
      const double *g = w + ND + (a & 1) * NE;
#pragma unroll
      for (int k = 0; k < NE; ++k) acc = fma(sEChi[j * NE + k], g[k], acc);
      const size_t idx = (size_t)e0 * M * NP + i;
      double v = s * (uvol[idx] + acc);
      if (X) v = fma(x0, X[idx], v);
      if (Y) v = fma(x1, Y[idx], v);
      if (Z) v = fma(x2, Z[idx], v);
      out[idx] = v;
    }
  }
}

template <int P, int NE>
int run_adj_sf(const dg_mesh *m, const double *u, const double *lam, double *uvol, double *G, double *T, double *TB,
               const double *X, const double *Y, const double *Z, double x0, double x1, double x2, double s,
               double *out, cudaStream_t st) {
  using A = AdjSf<P, NE>;
  static PerDevice attr_set;
  if (!attr_set.test(m->device)) {
    cudaError_t e = cudaFuncSetAttribute(k_adj_element_sf<P, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, A::SMEM);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_adj_element_sf<P, NE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr_set.set(m->device);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_element_sf<P, NE>, kThreads, A::SMEM);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const int ntiles = (int)((m->N + A::EB - 1) / A::EB);
  int grid = ntiles < m->num_sms * per_sm ? ntiles : m->num_sms * per_sm;
  k_adj_element_sf<P, NE><<<grid, kThreads, A::SMEM, st>>>(u, lam, uvol, G, T, m->geo, m->tab, (int)m->N, m->gamma);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  const int64_t nf = m->F * NE;
  k_adj_face<NE><<<(int)((nf + kThreads - 1) / kThreads), kThreads, 0, st>>>(T, G, TB, m->face_conn, m->face_geo,
                                                                             m->bstate, m->N, m->F, m->gamma,
                                                                             m->err_flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  grid = ntiles < m->num_sms * 4 ? ntiles : m->num_sms * 4;
  k_adj_combine_sf<P, NE><<<grid, kThreads, 0, st>>>(uvol, TB, m->tab, X, Y, Z, x0, x1, x2, s, out, (int)m->N);
  return (int)cudaGetLastError();
}

template <int P, int NE, int Q>
int run_adj(const dg_mesh *m, const double *u, const double *lam, double *uvol, double *G, double *T,
            double *TB, const double *X, const double *Y, const double *Z, double x0, double x1, double x2,
            double s, double *out, cudaStream_t st) {
  using A = AdjCfg<P, NE, Q>;
  using C = Cfg<P, NE, Q>;
  static PerDevice attr_set;
  if (!attr_set.test(m->device)) {
    cudaError_t e = cudaFuncSetAttribute(k_adj_element<P, NE, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, A::SMEM);
    if (e != cudaSuccess) return (int)e;
    // all of the SM's unified L1/shared storage as shared memory, so that the
    // occupancy query and the launch see every CTA that fits
    e = cudaFuncSetAttribute(k_adj_element<P, NE, Q>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr_set.set(m->device);
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_element<P, NE, Q>, kThreads, A::SMEM);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const int ntiles = (int)((m->N + C::EB - 1) / C::EB);
  int grid = ntiles < m->num_sms * per_sm ? ntiles : m->num_sms * per_sm;
  k_adj_element<P, NE, Q><<<grid, kThreads, A::SMEM, st>>>(u, lam, uvol, G, T, m->geo, m->tab, (int)m->N, m->gamma);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  const int64_t nf = m->F * NE;
  k_adj_face<NE><<<(int)((nf + kThreads - 1) / kThreads), kThreads, 0, st>>>(T, G, TB, m->face_conn, m->face_geo,
                                                                             m->bstate, m->N, m->F, m->gamma,
                                                                             m->err_flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  grid = ntiles < m->num_sms * 4 ? ntiles : m->num_sms * 4;
  k_adj_combine<P, NE><<<grid, kThreads, 0, st>>>(uvol, TB, m->tab.BfT, X, Y, Z, x0, x1, x2, s, out, (int)m->N);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_rhs_vjp(const dg_mesh *m, const double *u, const double *lam, double *uvol, double *G, double *T,
                   double *TB, const double *X, const double *Y, const double *Z, double x0, double x1,
                   double x2, double s, double *out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
#define CALL(P, NE)                                                                                  \
  (m->rule == DG_RULE_SYMMETRIC                                                                      \
       ? run_adj<P, NE, sym_points(P)>(m, u, lam, uvol, G, T, TB, X, Y, Z, x0, x1, x2, s, out, st)  \
       : run_adj_sf<P, NE>(m, u, lam, uvol, G, T, TB, X, Y, Z, x0, x1, x2, s, out, st))
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaErrorInvalidValue;
}

}  // namespace dg
