/*
 * dg_element.cu -- the float64 element kernel of one stage (k_element_sf): the
 * volume integral (Eq. volume, Algorithm 1) sum-factorised on the collapsed
 * volume grid (or contracted directly on a symmetric rule of Q points), the lift
 * of the three edge fluxes (Algorithms 2-3), the 1/det J
 * scaling (Eq. 2ddg0), the Runge-Kutta stage update (with, for the classical
 * RK4, the running sum of its stages as a second output) and the next stage's
 * edge traces, for one tile of elements per CTA.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "dg_device.cuh"
#include "dg_internal.h"
#include "dg_limiter.cuh"

namespace dg {
namespace {

// ---------------------------------------------------------------------------
// element kernel, sum-factorised volume term (float64 path)
//
// The volume rule is a tensor grid in the collapsed coordinates (alpha, beta)
// and the basis factors as phi_j = P_a(alpha) chi_j(beta), so
//   interpolation  U(ia,ib) = sum_a P_a(alpha_ia) W(a,ib),  W(a,ib) = sum_{j:a(j)=a} chi_j(beta_ib) c_j
//   projection     V_j = sum_ib chiA_j(ib) Xa(a,ib) + dchiB_j(ib) Xb(a,ib),
//                  Xa(a,ib) = sum_ia wa P_a'(alpha_ia) Ha(ia,ib),  Xb(a,ib) = sum_ia wa P_a(alpha_ia) Hb(ia,ib),
// with Ha = G_r + (1+alpha)/2 G_s, Hb = G_s at the points and the weights and
// chain-rule factors of the collapsed map, d/dr = 2/(1-s) d/dalpha and
// d/ds = (1+alpha)/(1-s) d/dalpha + 2 d/dbeta, folded into the tables
// (chiA = chi wb / (4 (1-s)), dchiB = chi' wb / 4).  This is the same sum as the
// direct projection (Eq. volume), in (p+1)(N_p + (p+1)^2) instead of
// (p+1)^2 N_p products per variable for each of the two contractions.  The
// reference fluxes (G_r, G_s) = J^tau (F1, F2) are formed as the Euler flux
// along the two rows of J^tau, which are constant on the element.
// ---------------------------------------------------------------------------
//
// Q > 0 (a volume rule of Q points without tensor structure: the symmetric
// rules) contracts the volume term directly instead,
//   U(k) = sum_j phi_j(r_k) c_j,   V_j = sum_k w_k (d_r phi_j(r_k) G_r(k) + d_s phi_j(r_k) G_s(k)),
// Q N_p products per variable for each; the lift, the stage update and the
// traces are the same in both forms.
// ---------------------------------------------------------------------------
// EBX > 0 overrides the elements per tile (the fused small-mesh stepper's small
// tiles spread a small mesh over many SMs)
template <int P, int NE, int Q, int EBX = 0>
struct SfCfg {
  using C = Cfg<P, NE, Q>;
  static constexpr bool DIRECT = Q > 0;
  static constexpr int NP = C::NP, ND = C::ND, NQ = C::NQ, NF = C::NF;
  // the volume points in mirror pairs of the Gauss-Legendre nodes (p >= 3; at
  // p = 1 the pairing saves nothing, at p = 2 its registers would cost the
  // third resident CTA per SM).  The small-mesh stepper's tiles take the same
  // arithmetic, so that its results stay bitwise those of k_element_sf.
  static constexpr bool PAIRS = !DIRECT && P >= 3;
  // tiles of 32 elements on 128 threads at p = 1 (64 on 256 measured 2.5 %
  // slower there), 32 on 256 threads at p = 2 (16 on 128: 6 % slower), 16 on
  // 128 at p = 3 (four CTAs per SM instead of two with 32 on 256: 8 % faster;
  // 8 on 64: 8 % slower), 16 on 256 at p = 4-5 (8 on 128: 7 % slower at p = 4,
  // and at p = 5 no faster on the collapsed grid, 6 % slower on the symmetric
  // rule)
  static constexpr int EB = EBX > 0 ? EBX : (P <= 2 ? 32 : 16);
  static constexpr int THREADS = (P <= 1 || P == 3) ? 128 : kThreads;
  // per element and variable, the edge-flux buffer holds the NF gathered fluxes,
  // then (in place) the LW sums of the factorised lift
  static constexpr int LW = ND + 2 * NE;
  static constexpr int RS = NF > LW ? NF : LW;
  static constexpr int TAB = 3 * ND * ND + 3 * NP * ND + ND + 2 * NP * NE + 2 * ND * NE + NP + (DIRECT ? 3 * NP * NQ : 0);
  // per element: the sum-factorisation buffer (8 ND^2), or for the direct form
  // the new state (its point buffer is read until the last mode is done)
  static constexpr int XS = DIRECT ? M * NP : 8 * ND * ND;
  // per element (collapsed grid, p >= 3): the flux directions of H_alpha at the
  // ND alpha nodes and of H_beta, [ND + 1][2], formed once per tile (at p <= 2
  // the few points' FMAs are not worth the registers: at p = 2 they cost a
  // third resident CTA per SM)
  static constexpr bool PREDIR = !DIRECT && P >= 3;
  static constexpr int DS = PREDIR ? 2 * (ND + 1) : 0;
  static constexpr int TILE = EB * (M * NP + XS + 8 * NQ + RS * M + DS);
  static constexpr int SMEM = (TAB + TILE) * 8;
  static_assert(DIRECT || 8 * NQ >= M * NP, "the new state reuses the point buffer");
};

// The Euler flux of U along two directions a and b (Fa = F1 a_x + F2 a_y, ...).
// The Euler flux along a direction d is (rho v_d, rho u v_d + p d_x,
// rho v v_d + p d_y, (E + p) v_d) with v_d = (rho u d_x + rho v d_y) / rho.
__device__ __forceinline__ void flux_two_dirs(const double U[M], double ax, double ay, double bx, double by,
                                              double gamma, int *err, double Fa[M], double Fb[M]) {
  const double inv = recip(U[0]);
  const double p = (gamma - 1.0) * fma(fma(U[1], U[1], U[2] * U[2]), -0.5 * inv, U[3]);
  if (!(positive_finite(U[0]) & positive_finite(p))) atomicOr(err, kErrNonPhysical);
  const double Ep = U[3] + p;
  {
    const double mn = fma(U[1], ax, U[2] * ay), vd = mn * inv;
    Fa[0] = mn; Fa[1] = fma(U[1], vd, p * ax); Fa[2] = fma(U[2], vd, p * ay); Fa[3] = Ep * vd;
  }
  {
    const double mn = fma(U[1], bx, U[2] * by), vd = mn * inv;
    Fb[0] = mn; Fb[1] = fma(U[1], vd, p * bx); Fb[2] = fma(U[2], vd, p * by); Fb[3] = Ep * vd;
  }
}
// Reference fluxes at one volume point: G_r = J^tau row 0 . (F1, F2), G_s = row 1
// . (F1, F2).
__device__ __forceinline__ void ref_flux(const double U[M], const double *g, double gamma, int *err, double Gr[M],
                                         double Gs[M]) {
  flux_two_dirs(U, g[0], g[1], g[2], g[3], gamma, err, Gr, Gs);
}

// mode j -> a (first Dubiner index); modes are ordered by degree d = a+b, then b
__device__ __forceinline__ int mode_a(int j) {
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= j) ++d;
  return d - (j - d * (d + 1) / 2);
}

// the r-th mode (in mode order) whose first index a is >= 1: degree d holds d of
// them (b = 0 .. d-1), so it lies in the degree d with d(d-1)/2 <= r < d(d+1)/2
__device__ __forceinline__ int mode_a_ge1(int r) {
  int d = 1;
  while (d * (d + 1) / 2 <= r) ++d;
  return d * (d + 1) / 2 + (r - d * (d - 1) / 2);
}

// The element stage on the tiles block, block + nblocks, ... (k_element_sf, and
// the element phase of the fused small-mesh stepper); smem holds SfCfg::SMEM bytes.
template <int P, int NE, int Q, int EBX = 0>
__device__ __forceinline__ void element_sf_tiles(double *smem, const double *c, const double *u0, double *out,
                                                 double *__restrict__ trace_out, const double *__restrict__ fhat,
                                                 const double *__restrict__ geo, const int32_t *__restrict__ elem_face,
                                                 const DevTables &tab, int N, int64_t F, const StageUpdate &su,
                                                 int mode, double gamma, int *err, int block, int nblocks) {
  using S = SfCfg<P, NE, Q, EBX>;
  constexpr int NP = S::NP, ND = S::ND, NQ = S::NQ, NF = S::NF, EB = S::EB;
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
  double *sEChiM1 = sEWPa + ND * NE;   // [NP]       chi_j(-1)
  double *sEPa = sEChiM1 + NP;         // [ND][NE]   P_a(xi_k)
  double *sBvT = sEPa + ND * NE;       // direct form: [NP][NQ] phi_j(r_k)
  double *sDr = sBvT + (S::DIRECT ? NP * NQ : 0);   //  [NQ][NP] w_k d_r phi_j(r_k)
  double *sDs = sDr + (S::DIRECT ? NQ * NP : 0);    //  [NQ][NP] w_k d_s phi_j(r_k)
  double *sC = sDs + (S::DIRECT ? NQ * NP : 0);     // [EB][M][NP]        stage input
  double *sX = sC + EB * M * NP;       // [EB][ND][ND][8]    W (first 4), then Xa, Xb (direct: the new state)
  double *sH = sX + EB * S::XS;        // [EB][NQ][8]        Ha, Hb (direct: G_r, G_s); later the new state
  double *sF = sH + EB * NQ * 8;       // [EB][RS][M]        -F_hat_out * l, then the lift sums
  double *sDir = sF + EB * S::RS * M;  // [EB][ND+1][2]      J^tau row 0 + half_ia row 1 (ia < ND), row 1
  double *sO = S::DIRECT ? sX : sH;
  constexpr int RS = S::RS;

  for (int i = threadIdx.x; i < ND * ND; i += blockDim.x) {
    sPa[i] = tab.SPa[i]; sPaW[i] = tab.SPaW[i]; sdPaW[i] = tab.SdPaW[i];
  }
  for (int i = threadIdx.x; i < NP * ND; i += blockDim.x) {
    sChi[i] = tab.SChi[i]; sChiA[i] = tab.SChiA[i]; sdChiB[i] = tab.SdChiB[i];
  }
  for (int i = threadIdx.x; i < ND; i += blockDim.x) sHalf[i] = tab.SHalf[i];
  for (int i = threadIdx.x; i < NP * NE; i += blockDim.x) { sEChi[i] = tab.EChi[i]; sEWChi[i] = tab.EWChi[i]; }
  for (int i = threadIdx.x; i < ND * NE; i += blockDim.x) sEWPa[i] = tab.EWPa[i];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sEChiM1[i] = tab.EChiM1[i];
  for (int i = threadIdx.x; i < ND * NE; i += blockDim.x) sEPa[i] = tab.EPa[i];
  if constexpr (S::DIRECT) {
    for (int i = threadIdx.x; i < NP * NQ; i += blockDim.x) {
      sBvT[i] = tab.BvT[i]; sDr[i] = tab.Dr[i]; sDs[i] = tab.Ds[i];
    }
  }

  const int ntiles = (N + EB - 1) / EB;
  for (int tile = block; tile < ntiles; tile += nblocks) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *src = c + (size_t)e0 * M * NP;
    for (int i = threadIdx.x; i < EB * M * NP; i += blockDim.x)
      sC[i] = i < ecount * M * NP ? src[i] : 0.0;
    if constexpr (S::PREDIR) {
      // the flux is linear in its direction: H_alpha = G_r + half G_s is the flux
      // along J^tau row 0 + half row 1, H_beta = G_s the flux along row 1
      for (int i = threadIdx.x; i < EB * (ND + 1); i += blockDim.x) {
        const int el = i / (ND + 1), ia = i - el * (ND + 1);
        double dx = 0.0, dy = 0.0;
        if (el < ecount) {
          const double *g = geo + (size_t)(e0 + el) * GEO;
          if (ia < ND) {
            const double half = sHalf[ia];
            dx = fma(half, g[2], g[0]);
            dy = fma(half, g[3], g[1]);
          } else {
            dx = g[2];
            dy = g[3];
          }
        }
        sDir[2 * i] = dx;
        sDir[2 * i + 1] = dy;
      }
    }
    for (int i = threadIdx.x; i < EB * NF; i += blockDim.x) {
      const int el = i / NF, qk = i - el * NF;
      double v[M] = {0.0, 0.0, 0.0, 0.0};
      if (el < ecount) {
        const int q = qk / NE, k = qk - q * NE;
        const int ef = elem_face[(size_t)(e0 + el) * 3 + q];
        const int64_t f = checked(ef >> 1, F, err);
        const int side = ef & 1;
        const double *fp = fhat + ((size_t)f * NE + (side ? NE - 1 - k : k)) * M;
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = side ? fp[m] : tc::neg_bits(fp[m]);
      }
#pragma unroll
      for (int m = 0; m < M; ++m) sF[(el * RS + qk) * M + m] = v[m];
    }
    __syncthreads();

    // the lift's edge sums, in place of the element's fluxes of one variable:
    //   Q_a = sum_k omega_k P_a(xi_k) F0_k                            (face 0)
    //   G_even,k / G_odd,k = F1_k +/- F2_{NE-1-k}                   (faces 1, 2)
    // so that the lift of mode j = (a, b) is
    //   chi_j(-1) Q_a + sum_k omega_k chi_j(xi_k) G_{a mod 2, k}
    for (int i = threadIdx.x; i < EB * M; i += blockDim.x) {
      double *fe = sF + (i / M) * RS * M + (i % M);
      double f[NF];
#pragma unroll
      for (int x = 0; x < NF; ++x) f[x] = fe[x * M];
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < NE; ++k) q = fma(sEWPa[a * NE + k], f[k], q);
        fe[a * M] = q;
      }
#pragma unroll
      for (int k = 0; k < NE; ++k) {
        fe[(ND + k) * M] = f[NE + k] + f[3 * NE - 1 - k];
        fe[(ND + NE + k) * M] = f[NE + k] - f[3 * NE - 1 - k];
      }
    }

    if constexpr (S::DIRECT) {
      // volume points: U = sum_j phi_j c_j, then G_r, G_s; one item per (element, point)
      for (int i = threadIdx.x; i < EB * NQ; i += blockDim.x) {
        const int el = i / NQ, k = i - el * NQ;
        double U[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const double b = sBvT[j * NQ + k];
#pragma unroll
          for (int m = 0; m < M; ++m) U[m] = fma(b, sC[(el * M + m) * NP + j], U[m]);
        }
        double Gr[M] = {0.0, 0.0, 0.0, 0.0}, Gs[M] = {0.0, 0.0, 0.0, 0.0};
        if (el < ecount) ref_flux(U, geo + (size_t)(e0 + el) * GEO, gamma, err, Gr, Gs);
        double *h = sH + (size_t)i * 8;
#pragma unroll
        for (int m = 0; m < M; ++m) { h[m] = Gr[m]; h[4 + m] = Gs[m]; }
      }
      __syncthreads();
    } else {
      // W(a, ib) = sum over the modes with first index a of chi_j(beta_ib) c_j; one
      // item per (element, ib, variable) runs over all modes (the same unrolled
      // sequence in every lane)
      for (int i = threadIdx.x; i < EB * ND * M; i += blockDim.x) {
        const int el = i / (ND * M), ib = (i / M) % ND, m = i % M;
        const double *cm = sC + (el * M + m) * NP;
        double w[ND];
#pragma unroll
        for (int a = 0; a < ND; ++a) w[a] = 0.0;
#pragma unroll
        for (int d = 0; d <= P; ++d)
#pragma unroll
          for (int b = 0; b <= d; ++b) {
            const int j = d * (d + 1) / 2 + b;
            w[d - b] = fma(sChi[j * ND + ib], cm[j], w[d - b]);
          }
#pragma unroll
        for (int a = 0; a < ND; ++a) sX[((el * ND + a) * ND + ib) * 8 + m] = w[a];
      }
      __syncthreads();

      // volume points: U = sum_a P_a W; Euler flux; Ha, Hb.
      // PAIRS (p >= 3): one item per (element, ib, mirror pair ia, ia' = ND-1-ia
      // of the Gauss-Legendre nodes), then (p + 1 odd) one per (element, ib) for
      // the middle node.  With P_a(alpha_ia') = (-1)^a P_a(alpha_ia) the pair's
      // states are E +/- O, E = sum_{a even} P_a W, O = sum_{a odd} P_a W, and the
      // point slots of the pair receive the sums and differences the folded
      // projection takes: slot ia (Ha + Ha', Hb + Hb'), slot ia' (Ha - Ha',
      // Hb - Hb'); the middle slot keeps (Ha, Hb).
      if constexpr (S::PAIRS) {
        constexpr int NH = ND / 2, NPAIR = EB * ND * NH, NMID = (ND & 1) ? EB * ND : 0;
        for (int i = threadIdx.x; i < NPAIR + NMID; i += blockDim.x) {
          if ((ND & 1) && i >= NPAIR) {
            // the middle node alpha = 0 (p + 1 odd), after all the pairs so that
            // warps stay uniform: P_a(0) = 0 for odd a
            const int el = (i - NPAIR) / ND, ib = (i - NPAIR) - el * ND;
            constexpr int MID = ND / 2;
            const double *w0 = sX + ((el * ND) * ND + ib) * 8;
            double U[M] = {w0[0], w0[1], w0[2], w0[3]};
#pragma unroll
            for (int a = 2; a < ND; a += 2) {
              const double pa = sPa[a * ND + MID];
              const double *w = sX + ((el * ND + a) * ND + ib) * 8;
#pragma unroll
              for (int m = 0; m < M; ++m) U[m] = fma(pa, w[m], U[m]);
            }
            double Ha[M], Hb[M];
            if (el < ecount) {
              const double *dir = sDir + el * 2 * (ND + 1);
              flux_two_dirs(U, dir[2 * MID], dir[2 * MID + 1], dir[2 * ND], dir[2 * ND + 1], gamma, err, Ha, Hb);
            } else {
#pragma unroll
              for (int m = 0; m < M; ++m) { Ha[m] = 0.0; Hb[m] = 0.0; }
            }
            double *h = sH + ((size_t)el * NQ + ib * ND + MID) * 8;
#pragma unroll
            for (int m = 0; m < M; ++m) { h[m] = Ha[m]; h[4 + m] = Hb[m]; }
            continue;
          }
          const int el = i / (ND * NH), r = i - el * (ND * NH), ib = r / NH, ia = r - ib * NH;
          const int ia2 = ND - 1 - ia;
          const double *w0 = sX + ((el * ND) * ND + ib) * 8;
          double E[M] = {w0[0], w0[1], w0[2], w0[3]}, O[M];
#pragma unroll
          for (int a = 1; a < ND; ++a) {
            const double pa = sPa[a * ND + ia];
            const double *w = sX + ((el * ND + a) * ND + ib) * 8;
#pragma unroll
            for (int m = 0; m < M; ++m) {
              if (a == 1) O[m] = pa * w[m];
              else if (a & 1) O[m] = fma(pa, w[m], O[m]);
              else E[m] = fma(pa, w[m], E[m]);
            }
          }
          double S1[M], D1[M], S2[M], D2[M];
          if (el < ecount) {
            const double *dir = sDir + el * 2 * (ND + 1);
            const double bx = dir[2 * ND], by = dir[2 * ND + 1];
            double U[M], Ha[M], Hb[M], Ha2[M], Hb2[M];
#pragma unroll
            for (int m = 0; m < M; ++m) U[m] = E[m] + O[m];
            flux_two_dirs(U, dir[2 * ia], dir[2 * ia + 1], bx, by, gamma, err, Ha, Hb);
#pragma unroll
            for (int m = 0; m < M; ++m) U[m] = E[m] - O[m];
            flux_two_dirs(U, dir[2 * ia2], dir[2 * ia2 + 1], bx, by, gamma, err, Ha2, Hb2);
#pragma unroll
            for (int m = 0; m < M; ++m) {
              S1[m] = Ha[m] + Ha2[m]; D1[m] = Ha[m] - Ha2[m];
              S2[m] = Hb[m] + Hb2[m]; D2[m] = Hb[m] - Hb2[m];
            }
          } else {
#pragma unroll
            for (int m = 0; m < M; ++m) { S1[m] = 0.0; D1[m] = 0.0; S2[m] = 0.0; D2[m] = 0.0; }
          }
          double *h1 = sH + ((size_t)el * NQ + ib * ND + ia) * 8, *h2 = sH + ((size_t)el * NQ + ib * ND + ia2) * 8;
#pragma unroll
          for (int m = 0; m < M; ++m) {
            h1[m] = S1[m]; h1[4 + m] = S2[m];
            h2[m] = D1[m]; h2[4 + m] = D2[m];
          }
        }
      } else {
        for (int i = threadIdx.x; i < EB * NQ; i += blockDim.x) {
          const int el = i / NQ, k = i - el * NQ, ib = k / ND, ia = k - ib * ND;
          // P_0 = 1: the a = 0 term is W(0, ib) itself
          const double *w0 = sX + ((el * ND) * ND + ib) * 8;
          double U[M] = {w0[0], w0[1], w0[2], w0[3]};
#pragma unroll
          for (int a = 1; a < ND; ++a) {
            const double pa = sPa[a * ND + ia];
            const double *w = sX + ((el * ND + a) * ND + ib) * 8;
#pragma unroll
            for (int m = 0; m < M; ++m) U[m] += pa * w[m];
          }
          double Ha[M], Hb[M];
          if (el < ecount) {
            if constexpr (S::PREDIR) {
              const double *dir = sDir + el * 2 * (ND + 1);
              flux_two_dirs(U, dir[2 * ia], dir[2 * ia + 1], dir[2 * ND], dir[2 * ND + 1], gamma, err, Ha, Hb);
            } else {
              // the flux along J^tau row 0 + half row 1 and along row 1
              const double *g = geo + (size_t)(e0 + el) * GEO;
              const double half = sHalf[ia];
              flux_two_dirs(U, fma(half, g[2], g[0]), fma(half, g[3], g[1]), g[2], g[3], gamma, err, Ha, Hb);
            }
          } else {
#pragma unroll
            for (int m = 0; m < M; ++m) { Ha[m] = 0.0; Hb[m] = 0.0; }
          }
          double *h = sH + (size_t)i * 8;
#pragma unroll
          for (int m = 0; m < M; ++m) { h[m] = Ha[m]; h[4 + m] = Hb[m]; }
        }
      }
      __syncthreads();

      if constexpr (P >= 2 && P <= 4) {
        // Xa(a, ib) = sum_ia Ha wa P_a', Xb(a, ib) = sum_ia Hb wa P_a, one item per
        // (element, ib, variable) over every a, folded on the mirror pairs of the
        // Gauss-Legendre nodes (alpha_{ND-1-ia} = -alpha_ia, the same weight):
        // P_a(-x) = (-1)^a P_a(x) and P_a'(-x) = (-1)^(a+1) P_a'(x), so
        //   Xb(a) = sum_{ia < ND/2} wa P_a(alpha_ia) (Hb_ia +/- Hb_ia'),  + for a even
        //   Xa(a) = sum_{ia < ND/2} wa P_a'(alpha_ia) (Ha_ia -/+ Ha_ia'), - for a even,
        // and for ND odd the middle node alpha = 0 enters Xb of the even a and Xa
        // of the odd a only (P_a(0) = 0 for a odd, P_a'(0) = 0 for a even).  Per item
        // that is 4 (ND / 2) additions (already formed by the point phase when
        // PAIRS) and about half the products of the plain sums; Xa(0, ib) = 0
        // (P_0' = 0) costs no arithmetic.
        constexpr int NH = ND / 2, MID = ND / 2;
        for (int i = threadIdx.x; i < EB * ND * M; i += blockDim.x) {
          const int el = i / (ND * M), ib = (i / M) % ND, m = i % M;
          const double *hrow = sH + ((el * NQ) + ib * ND) * 8;
          double ea[NH], oa[NH], eb[NH], ob[NH];
#pragma unroll
          for (int ia = 0; ia < NH; ++ia) {
            const double *h1 = hrow + ia * 8, *h2 = hrow + (ND - 1 - ia) * 8;
            const double a1 = h1[m], a2 = h2[m], b1 = h1[4 + m], b2 = h2[4 + m];
            if constexpr (S::PAIRS) {
              ea[ia] = a1; oa[ia] = a2;
              eb[ia] = b1; ob[ia] = b2;
            } else {
              ea[ia] = a1 + a2; oa[ia] = a1 - a2;
              eb[ia] = b1 + b2; ob[ia] = b1 - b2;
            }
          }
          double xa[ND], xb[ND];
#pragma unroll
          for (int a = 0; a < ND; ++a) {
            const double *fb = (a & 1) ? ob : eb, *fa = (a & 1) ? ea : oa;
            double sb = 0.0, sa = 0.0;
            if ((ND & 1) && !(a & 1)) sb = hrow[MID * 8 + 4 + m] * sPaW[a * ND + MID];
            if ((ND & 1) && (a & 1)) sa = hrow[MID * 8 + m] * sdPaW[a * ND + MID];
#pragma unroll
            for (int ia = 0; ia < NH; ++ia) {
              sb = fma(fb[ia], sPaW[a * ND + ia], sb);
              if (a > 0) sa = fma(fa[ia], sdPaW[a * ND + ia], sa);
            }
            xa[a] = sa;
            xb[a] = sb;
          }
#pragma unroll
          for (int a = 0; a < ND; ++a) {
            double *x = sX + ((el * ND + a) * ND + ib) * 8;
            x[m] = xa[a];
            x[4 + m] = xb[a];
          }
        }
      } else if constexpr (P <= 4) {
        // p = 1: the plain sums (the folding would add more than it saves)
        for (int i = threadIdx.x; i < EB * ND * M; i += blockDim.x) {
          const int el = i / (ND * M), ib = (i / M) % ND, m = i % M;
          double xa[ND], xb[ND];
#pragma unroll
          for (int a = 0; a < ND; ++a) { xa[a] = 0.0; xb[a] = 0.0; }
#pragma unroll
          for (int ia = 0; ia < ND; ++ia) {
            const double *h = sH + ((el * NQ) + ib * ND + ia) * 8;
            const double ha = h[m], hb = h[4 + m];
#pragma unroll
            for (int a = 1; a < ND; ++a) xa[a] = fma(ha, sdPaW[a * ND + ia], xa[a]);
#pragma unroll
            for (int a = 0; a < ND; ++a) xb[a] = fma(hb, sPaW[a * ND + ia], xb[a]);
          }
#pragma unroll
          for (int a = 0; a < ND; ++a) {
            double *x = sX + ((el * ND + a) * ND + ib) * 8;
            x[m] = xa[a];
            x[4 + m] = xb[a];
          }
        }
      } else {
        // p = 5: one item per (element, a, ib) for all four variables (the
        // per-variable form above would spill at this size), on the pair sums and
        // differences of the point phase (PAIRS): Xa(a) takes the sums of Ha for
        // a odd and the differences for a even, Xb(a) the sums of Hb for a even
        // and the differences for a odd, over the ND / 2 pairs
        static_assert(S::PAIRS && S::PREDIR, "p = 5 has mirror pairs");
        constexpr int NH = ND / 2;
        for (int i = threadIdx.x; i < EB * ND * ND; i += blockDim.x) {
          const int el = i / (ND * ND), a = (i / ND) % ND, ib = i % ND;
          double xa[M] = {0.0, 0.0, 0.0, 0.0}, xb[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
          for (int ia = 0; ia < NH; ++ia) {
            const double dp = sdPaW[a * ND + ia], pa = sPaW[a * ND + ia];
            const double *hs = sH + ((el * NQ) + ib * ND + ia) * 8, *hd = sH + ((el * NQ) + ib * ND + ND - 1 - ia) * 8;
            const double *fa = (a & 1) ? hs : hd, *fb = (a & 1) ? hd : hs;
#pragma unroll
            for (int m = 0; m < M; ++m) { xa[m] = fma(fa[m], dp, xa[m]); xb[m] = fma(fb[4 + m], pa, xb[m]); }
          }
          double *x = sX + (size_t)i * 8;
#pragma unroll
          for (int m = 0; m < M; ++m) { x[m] = xa[m]; x[4 + m] = xb[m]; }
        }
      }
      __syncthreads();

    }

    // modes: V_j + lifted edge fluxes, 1/det J, stage update.  Sum-factorised:
    // the items of the modes with a >= 1 come first and those of the modes with
    // a = 0 (b = d) last, so that warps take one branch of the projection (for
    // a = 0, Xa(0, .) = 0 and only the Xb term is formed)
    for (int i = threadIdx.x; i < EB * NP; i += blockDim.x) {
      int el, j;
      if constexpr (S::DIRECT) {
        el = i / NP;
        j = i - el * NP;
      } else {
        constexpr int NB = NP - ND;                   // modes with a >= 1
        if (i < EB * NB) {
          el = i / NB;
          j = mode_a_ge1(i - el * NB);
        } else {
          const int i2 = i - EB * NB;
          el = i2 / ND;
          const int d = i2 - el * ND;
          j = d * (d + 1) / 2 + d;
        }
      }
      const int a = mode_a(j);
      double acc[M] = {0.0, 0.0, 0.0, 0.0};
      if constexpr (S::DIRECT) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          const double dr = sDr[k * NP + j], ds = sDs[k * NP + j];
          const double *h = sH + (el * NQ + k) * 8;
#pragma unroll
          for (int m = 0; m < M; ++m) acc[m] = fma(ds, h[4 + m], fma(dr, h[m], acc[m]));
        }
      } else if (a > 0) {
#pragma unroll
        for (int ib = 0; ib < ND; ++ib) {
          const double ch = sChiA[j * ND + ib], dch = sdChiB[j * ND + ib];
          const double *x = sX + ((el * ND + a) * ND + ib) * 8;
#pragma unroll
          for (int m = 0; m < M; ++m) acc[m] = fma(dch, x[4 + m], fma(ch, x[m], acc[m]));
        }
      } else {
#pragma unroll
        for (int ib = 0; ib < ND; ++ib) {
          const double dch = sdChiB[j * ND + ib];
          const double *x = sX + (el * ND * ND + ib) * 8;
#pragma unroll
          for (int m = 0; m < M; ++m) acc[m] = fma(dch, x[4 + m], acc[m]);
        }
      }
      {
        const double *fl = sF + el * RS * M;
        const double c1 = sEChiM1[j];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] = fma(c1, fl[a * M + m], acc[m]);
        const double *g = fl + (ND + (a & 1) * NE) * M;
#pragma unroll
        for (int k = 0; k < NE; ++k) {
          const double l = sEWChi[j * NE + k];
#pragma unroll
          for (int m = 0; m < M; ++m) acc[m] = fma(l, g[k * M + m], acc[m]);
        }
      }
      double nv[M] = {0.0, 0.0, 0.0, 0.0};
      if (el < ecount) {
        const size_t e = (size_t)(e0 + el);
        const double inv = geo[e * GEO + 4];
        // stage update a0 u0 + b0 c + g dt R with R = acc / det J, as
        // b0 c + a0 u0 + (g dt / det J) acc (and the second output alike)
        const double kap = su.g * su.dt * inv;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const size_t idx = (e * M + m) * NP + j;
          double v;
          if (mode == 0) {
            v = acc[m] * inv;
          } else {
            double t = su.b0 * sC[(el * M + m) * NP + j];
            if (su.a0 != 0.0) t = fma(su.a0, u0[idx], t);
            v = fma(kap, acc[m], t);
            if (su.out2) {
              double t2 = su.y * v;
              if (su.x != 0.0) t2 = fma(su.x, su.acc[idx], t2);
              su.out2[idx] = fma(su.w * su.dt * inv, acc[m], t2);
            }
          }
          out[idx] = v;
          nv[m] = v;
        }
      }
      // the new state, for the next stage's traces (sum-factorised: sH is free,
      // every thread has passed the barrier after the X phase, the last reader of
      // sH; direct: a buffer of its own, the modes still read sH)
#pragma unroll
      for (int m = 0; m < M; ++m) sO[(el * M + m) * NP + j] = nv[m];
    }

    if (trace_out) {
      __syncthreads();
      // Z_a of the new state (face 0 lies on beta = -1), one item per (element,
      // variable), in the buffer the modes have finished reading (sX; direct: sH)
      double *sZ = S::DIRECT ? sH : sX;
      for (int i = threadIdx.x; i < ecount * M; i += blockDim.x) {
        double z[ND + 1];
        face_sums<P>(sO + i * NP, sEChiM1, sEChi[0], z);
#pragma unroll
        for (int a = 0; a <= ND; ++a) sZ[i * (ND + 1) + a] = z[a];
      }
      __syncthreads();
      // edge traces of the new state, one item per (element, variable, edge point k):
      //   T0_k = sum_a P_a(xi_k) Z_a,
      //   T1_k = sum_a Y_a(xi_k),  T2_{NE-1-k} = sum_a (-1)^a Y_a(xi_k),
      //   Y_a(xi) = sum_b chi_ab(xi) c_ab
      for (int i = threadIdx.x; i < ecount * M * NE; i += blockDim.x) {
        const int el = i / (M * NE), m = (i / NE) % M, k = i % NE;
        const double *cj = sO + (el * M + m) * NP;
        double *dst = trace_out + (size_t)(e0 + el) * NF * M + m;
        double t0, t1, t2;
        edge_traces_unit<P, NE>(cj, sZ + (el * M + m) * (ND + 1), sEPa, sEChi, k, t0, t1, t2);
        dst[k * M] = t0;
        dst[(NE + k) * M] = t1;
        dst[(3 * NE - 1 - k) * M] = t2;
      }
    }
  }
}

template <int P, int NE, int Q>
__global__ void __launch_bounds__(kThreads, 2)
k_element_sf(const double *c, const double *u0, double *out, double *__restrict__ trace_out,
             const double *__restrict__ fhat, const double *__restrict__ geo,
             const int32_t *__restrict__ elem_face, DevTables tab, int N, int64_t F, StageUpdate su, int mode,
             double gamma, int *err) {
  extern __shared__ double smem[];
  element_sf_tiles<P, NE, Q>(smem, c, u0, out, trace_out, fhat, geo, elem_face, tab, N, F, su, mode, gamma, err,
                             blockIdx.x, gridDim.x);
}


// CTAs of k_element_sf per SM (the kernel's shared memory attribute set first)
template <int P, int NE, int Q>
int element_sf_per_sm(const dg_mesh *m, int *per_sm) {
  using S = SfCfg<P, NE, Q>;
  static PerDevice attr_set;
  if (!attr_set.test(m->device)) {
    cudaError_t e = cudaFuncSetAttribute(k_element_sf<P, NE, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_element_sf<P, NE, Q>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr_set.set(m->device);
  }
  *per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_element_sf<P, NE, Q>, S::THREADS, S::SMEM);
  if (e != cudaSuccess) return (int)e;
  if (*per_sm < 1) *per_sm = 1;
  return (int)cudaSuccess;
}

// Elements [e0, e1) of the mesh (e1 < 0: all): the kernel runs on the views of
// the arrays that start at element e0.  Each element's arithmetic does not
// depend on the tile it falls in, so a range launch gives the same bits.
template <int P, int NE, int Q>
int run_element_sf(const dg_mesh *m, const double *c, const double *u0, double *out, double *trace_out,
                   const double *fhat, const StageUpdate &su0, int mode, cudaStream_t s, int64_t e0 = 0,
                   int64_t e1 = -1) {
  using S = SfCfg<P, NE, Q>;
  int per_sm = 0;
  int err = element_sf_per_sm<P, NE, Q>(m, &per_sm);
  if (err != (int)cudaSuccess) return err;
  if (e1 < 0) e1 = m->N;
  const int64_t n = e1 - e0;
  if (n <= 0) return (int)cudaSuccess;
  const size_t so = (size_t)e0 * M * S::NP;           // state rows of the range
  StageUpdate su = su0;
  if (su.acc) su.acc += so;
  if (su.out2) su.out2 += so;
  const int ntiles = (int)((n + S::EB - 1) / S::EB);
  const int grid = ntiles < m->num_sms * per_sm ? ntiles : m->num_sms * per_sm;
  k_element_sf<P, NE, Q><<<grid, S::THREADS, S::SMEM, s>>>(
      c + so, u0 ? u0 + so : nullptr, out + so, trace_out ? trace_out + (size_t)e0 * S::NF * M : nullptr, fhat,
      m->geo + (size_t)e0 * GEO, m->elem_face + (size_t)e0 * 3, m->tab, (int)n, m->F, su, mode, m->gamma,
      m->err_flag);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fused small-mesh stepper
//
// On a mesh whose element tiles fit in one wave of the GPU, a stage's two
// launches (edge flux, element) do a few microseconds of work each and the step
// is bound by launch latency (the paper's Section 7.1 finds its small meshes
// alike).  This kernel runs every stage of a whole call inside one cooperative
// launch: the edge phase (face_flux_points) and the element phase
// (element_sf_tiles) of the same code as k_face and k_element_sf, separated by a
// barrier over the grid, so the results are bitwise those of the separate
// launches.
// ---------------------------------------------------------------------------
constexpr uint64_t kGridWaitNs = 2000000000ull;    // 2 s per barrier before giving up

// All blocks of the (co-resident) grid meet here: one thread per block arrives on
// a counter, the last one resets it and advances the generation the others
// wait on.  The wait is bounded: after kGridWaitNs it records kErrTimeout and
// returns false, and the caller leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, int *err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();                                  // this block's writes before its arrival
    int ok = 1;
    if (atomicAdd(bar, 1u) + 1u == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = tc::global_ns();
      while (*gen == g) {
        if (tc::global_ns() - t0 > kGridWaitNs) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();                                  // the other blocks' writes after it
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

constexpr int kSmallThreads = 128;
constexpr int kSmallTiles[2] = {4, 8};          // elements per tile of the two variants

template <int P, int NE, int Q, int EBX>
__global__ void __launch_bounds__(kSmallThreads, 4)
k_rk_small(double *c, double *S, double *A, double *trace, double *fhat, const double *__restrict__ geo,
           const int32_t *__restrict__ elem_face, const FaceConn *__restrict__ conn, const FaceGeo *__restrict__ fg,
           const double *__restrict__ bstate, const int32_t *__restrict__ elem_nbr, DevTables tab, int N, int64_t F,
           double gamma, double phi1, double dt, int nsteps, int method, int limit, unsigned *bar, int *err) {
  extern __shared__ double smem[];
  const unsigned nb = gridDim.x;
  const int ns = rk_num_stages(method);
  for (int step = 0; step < nsteps; ++step)
    for (int i = 0; i < ns; ++i) {
      const RkStage st = rk_stage(method, i, dt, c, S, A);
      face_flux_points<NE>(trace, fhat, conn, fg, bstate, N, F, gamma, err, blockIdx.x, nb);
      if (!grid_barrier(bar, nb, err)) return;
      element_sf_tiles<P, NE, Q, EBX>(smem, st.cin, st.u0, st.out, trace, fhat, geo, elem_face, tab, N, F, st.su, 1,
                                      gamma, err, blockIdx.x, nb);
      if (!grid_barrier(bar, nb, err)) return;
      if constexpr (P == 1) {
        // with the limiter on, every stage value is limited in place (and the
        // traces of the elements it limits rewritten) before the next stage
        if (limit) {
          limit_p1_items<true>(st.out, trace, elem_nbr, tab.EPa, tab.EChiM1, tab.EChi, phi1, N, err, blockIdx.x, nb);
          if (!grid_barrier(bar, nb, err)) return;
        }
      }
    }
}

// Resident blocks per SM of the two variants on the mesh's device (0: not
// launchable), asked once per device.
template <int P, int NE, int Q>
const int *small_per_sm(int dev) {
  static PerDevice ready;
  static int per_sm[64][2];
  static int fallback[2];
  int *r = dev >= 0 && dev < 64 ? per_sm[dev] : fallback;
  if (dev >= 0 && dev < 64 && ready.test(dev)) return r;
  auto k0 = k_rk_small<P, NE, Q, kSmallTiles[0]>;
  auto k1 = k_rk_small<P, NE, Q, kSmallTiles[1]>;
  const int s0 = SfCfg<P, NE, Q, kSmallTiles[0]>::SMEM, s1 = SfCfg<P, NE, Q, kSmallTiles[1]>::SMEM;
  r[0] = r[1] = 0;
  if (cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, s0) != cudaSuccess ||
      cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, s1) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[0], k0, kSmallThreads, s0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[1], k1, kSmallThreads, s1) != cudaSuccess) {
    cudaGetLastError();
    r[0] = r[1] = 0;
  }
  if (dev >= 0 && dev < 64) ready.set(dev);
  return r;
}

// the variant whose tiles of the mesh fit in one wave (its blocks all resident),
// the smaller tiles first; -1 if neither
template <int P, int NE, int Q>
int small_variant(const dg_mesh *m) {
  const int *per_sm = small_per_sm<P, NE, Q>(m->device);
  for (int v = 0; v < 2; ++v) {
    const int64_t nb = (m->N + kSmallTiles[v] - 1) / kSmallTiles[v];
    if (per_sm[v] > 0 && nb <= (int64_t)m->num_sms * per_sm[v]) return v;
  }
  return -1;
}

template <int P, int NE, int Q, int EBX>
int run_rk_small(dg_mesh *m, double *c, double dt, int nsteps, int method, cudaStream_t s) {
  using Sc = SfCfg<P, NE, Q, EBX>;
  auto kern = k_rk_small<P, NE, Q, EBX>;
  // one tile per block (the variant was chosen so that they are all resident);
  // the edge phase spreads its points over the same blocks
  const int64_t nb = (m->N + EBX - 1) / EBX;
  cudaError_t e = cudaMemsetAsync(m->gbar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return (int)e;
  double *S = m->stage, *A = m->rk_acc, *tr = m->trace, *fh = m->fhat;
  const double *geo = m->geo, *bst = m->bstate;
  const int32_t *ef = m->elem_face;
  const FaceConn *conn = m->face_conn;
  const FaceGeo *fg = m->face_geo;
  DevTables tab = m->tab;
  int N = (int)m->N;
  int64_t F = m->F;
  double gamma = m->gamma;
  unsigned *bar = m->gbar;
  int *err = m->err_flag;
  const int32_t *nbr = m->elem_nbr;
  double phi1 = m->phi1;
  int limit = m->limiter ? 1 : 0;
  void *args[] = {&c,   &S, &A, &tr,    &fh,   &geo, &ef,     &conn,  &fg,   &bst, &nbr, &tab,
                  &N,   &F, &gamma, &phi1, &dt,   &nsteps, &method, &limit, &bar, &err};
  return (int)cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)nb), dim3(kSmallThreads), args,
                                          Sc::SMEM, s);
}

template <int P, int NE, int Q>
int run_small(dg_mesh *m, double *c, double dt, int nsteps, int method, cudaStream_t s) {
  switch (small_variant<P, NE, Q>(m)) {
    case 0: return run_rk_small<P, NE, Q, kSmallTiles[0]>(m, c, dt, nsteps, method, s);
    case 1: return run_rk_small<P, NE, Q, kSmallTiles[1]>(m, c, dt, nsteps, method, s);
    default: return (int)cudaErrorCooperativeLaunchTooLarge;
  }
}

template <int P, int NE, int Q>
bool fits_small(const dg_mesh *m) {
  return small_variant<P, NE, Q>(m) >= 0;
}

}  // namespace

bool small_rk_fits(const dg_mesh *m) {
#define CALL(P, NE) (m->rule == DG_RULE_SYMMETRIC ? fits_small<P, NE, sym_points(P)>(m) : fits_small<P, NE, 0>(m))
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return false;
}

int launch_rk_small(dg_mesh *m, double *c, double dt, int nsteps, int method, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
#define CALL(P, NE)                                                                        \
  (m->rule == DG_RULE_SYMMETRIC ? run_small<P, NE, sym_points(P)>(m, c, dt, nsteps, method, s) \
                                : run_small<P, NE, 0>(m, c, dt, nsteps, method, s))
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaErrorInvalidValue;
}

int element_wave(const dg_mesh *m, int *tiles, int *elems_per_tile) {
#define CALL(P, NE)                                                                                 \
  (m->rule == DG_RULE_SYMMETRIC                                                                     \
       ? (*elems_per_tile = SfCfg<P, NE, sym_points(P)>::EB, element_sf_per_sm<P, NE, sym_points(P)>(m, tiles)) \
       : (*elems_per_tile = SfCfg<P, NE, 0>::EB, element_sf_per_sm<P, NE, 0>(m, tiles)))
  int e = (int)cudaErrorInvalidValue;
  if (m->p == 1 && m->ne == 2) e = CALL(1, 2);
  else if (m->p == 2 && m->ne == 3) e = CALL(2, 3);
  else if (m->p == 3 && m->ne == 4) e = CALL(3, 4);
  else if (m->p == 3 && m->ne == 3) e = CALL(3, 3);
  else if (m->p == 4 && m->ne == 5) e = CALL(4, 5);
  else if (m->p == 5 && m->ne == 6) e = CALL(5, 6);
#undef CALL
  if (e == (int)cudaSuccess) *tiles *= m->num_sms;
  return e;
}

int launch_element(const dg_mesh *m, const double *c, const double *u0, double *out, double *trace_out,
                   const double *fhat, const StageUpdate &su, int mode, void *stream, int64_t e0, int64_t e1) {
  cudaStream_t s = (cudaStream_t)stream;
#define CALL(P, NE)                                                                                        \
  (m->rule == DG_RULE_SYMMETRIC                                                                            \
       ? run_element_sf<P, NE, sym_points(P)>(m, c, u0, out, trace_out, fhat, su, mode, s, e0, e1)        \
       : run_element_sf<P, NE, 0>(m, c, u0, out, trace_out, fhat, su, mode, s, e0, e1))
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
