/*
 * dg_element.cu -- the float64 element kernel of one stage (k_element_sf): the
 * volume integral (Eq. volume, Algorithm 1) sum-factorised on the collapsed
 * volume grid, the lift of the three edge fluxes (Algorithms 2-3), the 1/det J
 * scaling (Eq. 2ddg0), the Runge-Kutta stage update (with, for the classical
 * RK4, the running sum of its stages as a second output) and the next stage's
 * edge traces, for one tile of elements per CTA.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

// ---------------------------------------------------------------------------
// element kernel, sum-factorised volume term (float64 path)
//
// The volume rule is a tensor grid in the collapsed coordinates (alpha, beta)
// and the basis factors as phi_j = P_a(alpha) chi_j(beta), so
//   interpolation  U(ia,ib) = sum_a P_a(alpha_ia) W(a,ib),  W(a,ib) = sum_{j:a(j)=a} chi_j(beta_ib) c_j
//   projection     V_j = sum_ib chi_j(beta_ib) Xa(a,ib) + chi_j'(beta_ib) Xb(a,ib),
//                  Xa(a,ib) = sum_ia Ha(ia,ib) P_a'(alpha_ia),  Xb(a,ib) = sum_ia Hb(ia,ib) P_a(alpha_ia),
// with Ha = w (2 G_r + (1+alpha) G_s)/(1-s) and Hb = 2 w G_s from the chain rule
// d/dr = 2/(1-s) d/dalpha, d/ds = (1+alpha)/(1-s) d/dalpha + 2 d/dbeta.  This is the
// same sum as the direct projection (Eq. volume), in (p+1)(N_p + (p+1)^2) instead
// of (p+1)^2 N_p products per variable for each of the two contractions.
// ---------------------------------------------------------------------------
template <int P, int NE>
struct SfCfg {
  using C = Cfg<P, NE>;
  static constexpr int NP = C::NP, ND = C::ND, NQ = C::NQ, NF = C::NF;
  static constexpr int EB = P <= 1 ? 64 : (P <= 3 ? 32 : 16);
  static constexpr int TAB = 2 * ND * ND + 2 * NP * ND + 3 * NQ + 2 * NF * NP;
  static constexpr int TILE = EB * (M * NP + 8 * ND * ND + 8 * NQ + NF * M);
  static constexpr int SMEM = (TAB + TILE) * 8;
  static_assert(8 * NQ >= M * NP, "the new state reuses the point buffer");
};

// mode j -> a (first Dubiner index); modes are ordered by degree d = a+b, then b
__device__ __forceinline__ int mode_a(int j) {
  int d = 0;
  while ((d + 1) * (d + 2) / 2 <= j) ++d;
  return d - (j - d * (d + 1) / 2);
}

template <int P, int NE>
__global__ void __launch_bounds__(kThreads)
k_element_sf(const double *c, const double *u0, double *out, double *__restrict__ trace_out,
             const double *__restrict__ fhat, const double *__restrict__ geo,
             const int32_t *__restrict__ elem_face, DevTables tab, int N, StageUpdate su, int mode,
             double gamma, int *err) {
  using S = SfCfg<P, NE>;
  constexpr int NP = S::NP, ND = S::ND, NQ = S::NQ, NF = S::NF, EB = S::EB;
  extern __shared__ double smem[];
  double *sPa = smem;                  // [ND][ND]
  double *sdPa = sPa + ND * ND;        // [ND][ND]
  double *sChi = sdPa + ND * ND;       // [NP][ND]
  double *sdChi = sChi + NP * ND;      // [NP][ND]
  double *sK = sdChi + NP * ND;        // [3][NQ]
  double *sLf = sK + 3 * NQ;           // [NF][NP]
  double *sBfT = sLf + NF * NP;        // [NP][NF]
  double *sC = sBfT + NP * NF;         // [EB][M][NP]        stage input
  double *sX = sC + EB * M * NP;       // [EB][ND][ND][8]    W (first 4), then Xa, Xb
  double *sH = sX + EB * ND * ND * 8;  // [EB][NQ][8]        Ha, Hb; later the new state
  double *sF = sH + EB * NQ * 8;       // [EB][NF][M]        -F_hat_out * l
  double *sO = sH;

  for (int i = threadIdx.x; i < ND * ND; i += blockDim.x) { sPa[i] = tab.SPa[i]; sdPa[i] = tab.SdPa[i]; }
  for (int i = threadIdx.x; i < NP * ND; i += blockDim.x) { sChi[i] = tab.SChi[i]; sdChi[i] = tab.SdChi[i]; }
  for (int i = threadIdx.x; i < 3 * NQ; i += blockDim.x) sK[i] = tab.SK[i];
  for (int i = threadIdx.x; i < NF * NP; i += blockDim.x) { sLf[i] = tab.Lf[i]; sBfT[i] = tab.BfT[i]; }

  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *src = c + (size_t)e0 * M * NP;
    for (int i = threadIdx.x; i < EB * M * NP; i += blockDim.x)
      sC[i] = i < ecount * M * NP ? src[i] : 0.0;
    for (int i = threadIdx.x; i < EB * NF; i += blockDim.x) {
      const int el = i / NF, qk = i - el * NF;
      double v[M] = {0.0, 0.0, 0.0, 0.0};
      if (el < ecount) {
        const int q = qk / NE, k = qk - q * NE;
        const int ef = elem_face[(size_t)(e0 + el) * 3 + q];
        const int f = ef >> 1, side = ef & 1;
        const double *fp = fhat + ((size_t)f * NE + (side ? NE - 1 - k : k)) * M;
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = side ? fp[m] : tc::neg_bits(fp[m]);
      }
#pragma unroll
      for (int m = 0; m < M; ++m) sF[i * M + m] = v[m];
    }
    __syncthreads();

    // W(a, ib) = sum over the modes with first index a of chi_j(beta_ib) c_j
    for (int i = threadIdx.x; i < EB * ND * ND; i += blockDim.x) {
      const int el = i / (ND * ND), a = (i / ND) % ND, ib = i % ND;
      double w[M] = {0.0, 0.0, 0.0, 0.0};
      for (int b = 0; b <= P - a; ++b) {
        const int d = a + b, j = d * (d + 1) / 2 + b;
        const double x = sChi[j * ND + ib];
#pragma unroll
        for (int m = 0; m < M; ++m) w[m] += x * sC[(el * M + m) * NP + j];
      }
#pragma unroll
      for (int m = 0; m < M; ++m) sX[i * 8 + m] = w[m];
    }
    __syncthreads();

    // volume points: U = sum_a P_a W; Euler flux; Ha, Hb
    for (int i = threadIdx.x; i < EB * NQ; i += blockDim.x) {
      const int el = i / NQ, k = i - el * NQ, ib = k / ND, ia = k - ib * ND;
      double U[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        const double pa = sPa[a * ND + ia];
        const double *w = sX + ((el * ND + a) * ND + ib) * 8;
#pragma unroll
        for (int m = 0; m < M; ++m) U[m] += pa * w[m];
      }
      double Ha[M], Hb[M];
      if (el < ecount) {
        const double *g = geo + (size_t)(e0 + el) * GEO;
        const double ka = sK[k], kb = sK[NQ + k], kc = sK[2 * NQ + k];
        // (Ha, Hb) = (ka G_r + kb G_s, kc G_s) with (G_r, G_s) = J^tau (F1, F2)
        const double A1 = ka * g[0] + kb * g[2], A2 = ka * g[1] + kb * g[3];
        const double B1 = kc * g[2], B2 = kc * g[3];
        const double inv = recip(U[0]);
        const double u = U[1] * inv, v = U[2] * inv;
        const double p = (gamma - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));
        if (!(positive_finite(U[0]) & positive_finite(p))) atomicOr(err, kErrNonPhysical);
        double F1[M], F2[M];
        F1[0] = U[1];           F2[0] = U[2];
        F1[1] = U[1] * u + p;   F2[1] = U[1] * v;
        F1[2] = U[2] * u;       F2[2] = U[2] * v + p;
        F1[3] = (U[3] + p) * u; F2[3] = (U[3] + p) * v;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          Ha[m] = A1 * F1[m] + A2 * F2[m];
          Hb[m] = B1 * F1[m] + B2 * F2[m];
        }
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) { Ha[m] = 0.0; Hb[m] = 0.0; }
      }
      double *h = sH + (size_t)i * 8;
#pragma unroll
      for (int m = 0; m < M; ++m) { h[m] = Ha[m]; h[4 + m] = Hb[m]; }
    }
    __syncthreads();

    // Xa(a, ib) = sum_ia Ha P_a', Xb(a, ib) = sum_ia Hb P_a
    for (int i = threadIdx.x; i < EB * ND * ND; i += blockDim.x) {
      const int el = i / (ND * ND), a = (i / ND) % ND, ib = i % ND;
      double xa[M] = {0.0, 0.0, 0.0, 0.0}, xb[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int ia = 0; ia < ND; ++ia) {
        const double dp = sdPa[a * ND + ia], pa = sPa[a * ND + ia];
        const double *h = sH + ((el * NQ) + ib * ND + ia) * 8;
#pragma unroll
        for (int m = 0; m < M; ++m) { xa[m] += h[m] * dp; xb[m] += h[4 + m] * pa; }
      }
      double *x = sX + (size_t)i * 8;
#pragma unroll
      for (int m = 0; m < M; ++m) { x[m] = xa[m]; x[4 + m] = xb[m]; }
    }
    __syncthreads();

    // modes: V_j + lifted edge fluxes, 1/det J, stage update
    for (int i = threadIdx.x; i < EB * NP; i += blockDim.x) {
      const int el = i / NP, j = i - el * NP, a = mode_a(j);
      double acc[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int ib = 0; ib < ND; ++ib) {
        const double ch = sChi[j * ND + ib], dch = sdChi[j * ND + ib];
        const double *x = sX + ((el * ND + a) * ND + ib) * 8;
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] += ch * x[m] + dch * x[4 + m];
      }
#pragma unroll
      for (int qk = 0; qk < NF; ++qk) {
        const double *fv = sF + (el * NF + qk) * M;
        const double l = sLf[qk * NP + j];
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] += fv[m] * l;
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
      // the new state, for the next stage's traces (sH is free: every thread has
      // passed the barrier after the X phase, the last reader of sH)
#pragma unroll
      for (int m = 0; m < M; ++m) sO[(el * M + m) * NP + j] = nv[m];
    }

    if (trace_out) {
      __syncthreads();
      for (int i = threadIdx.x; i < ecount * NF; i += blockDim.x) {
        const int el = i / NF, qk = i - el * NF;
        double T[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const double b = sBfT[j * NF + qk];
#pragma unroll
          for (int m = 0; m < M; ++m) T[m] += sO[(el * M + m) * NP + j] * b;
        }
        double *dst = trace_out + ((size_t)(e0 + el) * NF + qk) * M;
#pragma unroll
        for (int m = 0; m < M; ++m) dst[m] = T[m];
      }
    }
  }
}


template <int P, int NE>
int run_element_sf(const dg_mesh *m, const double *c, const double *u0, double *out, double *trace_out,
                   const double *fhat, const StageUpdate &su, int mode, cudaStream_t s) {
  using S = SfCfg<P, NE>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_element_sf<P, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_element_sf<P, NE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr_set = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_element_sf<P, NE>, kThreads, S::SMEM);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const int ntiles = (int)((m->N + S::EB - 1) / S::EB);
  const int grid = ntiles < m->num_sms * per_sm ? ntiles : m->num_sms * per_sm;
  k_element_sf<P, NE><<<grid, kThreads, S::SMEM, s>>>(c, u0, out, trace_out, fhat, m->geo, m->elem_face, m->tab,
                                                      (int)m->N, su, mode, m->gamma, m->err_flag);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_element(const dg_mesh *m, const double *c, const double *u0, double *out, double *trace_out,
                   const double *fhat, const StageUpdate &su, int mode, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
#define CALL(P, NE) run_element_sf<P, NE>(m, c, u0, out, trace_out, fhat, su, mode, s)
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
