/*
 * dg_kernels.cu -- float64 kernels of the DG right-hand side and SSP-RK3 stage
 * on sm_103a.
 *
 * One stage of the method (the paper's Section 4.3: volume kernel, edge kernel,
 * combining kernel) is organised here as two launches:
 *
 *   k_face     one thread per (edge, edge point): gathers the two traces, the
 *              right element's at the reversed point (Eq. edgeint), evaluates the
 *              local Lax-Friedrichs flux once per edge and stores it scaled by the
 *              edge Jacobian l = |edge|/2 (Eq. len).
 *   k_element_sf  one CTA per tile of EB elements, staged through shared memory:
 *              interpolation to the volume points, Euler flux and the reference
 *              flux G = J^tau F, projection onto the weighted basis gradients
 *              (Eq. volume, Algorithm 1) -- both sum-factorised on the collapsed
 *              volume grid -- lifting of the three edge fluxes (Algorithm 3),
 *              scaling by 1/det J (Eq. 2ddg0), the Runge-Kutta stage update, and,
 *              for the next stage, the edge traces of the new state.  Writing the
 *              traces from the element that owns the state replaces a separate
 *              pass over the coefficients.
 *
 * The paper's per-edge temporaries (rhs_surface_left/right) become one flux
 * block per edge; each element gathers its three blocks, so no atomics are used
 * and every result is deterministic.
 */
#include <cuda_runtime.h>

#include <cstdint>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

// ---------------------------------------------------------------------------
// edge traces of a coefficient array: trace[e][q*NE+k][m] = sum_j c[e][m][j] phi_j(r_{q,k})
// ---------------------------------------------------------------------------
template <int P, int NE>
__global__ void __launch_bounds__(kThreads)
k_traces(const double *__restrict__ c, double *__restrict__ trace, const double *__restrict__ BfT,
         int N) {
  using C = Cfg<P, NE>;
  constexpr int NP = C::NP, NF = C::NF, EB = C::EB;
  __shared__ double sB[NP * NF];
  __shared__ double sC[EB * M * NP];
  for (int i = threadIdx.x; i < NP * NF; i += blockDim.x) sB[i] = BfT[i];
  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *src = c + (size_t)e0 * M * NP;
    for (int i = threadIdx.x; i < EB * M * NP; i += blockDim.x)
      sC[i] = i < ecount * M * NP ? src[i] : 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < ecount * NF; i += blockDim.x) {
      const int el = i / NF, qk = i - el * NF;
      double T[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const double b = sB[j * NF + qk];
#pragma unroll
        for (int m = 0; m < M; ++m) T[m] += sC[(el * M + m) * NP + j] * b;
      }
      double *dst = trace + ((size_t)(e0 + el) * NF + qk) * M;
#pragma unroll
      for (int m = 0; m < M; ++m) dst[m] = T[m];
    }
  }
}

// ---------------------------------------------------------------------------
// edge flux: fhat[f][k][m] = l_f * F_hat(U_l(r_{L,k}), U_r(r_{R,NE-1-k}), n_f)
// ---------------------------------------------------------------------------
template <int NE, bool FAST_ALPHA>
__global__ void __launch_bounds__(kThreads)
k_face(const double *__restrict__ trace, double *__restrict__ fhat, const FaceConn *__restrict__ conn,
       const FaceGeo *__restrict__ fg, int64_t F, double gamma) {
  constexpr int NF = 3 * NE;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F * NE) return;
  const int64_t f = i / NE;
  const int k = (int)(i - f * NE);
  const FaceConn cn = conn[f];
  const FaceGeo g = fg[f];
  const double *pl = trace + ((size_t)cn.l * NF + cn.L * NE + k) * M;
  const double *pr = trace + ((size_t)cn.r * NF + cn.R * NE + (NE - 1 - k)) * M;
  double ul[M], ur[M], Fh[M];
#pragma unroll
  for (int m = 0; m < M; ++m) { ul[m] = pl[m]; ur[m] = pr[m]; }
  // l * F_hat = (l/2) (F(Ul).n + F(Ur).n - alpha (Ur - Ul))
  lax_friedrichs_scaled<FAST_ALPHA>(ul, ur, g.nx, g.ny, gamma, 0.5 * g.hl, Fh);
  double *dst = fhat + (size_t)i * M;
#pragma unroll
  for (int m = 0; m < M; ++m) dst[m] = Fh[m];
}

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
             const int32_t *__restrict__ elem_face, DevTables tab, int N, double dt, double a0,
             double b0, int mode, double gamma) {
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
        // stage update b0 (c + dt R) + a0 u0 with R = acc / det J, as
        // b0 c + a0 u0 + (b0 dt / det J) acc
        const double kap = b0 * dt * inv;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const size_t idx = (e * M + m) * NP + j;
          double v;
          if (mode == 0) {
            v = acc[m] * inv;
          } else {
            double t = b0 * sC[(el * M + m) * NP + j];
            if (a0 != 0.0) t = fma(a0, u0[idx], t);
            v = fma(kap, acc[m], t);
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

// ---------------------------------------------------------------------------
// projection of point data and volume point coordinates
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads)
k_project(const double *__restrict__ u, double *__restrict__ c, const double *__restrict__ Pw, int N) {
  constexpr int NP = (P + 1) * (P + 2) / 2, NQ = (P + 1) * (P + 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)N * NP) return;
  const int64_t e = i / NP;
  const int j = (int)(i - e * NP);
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  const double *ue = u + (size_t)e * NQ * M;
  for (int k = 0; k < NQ; ++k) {
    const double w = Pw[k * NP + j];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += w * ue[k * M + m];
  }
#pragma unroll
  for (int m = 0; m < M; ++m) c[((size_t)e * M + m) * NP + j] = acc[m];
}

__global__ void __launch_bounds__(kThreads)
k_volume_points(const double *__restrict__ xy, const double *__restrict__ vr,
                const double *__restrict__ vs, double *__restrict__ out, int N, int nq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)N * nq) return;
  const int64_t e = i / nq;
  const int k = (int)(i - e * nq);
  const double *v = xy + e * 6;
  const double r = vr[k], s = vs[k], l0 = 1.0 - r - s;
  out[i * 2 + 0] = v[0] * l0 + v[2] * r + v[4] * s;
  out[i * 2 + 1] = v[1] * l0 + v[3] * r + v[5] * s;
}

// ---------------------------------------------------------------------------
// conserved totals: fixed-order two-pass reduction of det J * c[e][m][0]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_totals_partial(const double *__restrict__ c, const double *__restrict__ geo, int N, int np,
                 double *__restrict__ partial) {
  __shared__ double red[M][kThreads];
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  const int64_t chunk = ((int64_t)N + gridDim.x - 1) / gridDim.x;
  const int64_t beg = blockIdx.x * chunk;
  const int64_t end = min((int64_t)N, beg + chunk);
  for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const double dj = geo[e * GEO + 5];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += dj * c[(e * M + m) * np];
  }
#pragma unroll
  for (int m = 0; m < M; ++m) red[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int m = 0; m < M; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < M) partial[blockIdx.x * M + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(kThreads)
k_totals_final(const double *__restrict__ partial, int nb, double *__restrict__ out) {
  __shared__ double red[M][kThreads];
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += partial[b * M + m];
#pragma unroll
  for (int m = 0; m < M; ++m) red[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int m = 0; m < M; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + s];
    __syncthreads();
  }
  // int phi_1 over the reference triangle is 1/sqrt(2); the other modes have zero mean
  if (threadIdx.x < M) out[threadIdx.x] = red[threadIdx.x][0] * 0.70710678118654752440;
}

// ---------------------------------------------------------------------------
// FMA-rate probe: 8 independent dependency chains per thread, all in registers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, double *out) {
  const T x = (T)(1.0 + 1e-7 * threadIdx.x), y = (T)(1e-9 * blockIdx.x);
  T acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = fma(acc[i], x, y);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += acc[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int P, int NE>
int run_element_sf(const dg_mesh *m, const double *c, const double *u0, double *out, double *trace_out,
                   const double *fhat, double dt, double a0, double b0, int mode, cudaStream_t s) {
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
                                                      (int)m->N, dt, a0, b0, mode, m->gamma);
  return (int)cudaGetLastError();
}

template <int P, int NE>
int run_traces(const dg_mesh *m, const double *c, double *trace, cudaStream_t s) {
  using C = Cfg<P, NE>;
  const int ntiles = (int)((m->N + C::EB - 1) / C::EB);
  const int grid = ntiles < m->num_sms * 4 ? ntiles : m->num_sms * 4;
  k_traces<P, NE><<<grid, kThreads, 0, s>>>(c, trace, m->tab.BfT, (int)m->N);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_traces(const dg_mesh *m, const double *c, double *trace, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
#define CALL(P, NE) run_traces<P, NE>(m, c, trace, s)
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaErrorInvalidValue;
}

int launch_face_flux(const dg_mesh *m, const double *trace, double *fhat, void *stream, bool fast_alpha) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = m->F * m->ne;
  const int grid = (int)((n + kThreads - 1) / kThreads);
#define FACE(NE)                                                                                      \
  (fast_alpha ? (k_face<NE, true><<<grid, kThreads, 0, s>>>(trace, fhat, m->face_conn, m->face_geo, m->F, m->gamma), 0) \
              : (k_face<NE, false><<<grid, kThreads, 0, s>>>(trace, fhat, m->face_conn, m->face_geo, m->F, m->gamma), 0))
  switch (m->ne) {
    case 2: FACE(2); break;
    case 3: FACE(3); break;
    case 4: FACE(4); break;
    case 5: FACE(5); break;
    case 6: FACE(6); break;
    default: return (int)cudaErrorInvalidValue;
  }
#undef FACE
  return (int)cudaGetLastError();
}

int launch_element(const dg_mesh *m, const double *c, const double *u0, double *out, double *trace_out,
                   const double *fhat, double dt, double a0, double b0, int mode, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
#define CALL(P, NE) run_element_sf<P, NE>(m, c, u0, out, trace_out, fhat, dt, a0, b0, mode, s)
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaErrorInvalidValue;
}

int launch_project(const dg_mesh *m, const double *u, double *c, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = m->N * m->np;
  const int grid = (int)((n + kThreads - 1) / kThreads);
  switch (m->p) {
    case 1: k_project<1><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N); break;
    case 2: k_project<2><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N); break;
    case 3: k_project<3><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N); break;
    case 4: k_project<4><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N); break;
    case 5: k_project<5><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_volume_points(const dg_mesh *m, double *xy, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = m->N * m->nq;
  const int grid = (int)((n + kThreads - 1) / kThreads);
  k_volume_points<<<grid, kThreads, 0, s>>>(m->xy, m->tab.vr, m->tab.vs, xy, (int)m->N, m->nq);
  return (int)cudaGetLastError();
}

int launch_fma_probe(int fp64, int blocks, int threads, int iters, double *out, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (threads != kThreads) return (int)cudaErrorInvalidValue;
  if (fp64) k_fma_probe<double><<<blocks, threads, 0, s>>>(iters, out);
  else k_fma_probe<float><<<blocks, threads, 0, s>>>(iters, out);
  return (int)cudaGetLastError();
}

int launch_totals(const dg_mesh *m, const double *c, double *out_dev, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_totals_partial<<<m->totals_blocks, kThreads, 0, s>>>(c, m->geo, (int)m->N, m->np, m->partial);
  k_totals_final<<<1, kThreads, 0, s>>>(m->partial, m->totals_blocks, out_dev);
  return (int)cudaGetLastError();
}

}  // namespace dg
