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
        double b1[M], b2[M], o1[M], o2[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          b1[m] = ar[m] * g[0] + as[m] * g[2];
          b2[m] = ar[m] * g[1] + as[m] * g[3];
        }
        flux_jac_t(U, 1.0, 0.0, gamma, b1, o1);
        flux_jac_t(U, 0.0, 1.0, gamma, b2, o2);
#pragma unroll
        for (int m = 0; m < M; ++m) ub[m] = o1[m] + o2[m];
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
       : run_adj<P, NE, 0>(m, u, lam, uvol, G, T, TB, X, Y, Z, x0, x1, x2, s, out, st))
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
