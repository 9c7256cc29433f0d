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
 *   k_element_sf  (dg_element.cu) one CTA per tile of EB elements, staged through shared memory:
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
#include "dg_limiter.cuh"

namespace dg {
namespace {

// ---------------------------------------------------------------------------
// edge traces of a coefficient array: trace[e][q*NE+k][m] = sum_j c[e][m][j] phi_j(r_{q,k}),
// by the same factorised sums (face_sums, edge_traces_unit) as the element kernel's epilogue
// ---------------------------------------------------------------------------
template <int P, int NE>
__global__ void __launch_bounds__(kThreads)
k_traces(const double *__restrict__ c, double *__restrict__ trace, const double *__restrict__ EPa,
         const double *__restrict__ EChiM1, const double *__restrict__ EChi, int N, double *__restrict__ copy) {
  using C = Cfg<P, NE>;
  constexpr int NP = C::NP, ND = C::ND, NF = C::NF, EB = C::EB;
  __shared__ double sPa[ND * NE], sChiM1[NP], sChi[NP * NE];
  __shared__ double sC[EB * M * NP];
  __shared__ double sZ[EB * M * (ND + 1)];
  for (int i = threadIdx.x; i < NP * NE; i += blockDim.x) sChi[i] = EChi[i];
  for (int i = threadIdx.x; i < ND * NE; i += blockDim.x) sPa[i] = EPa[i];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sChiM1[i] = EChiM1[i];
  const int ntiles = (N + EB - 1) / EB;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    __syncthreads();
    const double *src = c + (size_t)e0 * M * NP;
    for (int i = threadIdx.x; i < EB * M * NP; i += blockDim.x)
      sC[i] = i < ecount * M * NP ? src[i] : 0.0;
    __syncthreads();
    // (c in host memory the device can reach: the device copy the steps run on)
    if (copy)
      for (int i = threadIdx.x; i < ecount * M * NP; i += blockDim.x) copy[(size_t)e0 * M * NP + i] = sC[i];
    // Z_a of face 0, once per (element, variable), as the element kernel forms them
    for (int i = threadIdx.x; i < ecount * M; i += blockDim.x) {
      double z[ND + 1];
      face_sums<P>(sC + i * NP, sChiM1, sChi[0], z);
#pragma unroll
      for (int a = 0; a <= ND; ++a) sZ[i * (ND + 1) + a] = z[a];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ecount * M * NE; i += blockDim.x) {
      const int el = i / (M * NE), m = (i / NE) % M, k = i % NE;
      const double *cj = sC + (el * M + m) * NP;
      double t0, t1, t2;
      edge_traces_unit<P, NE>(cj, sZ + (el * M + m) * (ND + 1), sPa, sChi, k, t0, t1, t2);
      double *dst = trace + (size_t)(e0 + el) * NF * M + m;
      dst[k * M] = t0;
      dst[(NE + k) * M] = t1;
      dst[(3 * NE - 1 - k) * M] = t2;
    }
  }
}

// ---------------------------------------------------------------------------
// edge flux: fhat[f][k][m] = l_f * F_hat(U_l(r_{L,k}), U_r(r_{R,NE-1-k}), n_f)
// ---------------------------------------------------------------------------
template <int NE>
__global__ void __launch_bounds__(kThreads)
k_face(const double *__restrict__ trace, double *__restrict__ fhat, const FaceConn *__restrict__ conn,
       const FaceGeo *__restrict__ fg, const double *__restrict__ bstate, int64_t N, int64_t F, double gamma,
       int *err) {
  face_flux_points<NE>(trace, fhat, conn, fg, bstate, N, F, gamma, err, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// projection of point data and volume point coordinates
// ---------------------------------------------------------------------------
template <int P, int NQ>
__global__ void __launch_bounds__(kThreads)
k_project(const double *__restrict__ u, double *__restrict__ c, const double *__restrict__ Pw, int N) {
  constexpr int NP = (P + 1) * (P + 2) / 2;
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

// out[e][k][m] = sum_j c[e][m][j] tab[k][j] for npts points
__global__ void __launch_bounds__(kThreads)
k_eval_points(const double *__restrict__ c, const double *__restrict__ tab, double *__restrict__ out, int N,
              int np, int npts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)N * npts) return;
  const int64_t e = i / npts;
  const int k = (int)(i - e * npts);
  const double *ce = c + (size_t)e * M * np;
  const double *t = tab + (size_t)k * np;
  double u[M] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < np; ++j) {
    const double b = t[j];
#pragma unroll
    for (int m = 0; m < M; ++m) u[m] += ce[m * np + j] * b;
  }
#pragma unroll
  for (int m = 0; m < M; ++m) out[i * M + m] = u[m];
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
// conserved totals: fixed-order reduction of det J * c[e][m][0] -- per thread
// over a strided range, then warp shuffles, then across the warps of the block,
// then one block over the block partials.  The order never depends on timing,
// so repeated calls give the same bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_sum4(double acc[M]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += __shfl_down_sync(0xFFFFFFFFu, acc[m], off);
}

// lane 0 of warp 0 ends with the block sum of acc
__device__ __forceinline__ void block_sum4(double acc[M]) {
  __shared__ double red[kThreads / 32][M];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum4(acc);
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) red[warp][m] = acc[m];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = lane < kThreads / 32 ? red[lane][m] : 0.0;
    warp_sum4(acc);
  }
}

__global__ void __launch_bounds__(kThreads)
k_totals_partial(const double *__restrict__ c, const double *__restrict__ geo, int N, int np,
                 double *__restrict__ partial) {
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  const int64_t chunk = ((int64_t)N + gridDim.x - 1) / gridDim.x;
  const int64_t beg = blockIdx.x * chunk;
  const int64_t end = min((int64_t)N, beg + chunk);
  for (int64_t e = beg + threadIdx.x; e < end; e += blockDim.x) {
    const double dj = geo[e * GEO + 5];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += dj * c[(e * M + m) * np];
  }
  block_sum4(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) partial[blockIdx.x * M + m] = acc[m];
}

__global__ void __launch_bounds__(kThreads)
k_totals_final(const double *__restrict__ partial, int nb, double *__restrict__ out) {
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] += partial[b * M + m];
  block_sum4(acc);
  // int phi_1 over the reference triangle is 1/sqrt(2); the other modes have zero mean
  if (threadIdx.x == 0)
#pragma unroll
    for (int m = 0; m < M; ++m) out[m] = acc[m] * 0.70710678118654752440;
}

// ---------------------------------------------------------------------------
// element geometry for callers: det J of every element, physical points of a
// reference rule, and the L2 error of one variable against given point values
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_det_j(const double *__restrict__ geo, double *__restrict__ out, int64_t N) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N) out[e] = geo[e * GEO + 5];
}

// x(r, s) = x1 (1 - r - s) + x2 r + x3 s (Eq. 2dmap) at npts points per element
__global__ void __launch_bounds__(kThreads)
k_map_points(const double *__restrict__ xy, const double *__restrict__ rs, double *__restrict__ out, int64_t N,
             int npts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * npts) return;
  const int64_t e = i / npts;
  const int k = (int)(i - e * npts);
  const double *v = xy + e * 6;
  const double r = rs[2 * k], s = rs[2 * k + 1], l0 = 1.0 - r - s;
  out[i * 2 + 0] = v[0] * l0 + v[2] * r + v[4] * s;
  out[i * 2 + 1] = v[1] * l0 + v[3] * r + v[5] * s;
}

// per block: sum over its elements' points of det J w_k (U_h(r_k) - exact_k)^2 for
// one variable; tab = [npts][np] basis values, w = [npts] weights (device)
__global__ void __launch_bounds__(kThreads)
k_l2_partial(const double *__restrict__ c, const double *__restrict__ exact, const double *__restrict__ tab,
             const double *__restrict__ w, const double *__restrict__ geo, int64_t N, int np, int npts, int var,
             double *__restrict__ partial) {
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  const int64_t n = N * npts;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = blockIdx.x * chunk;
  const int64_t end = min(n, beg + chunk);
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const int64_t e = i / npts;
    const int k = (int)(i - e * npts);
    const double *ce = c + ((size_t)e * M + var) * np;
    const double *t = tab + (size_t)k * np;
    double u = 0.0;
    for (int j = 0; j < np; ++j) u = fma(ce[j], t[j], u);
    const double d = u - exact[(size_t)i * M + var];
    acc[0] = fma(geo[e * GEO + 5] * w[k], d * d, acc[0]);
  }
  block_sum4(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc[0];
}

__global__ void __launch_bounds__(kThreads)
k_l2_final(const double *__restrict__ partial, int nb, double *__restrict__ out) {
  double acc[M] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc[0] += partial[b];
  block_sum4(acc);
  if (threadIdx.x == 0) out[0] = sqrt(acc[0]);
}

// ---------------------------------------------------------------------------
// largest wave speed |v| + c over the volume points (max is exact, so the result
// does not depend on the order)
// ---------------------------------------------------------------------------
template <int P, int NQ>
__global__ void __launch_bounds__(kThreads)
k_wave_partial(const double *__restrict__ c, const double *__restrict__ BvT, int N, double gamma,
               double *__restrict__ partial, int *err) {
  constexpr int NP = (P + 1) * (P + 2) / 2;
  __shared__ double red[kThreads / 32];
  double smax = 0.0;
  const int64_t chunk = ((int64_t)N * NQ + gridDim.x - 1) / gridDim.x;
  const int64_t beg = blockIdx.x * chunk;
  const int64_t end = min((int64_t)N * NQ, beg + chunk);
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    const int64_t e = i / NQ;
    const int k = (int)(i - e * NQ);
    const double *ce = c + (size_t)e * M * NP;
    double U[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const double b = BvT[j * NQ + k];
#pragma unroll
      for (int m = 0; m < M; ++m) U[m] += ce[m * NP + j] * b;
    }
    const double inv = recip(U[0]);
    const double u = U[1] * inv, v = U[2] * inv;
    const double p = (gamma - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));
    if (!(U[0] > 0.0 && p > 0.0)) {
      atomicOr(err, kErrNonPhysical);
      continue;
    }
    smax = fmax(smax, sqrt(u * u + v * v) + sqrt(gamma * p * inv));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) smax = fmax(smax, __shfl_down_sync(0xFFFFFFFFu, smax, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) b = fmax(b, red[w]);
    partial[blockIdx.x] = b;
  }
}

__global__ void k_wave_final(const double *__restrict__ partial, int nb, double *__restrict__ out) {
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int i = 0; i < nb; ++i) b = fmax(b, partial[i]);
    out[0] = b;
  }
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
// Barth-Jespersen limiter for p = 1 (Section 4.3.5), in place on c: the items of
// limit_p1_items (dg_limiter.cuh) over the grid.
// ---------------------------------------------------------------------------
template <bool HAVE_TRACES>
__global__ void __launch_bounds__(kThreads)
k_limit_p1(double *c, double *__restrict__ trace, const int32_t *__restrict__ elem_nbr,
           const double *__restrict__ EPa, const double *__restrict__ EChiM1, const double *__restrict__ EChi,
           double phi1, int64_t N, int *err) {
  limit_p1_items<HAVE_TRACES>(c, trace, elem_nbr, EPa, EChiM1, EChi, phi1, N, err, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int P, int NE>
int run_traces(const dg_mesh *m, const double *c, double *trace, double *copy, cudaStream_t s) {
  using C = Cfg<P, NE>;
  const int ntiles = (int)((m->N + C::EB - 1) / C::EB);
  const int grid = ntiles < m->num_sms * 4 ? ntiles : m->num_sms * 4;
  k_traces<P, NE><<<grid, kThreads, 0, s>>>(c, trace, m->tab.EPa, m->tab.EChiM1, m->tab.EChi, (int)m->N, copy);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_traces(const dg_mesh *m, const double *c, double *trace, void *stream, double *copy) {
  cudaStream_t s = (cudaStream_t)stream;
#define CALL(P, NE) run_traces<P, NE>(m, c, trace, copy, s)
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaErrorInvalidValue;
}

// blocks of `threads` threads needed for n items, at most what is resident on
// the GPU at once (a grid-stride kernel covers the rest); per_sm is the kernel's
// resident blocks per SM (0: ask the occupancy calculator)
int resident_grid(const dg_mesh *m, const void *kernel, int threads, int64_t n, int *per_sm) {
  if (*per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    *per_sm = v;
  }
  const int64_t need = (n + threads - 1) / threads, cap = (int64_t)m->num_sms * *per_sm;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

int launch_limit(const dg_mesh *m, double *c, double *trace, int have_traces, void *stream) {
  if (m->p != 1 || m->ne != 2) return (int)cudaErrorInvalidValue;
  if (have_traces && !trace) return (int)cudaErrorInvalidValue;
  static int per_sm[2] = {0, 0};
  cudaStream_t s = (cudaStream_t)stream;
  if (have_traces)
    k_limit_p1<true><<<resident_grid(m, (const void *)k_limit_p1<true>, kThreads, m->N * M, &per_sm[1]), kThreads,
                        0, s>>>(c, trace, m->elem_nbr, m->tab.EPa, m->tab.EChiM1, m->tab.EChi, m->phi1, m->N,
                                m->err_flag);
  else
    k_limit_p1<false><<<resident_grid(m, (const void *)k_limit_p1<false>, kThreads, m->N * M, &per_sm[0]), kThreads,
                         0, s>>>(c, trace, m->elem_nbr, m->tab.EPa, m->tab.EChiM1, m->tab.EChi, m->phi1, m->N,
                                 m->err_flag);
  return (int)cudaGetLastError();
}

int launch_face_flux(const dg_mesh *m, const double *trace, double *fhat, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = m->F * m->ne;
#define FACE(NE)                                                                                        \
  do {                                                                                                  \
    static int per_sm = 0;                                                                              \
    k_face<NE><<<resident_grid(m, (const void *)k_face<NE>, kThreads, n, &per_sm), kThreads, 0, s>>>(   \
        trace, fhat, m->face_conn, m->face_geo, m->bstate, m->N, m->F, m->gamma, m->err_flag);          \
  } while (0)
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

int launch_project(const dg_mesh *m, const double *u, double *c, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = m->N * m->np;
  const int grid = (int)((n + kThreads - 1) / kThreads);
#define PROJ(P)                                                                                       \
  (m->rule == DG_RULE_SYMMETRIC ? k_project<P, sym_points(P)><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N) \
                                : k_project<P, (P + 1) * (P + 1)><<<grid, kThreads, 0, s>>>(u, c, m->tab.Pw, (int)m->N))
  switch (m->p) {
    case 1: PROJ(1); break;
    case 2: PROJ(2); break;
    case 3: PROJ(3); break;
    case 4: PROJ(4); break;
    case 5: PROJ(5); break;
    default: return (int)cudaErrorInvalidValue;
  }
#undef PROJ
  return (int)cudaGetLastError();
}

int launch_eval_points(const dg_mesh *m, const double *c, const double *tab, int npts, double *out, void *stream) {
  const int64_t n = m->N * (int64_t)npts;
  k_eval_points<<<(int)((n + kThreads - 1) / kThreads), kThreads, 0, (cudaStream_t)stream>>>(c, tab, out, (int)m->N,
                                                                                            m->np, npts);
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

int launch_wave_speed(const dg_mesh *m, const double *c, double *out_dev, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = m->totals_blocks;
#define WAVE(P)                                                                                        \
  (m->rule == DG_RULE_SYMMETRIC                                                                        \
       ? k_wave_partial<P, sym_points(P)><<<nb, kThreads, 0, s>>>(c, m->tab.BvT, (int)m->N, m->gamma,      \
                                                                  m->partial, m->err_flag)             \
       : k_wave_partial<P, (P + 1) * (P + 1)><<<nb, kThreads, 0, s>>>(c, m->tab.BvT, (int)m->N, m->gamma, \
                                                                      m->partial, m->err_flag))
  switch (m->p) {
    case 1: WAVE(1); break;
    case 2: WAVE(2); break;
    case 3: WAVE(3); break;
    case 4: WAVE(4); break;
    case 5: WAVE(5); break;
    default: return (int)cudaErrorInvalidValue;
  }
#undef WAVE
  k_wave_final<<<1, 32, 0, s>>>(m->partial, nb, out_dev);
  return (int)cudaGetLastError();
}

int launch_det_j(const dg_mesh *m, double *out, void *stream) {
  k_det_j<<<(int)((m->N + kThreads - 1) / kThreads), kThreads, 0, (cudaStream_t)stream>>>(m->geo, out, m->N);
  return (int)cudaGetLastError();
}

int launch_map_points(const dg_mesh *m, const double *rs, int npts, double *out, void *stream) {
  const int64_t n = m->N * npts;
  k_map_points<<<(int)((n + kThreads - 1) / kThreads), kThreads, 0, (cudaStream_t)stream>>>(m->xy, rs, out, m->N,
                                                                                           npts);
  return (int)cudaGetLastError();
}

int launch_l2_error(const dg_mesh *m, const double *c, const double *exact, const double *tab, const double *w,
                    int npts, int var, double *partial, int nb, double *out_dev, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_l2_partial<<<nb, kThreads, 0, s>>>(c, exact, tab, w, m->geo, m->N, m->np, npts, var, partial);
  k_l2_final<<<1, kThreads, 0, s>>>(partial, nb, out_dev);
  return (int)cudaGetLastError();
}

int launch_totals(const dg_mesh *m, const double *c, double *out_dev, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_totals_partial<<<m->totals_blocks, kThreads, 0, s>>>(c, m->geo, (int)m->N, m->np, m->partial);
  k_totals_final<<<1, kThreads, 0, s>>>(m->partial, m->totals_blocks, out_dev);
  return (int)cudaGetLastError();
}

}  // namespace dg
