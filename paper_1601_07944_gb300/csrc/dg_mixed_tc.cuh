/*
 * dg_mixed_tc.cuh -- the mixed-precision element kernel k_element_tc and its
 * launcher, included by the translation units that instantiate it: dg_mixed.cu
 * for the collapsed volume grid, dg_mixed_sym.cu for the symmetric rules (two
 * units, so that the two sets of instantiations compile in parallel).
 *
 * A tile is 32 elements = 128 accumulator rows, row r = 4 e + m (element e,
 * variable m).  Per tile:
 *   GEMM 1  U[128 x NQ]   = C[128 x NP] Phi[NP x NQ]            interpolation
 *           FP32 Euler flux and G = J^tau F at every volume point (SIMT)
 *   GEMM 2  D[128 x NP]   = [G_r | G_s | F_hat] [Dr; Ds; Lf]     projection on
 *           the weighted basis gradients and lifting of the edge fluxes, one
 *           accumulation (the paper's volume and surface terms, Algorithms 1-3)
 *           FP64: the mean mode's lift (the volume term of mode 1 vanishes), the
 *           1/det J scaling and the Runge-Kutta stage update
 *   GEMM 3  T[128 x NF]   = C_new[128 x NP] Phi_f[NP x NF]       next edge traces
 * (mode 2 runs GEMM 3 alone on the stage input: the first stage's traces.)
 * The volume rule enters only through its point count Q (0: the collapsed
 * (p+1)^2 grid) and the tables Phi, Dr, Ds built for it on the host.
 */
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dg_device.cuh"
#include "dg_internal.h"
#include "dg_tcgen05.cuh"

namespace dg {
namespace {

constexpr int pad8(int x) { return (x + 7) / 8 * 8; }
constexpr int pad16(int x) { return (x + 15) / 16 * 16; }
constexpr int align1k(int x) { return (x + 1023) / 1024 * 1024; }
constexpr int kTcThreads = 128;
constexpr int kTmemCols = 64;
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s per MMA batch before giving up

template <int P, int NE, bool X3, int Q>
struct Tc {
  using C = Cfg<P, NE, Q>;
  static constexpr int NP = C::NP, NQ = C::NQ, NF = C::NF;
  static constexpr int EB = 32, ROWS = 128;
  static constexpr int K1 = pad8(NP), N1 = pad16(NQ), K2 = pad8(2 * NQ + NF), N2 = pad16(NP), N4 = pad16(NF);
  static constexpr int NS = X3 ? 2 : 1;                     // TF32 planes: hi (, lo)
  static constexpr int A1P = ROWS * K1 * 4, A2P = ROWS * K2 * 4;
  static constexpr int B1P = N1 * K1 * 4, B2P = N2 * K2 * 4, B4P = N4 * K1 * 4;
  static constexpr int oA1 = 0;
  static constexpr int oA2 = align1k(oA1 + A1P * NS);
  static constexpr int oB1 = align1k(oA2 + A2P * NS);
  static constexpr int oB2 = align1k(oB1 + B1P * NS);
  static constexpr int oB4 = align1k(oB2 + B2P * NS);
  static constexpr int endB = align1k(oB4 + B4P * NS);
  static constexpr int SU = EB * NQ * M * 4;                 // float [EB][NQ][M]
  static constexpr bool U_IN_A1 = SU <= A1P * NS;            // reuse GEMM 1's A planes
  static constexpr int oU = U_IN_A1 ? oA1 : endB;
  static constexpr int oJ = U_IN_A1 ? endB : endB + SU;      // float [EB][4]  J^tau
  static constexpr int oBar = oJ + EB * 16;                  // mbarrier, TMEM slot
  static constexpr int SMEM = oBar + 16;
  // the new state and the new traces are staged for coalesced stores in GEMM 2's
  // A planes, which are free once GEMM 2 has completed
  static_assert(EB * M * NP * 8 <= A2P * NS && EB * NF * M * 4 <= A2P * NS, "staging");
  static_assert(N1 <= kTmemCols && N2 <= kTmemCols && N4 <= kTmemCols, "TMEM columns");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// writes v (rounded to TF32, and its TF32 remainder for the split product) at
// (row, k) of a K-major operand with ktot columns
template <bool X3>
__device__ __forceinline__ void put_at(unsigned char *base, int plane_bytes, int off, float v) {
  const float hi = tc::to_tf32(v);
  *reinterpret_cast<float *>(base + off) = hi;
  if (X3) *reinterpret_cast<float *>(base + plane_bytes + off) = tc::to_tf32(v - hi);
}
template <bool X3>
__device__ __forceinline__ void put(unsigned char *base, int plane_bytes, int row, int k, int ktot, float v) {
  put_at<X3>(base, plane_bytes, tc::kmaj(row, k, ktot), v);
}

// D (TMEM) = sum over k-steps of A B^T, split products when X3
template <bool X3, int KT>
__device__ __forceinline__ void gemm(uint32_t d, uint32_t a, int a_plane, uint32_t b, int b_plane, uint32_t idesc) {
#pragma unroll
  for (int s = 0; s < KT / 8; ++s) {
    const uint32_t off = (uint32_t)s * 256u;
    if (X3) {
      tc::mma_tf32(d, tc::desc(a + a_plane + off, KT), tc::desc(b + off, KT), idesc, s > 0 ? 1u : 0u);
      tc::mma_tf32(d, tc::desc(a + off, KT), tc::desc(b + b_plane + off, KT), idesc, 1u);
      tc::mma_tf32(d, tc::desc(a + off, KT), tc::desc(b + off, KT), idesc, 1u);
    } else {
      tc::mma_tf32(d, tc::desc(a + off, KT), tc::desc(b + off, KT), idesc, s > 0 ? 1u : 0u);
    }
  }
}

template <int N>
__device__ __forceinline__ void tmem_row(uint32_t taddr, float *v) {
#pragma unroll
  for (int c = 0; c < N / 16; ++c) tc::ld16(taddr + (uint32_t)(c * 16), v + c * 16);
  tc::wait_ld();
}

// float32 reference flux G = J^tau F at one point (Euler flux, Eq. euler)
__device__ __forceinline__ bool ref_flux_f32(const float U[M], const float *jt, float gamma, float Gr[M],
                                             float Gs[M]) {
  const float inv = 1.0f / U[0];
  const float u = U[1] * inv, v = U[2] * inv;
  const float p = (gamma - 1.0f) * (U[3] - 0.5f * (U[1] * u + U[2] * v));
  float F1[M], F2[M];
  F1[0] = U[1];           F2[0] = U[2];
  F1[1] = U[1] * u + p;   F2[1] = U[1] * v;
  F1[2] = U[2] * u;       F2[2] = U[2] * v + p;
  F1[3] = (U[3] + p) * u; F2[3] = (U[3] + p) * v;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    Gr[m] = jt[0] * F1[m] + jt[1] * F2[m];
    Gs[m] = jt[2] * F1[m] + jt[3] * F2[m];
  }
  return U[0] > 0.0f && p > 0.0f;      // false also for NaN
}

// OUT2: the stage also writes the classical RK4's running sum (StageUpdate::out2);
// a separate instantiation, so that the kernels without it keep their registers.
template <int P, int NE, bool X3, bool OUT2, int Q>
__global__ void __launch_bounds__(kTcThreads)
k_element_tc(const double *c, const double *u0, double *out, float *__restrict__ trace_out,
             const float *__restrict__ fhat, const double *__restrict__ fmean, const double *__restrict__ geo,
             const int32_t *__restrict__ elem_face, DevTables tab, int N, int64_t F, StageUpdate su, int mode,
             double gamma, int *err) {
  using T = Tc<P, NE, X3, Q>;
  constexpr int NP = T::NP, NQ = T::NQ, NF = T::NF, EB = T::EB;
  constexpr int K1 = T::K1, N1 = T::N1, K2 = T::K2, N2 = T::N2, N4 = T::N4;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *A1 = sm + T::oA1, *A2 = sm + T::oA2, *B1 = sm + T::oB1, *B2 = sm + T::oB2, *B4 = sm + T::oB4;
  double *sStage = reinterpret_cast<double *>(sm + T::oA2);   // after GEMM 2 only
  float *sU = reinterpret_cast<float *>(sm + T::oU);
  float *sJ = reinterpret_cast<float *>(sm + T::oJ);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + T::oBar);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + T::oBar + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t mbar = tc::smem_u32(bar);

  // ---- once per CTA: zeroed A planes, B operands (split), TMEM, mbarrier ----
  for (int i = tid; i < (T::A1P * T::NS) / 16; i += kTcThreads) reinterpret_cast<int4 *>(A1)[i] = make_int4(0, 0, 0, 0);
  for (int i = tid; i < (T::A2P * T::NS) / 16; i += kTcThreads) reinterpret_cast<int4 *>(A2)[i] = make_int4(0, 0, 0, 0);
  for (int i = tid; i < N1 * K1; i += kTcThreads) {
    const int n = i / K1, k = i - n * K1;
    const double v = (n < NQ && k < NP) ? tab.BvT[k * NQ + n] : 0.0;
    put<X3>(B1, T::B1P, n, k, K1, (float)v);
  }
  for (int i = tid; i < N2 * K2; i += kTcThreads) {
    const int n = i / K2, k = i - n * K2;
    double v = 0.0;
    if (n < NP) {
      if (k < NQ) v = tab.Dr[k * NP + n];
      else if (k < 2 * NQ) v = tab.Ds[(k - NQ) * NP + n];
      else if (k < 2 * NQ + NF) v = tab.Lf[(k - 2 * NQ) * NP + n];
    }
    put<X3>(B2, T::B2P, n, k, K2, (float)v);
  }
  for (int i = tid; i < N4 * K1; i += kTcThreads) {
    const int n = i / K1, k = i - n * K1;
    const double v = (n < NF && k < NP) ? tab.BfT[k * NF + n] : 0.0;
    put<X3>(B4, T::B4P, n, k, K1, (float)v);
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(slot), kTmemCols);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);       // this warp's 32 TMEM lanes
  const uint32_t uA1 = tc::smem_u32(A1), uA2 = tc::smem_u32(A2);
  const uint32_t uB1 = tc::smem_u32(B1), uB2 = tc::smem_u32(B2), uB4 = tc::smem_u32(B4);
  const float g32 = (float)gamma;
  const int row = tid, rel = row >> 2, rm = row & 3;                 // accumulator row = 4 e + m
  uint32_t phase = 0;

  int e0 = 0, ecount = 0;
  // GEMM 3: edge traces of the state held in A1's planes -> trace_out (float64),
  // staged through GEMM 2's A planes.  Returns false if the tensor-core wait
  // expired (recorded in *err).
  auto traces_of_A1 = [&]() -> bool {
    if (tid == 0) {
      gemm<X3, K1>(tmem, uA1, T::A1P, uB4, T::B4P, tc::idesc_tf32(128, N4));
      tc::commit(mbar);
    }
    const bool done = tc::mbar_wait(mbar, phase, kWaitNs);
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicOr(err, kErrTimeout);
      return false;
    }
    tc::fence_after_sync();
    float *sT = reinterpret_cast<float *>(sStage);
    {
      float v[N4];
      tmem_row<N4>(trow, v);
#pragma unroll
      for (int qk = 0; qk < NF; ++qk) sT[(rel * NF + qk) * M + rm] = v[qk];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // [EB][NF][M] float32 is whole float4s: NF * M is a multiple of 4
    const float4 *src4 = reinterpret_cast<const float4 *>(sT);
    float4 *dst4 = reinterpret_cast<float4 *>(trace_out + (size_t)e0 * NF * M);
    for (int i = tid; i < ecount * NF; i += kTcThreads) dst4[i] = src4[i];
    return true;
  };

  const int ntiles = (N + EB - 1) / EB;
  // Per-row inputs of a tile, loaded one tile ahead: while tile t runs through
  // its GEMMs and updates, the loads of tile t + gridDim.x are in flight.  The
  // edge-flux values depend on the edge records, so they are requested later in
  // the tile than the rest.  The second register set costs resident CTAs where
  // registers, not shared memory, bound them: at p = 5 it does not fit at all,
  // and for the 1xTF32 kernels at p = 2 and 4 (small shared memory) the CTAs it
  // displaces hide more latency than it does (measured); there the loads are
  // issued at the start of the tile itself.
  constexpr bool AHEAD = P <= 4 && (X3 || P == 3);
  struct RowIn {
    double c[NP], u[NP], s[3], inv;            // s: the three edges' mean-mode integrals
    double jt;                                 // entry rm of this row's element's J^tau
    float f[NF];
    int ef[3];
  };
  const bool need_u0 = mode == 1 && su.a0 != 0.0;
  auto load_head = [&](int t, RowIn &r) {
    const int base = t * EB;
    const bool lv = t < ntiles && rel < N - base;
    const size_t o = ((size_t)(base + rel) * M + rm) * NP;
#pragma unroll
    for (int q = 0; q < 3; ++q) r.ef[q] = lv && mode != 2 ? elem_face[(size_t)(base + rel) * 3 + q] : 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      r.c[j] = lv ? c[o + j] : 0.0;
      r.u[j] = lv && need_u0 ? u0[o + j] : 0.0;
    }
    r.inv = lv && mode != 2 ? geo[(size_t)(base + rel) * GEO + 4] : 0.0;
    r.jt = lv && mode != 2 ? geo[(size_t)(base + rel) * GEO + rm] : 0.0;
  };
  auto load_flux = [&](int t, RowIn &r) {
    const bool lv = t < ntiles && rel < N - t * EB && mode != 2;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int64_t f = checked(r.ef[q] >> 1, F, err);      // ef = 0 on rows past the mesh
      const int side = r.ef[q] & 1;
      r.s[q] = lv ? fmean[(size_t)f * M + rm] : 0.0;
#pragma unroll
      for (int k = 0; k < NE; ++k)
        r.f[q * NE + k] = lv ? fhat[((size_t)f * NE + (side ? NE - 1 - k : k)) * M + rm] : 0.0f;
    }
  };
  static_assert(EB * 4 == kTcThreads, "one J^tau entry per row");

  RowIn cur, nxt;
  if (AHEAD) { load_head(blockIdx.x, cur); load_flux(blockIdx.x, cur); }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    e0 = tile * EB;
    ecount = min(EB, N - e0);
    const bool live = rel < ecount;
    const int tnext = tile + gridDim.x;
    if (!AHEAD) { load_head(tile, cur); load_flux(tile, cur); }
    sJ[row] = tc::f64_to_f32(cur.jt);      // sJ[4 e + i]: entry i of element e's J^tau
    for (int k = 0; k < K1; ++k) put<X3>(A1, T::A1P, row, k, K1, k < NP ? tc::f64_to_f32(cur.c[k]) : 0.0f);
    if (mode == 2) {
      // ---- traces only: GEMM 3 on the stage input ----
      if (AHEAD) load_head(tnext, nxt);
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (!traces_of_A1()) break;
      __syncthreads();
      if (AHEAD) cur = nxt;
      continue;
    }
    // ---- its edge fluxes in the element's orientation and point order: the lift
    // columns of GEMM 2, and the mean mode's lift in float64 ----
    double sq[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int side = cur.ef[q] & 1;
      sq[q] = side ? cur.s[q] : tc::neg_bits(cur.s[q]);
#pragma unroll
      for (int k = 0; k < NE; ++k) {
        const float v = side ? cur.f[q * NE + k] : -cur.f[q * NE + k];
        put<X3>(A2, T::A2P, row, 2 * NQ + q * NE + k, K2, v);
      }
    }
    const double s0 = (sq[0] + sq[1]) + sq[2];
    for (int qk = 2 * NQ + NF; qk < K2; ++qk) put<X3>(A2, T::A2P, row, qk, K2, 0.0f);
    if (AHEAD) load_head(tnext, nxt);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- GEMM 1: interpolation to the volume points ----
    if (tid == 0) {
      gemm<X3, K1>(tmem, uA1, T::A1P, uB1, T::B1P, tc::idesc_tf32(128, N1));
      tc::commit(mbar);
    }
    // the part of the stage update that does not depend on the RHS, b0 c + a0 u0,
    // in float64 while the tensor core runs GEMM 1:
    // a0 u0 + b0 c + g dt R with R = D / det J is b0 c + a0 u0 + (g dt / det J) D
    double tb[NP];
    const double kap = su.g * su.dt * cur.inv;
    if (mode == 1) {
#pragma unroll
      for (int j = 0; j < NP; ++j) tb[j] = need_u0 ? fma(su.a0, cur.u[j], su.b0 * cur.c[j]) : su.b0 * cur.c[j];
    }
    bool ok = tc::mbar_wait(mbar, phase, kWaitNs);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) { if (tid == 0) atomicOr(err, kErrTimeout); break; }
    tc::fence_after_sync();
    {
      float v[N1];
      tmem_row<N1>(trow, v);
#pragma unroll
      for (int k = 0; k < NQ; ++k) sU[(rel * NQ + k) * M + rm] = v[k];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- float32 flux at the volume points -> G_r, G_s columns of GEMM 2 ----
    // Thread (element rel, kk = rm) takes the points k = kk + 4 i of its element.
    // Column C0 + kk + 4 i of row 4 rel + m sits at byte kmaj(4 rel, C0 + kk) +
    // 16 m + 128 i, so every store below is a fixed offset from two bases.
    {
      const int oGr = tc::kmaj(4 * rel, rm, K2), oGs = tc::kmaj(4 * rel, NQ + rm, K2);
      bool phys = true;
#pragma unroll
      for (int i = 0; i < (NQ + 3) / 4; ++i) {
        const int k = rm + 4 * i;
        if (k < NQ) {
          const float4 U4 = *reinterpret_cast<const float4 *>(sU + (rel * NQ + k) * M);
          const float U[M] = {U4.x, U4.y, U4.z, U4.w};
          float Gr[M], Gs[M];
          if (live) {
            phys &= ref_flux_f32(U, sJ + rel * 4, g32, Gr, Gs);
          } else {
#pragma unroll
            for (int m = 0; m < M; ++m) { Gr[m] = 0.0f; Gs[m] = 0.0f; }
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            put_at<X3>(A2, T::A2P, oGr + 16 * m + 128 * i, Gr[m]);
            put_at<X3>(A2, T::A2P, oGs + 16 * m + 128 * i, Gs[m]);
          }
        }
      }
      if (!phys) atomicOr(err, kErrNonPhysical);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- GEMM 2: volume projection + lift ----
    if (tid == 0) {
      gemm<X3, K2>(tmem, uA2, T::A2P, uB2, T::B2P, tc::idesc_tf32(128, N2));
      tc::commit(mbar);
    }
    if (AHEAD) load_flux(tnext, nxt);
    ok = tc::mbar_wait(mbar, phase, kWaitNs);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) { if (tid == 0) atomicOr(err, kErrTimeout); break; }
    tc::fence_after_sync();
    {
      float v[N2];
      tmem_row<N2>(trow, v);
      double cr[NP];
      if (live) {
        const double inv = cur.inv;
        if (mode == 0) {
#pragma unroll
          for (int j = 0; j < NP; ++j) cr[j] = (j == 0 ? s0 : tc::f32_to_f64(v[j])) * inv;
        } else {
          // with the second output (the classical RK4's running sum)
          // x acc + y out + (w dt / det J) D beside it
          const size_t o = ((size_t)(e0 + rel) * M + rm) * NP;
          const double kw = su.w * su.dt * inv;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            const double D = j == 0 ? s0 : tc::f32_to_f64(v[j]);
            cr[j] = fma(kap, D, tb[j]);
            if (OUT2) {
              double t2 = su.y * cr[j];
              if (su.x != 0.0) t2 = fma(su.x, su.acc[o + j], t2);
              su.out2[o + j] = fma(kw, D, t2);
            }
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) cr[j] = 0.0;
      }
      // GEMM 2 has completed: its A planes stage the new state
#pragma unroll
      for (int j = 0; j < NP; ++j) sStage[(rel * M + rm) * NP + j] = cr[j];
      if (trace_out)
        for (int k = 0; k < K1; ++k) put<X3>(A1, T::A1P, row, k, K1, k < NP ? tc::f64_to_f32(cr[k]) : 0.0f);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    {
      double *dst = out + (size_t)e0 * M * NP;
      for (int i = tid; i < ecount * M * NP; i += kTcThreads) dst[i] = sStage[i];
    }
    if (trace_out && !traces_of_A1()) break;
    __syncthreads();
    if (AHEAD) cur = nxt;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int P, int NE, bool X3, bool OUT2, int Q>
int run_tc(const dg_mesh *m, const double *c, const double *u0, double *out, float *trace_out, const float *fhat,
           const double *fmean, const StageUpdate &su, int mode, cudaStream_t s) {
  using T = Tc<P, NE, X3, Q>;
  static PerDevice attr_set;
  if (!attr_set.test(m->device)) {
    cudaError_t e = cudaFuncSetAttribute(k_element_tc<P, NE, X3, OUT2, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         T::SMEM);
    if (e != cudaSuccess) return (int)e;
    // all of the SM's unified L1/shared storage as shared memory, so that the
    // occupancy query and the launch see every CTA that fits
    e = cudaFuncSetAttribute(k_element_tc<P, NE, X3, OUT2, Q>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr_set.set(m->device);
  }
  // CTAs per SM from the shared memory and registers each needs (the occupancy
  // query under-reports for this kernel), at most 8 (TMEM: 512 columns per SM)
  static int per_sm = 0;
  if (per_sm == 0) {
    int smem_sm = 0, reserved = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device);
    if (e != cudaSuccess) return (int)e;
    e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, m->device);
    if (e != cudaSuccess) return (int)e;
    per_sm = smem_sm / (T::SMEM + reserved);
    // and from the registers (allocated per warp in units of 256)
    int regs_sm = 0;
    e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, m->device);
    if (e != cudaSuccess) return (int)e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_element_tc<P, NE, X3, OUT2, Q>);
    if (e != cudaSuccess) return (int)e;
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs_sm / (warp_regs * (kTcThreads / 32));
    if (per_sm > by_regs) per_sm = by_regs;
    if (per_sm > 512 / kTmemCols) per_sm = 512 / kTmemCols;
    if (per_sm < 1) per_sm = 1;
  }
  const int ntiles = (int)((m->N + T::EB - 1) / T::EB);
  const int grid = ntiles < m->num_sms * per_sm ? ntiles : m->num_sms * per_sm;
  k_element_tc<P, NE, X3, OUT2, Q><<<grid, kTcThreads, T::SMEM, s>>>(c, u0, out, trace_out, fhat, fmean, m->geo, m->elem_face,
                                                            m->tab, (int)m->N, m->F, su, mode, m->gamma,
                                                            m->err_flag);
  return (int)cudaGetLastError();
}

// SYM: the symmetric volume rule (Q = sym_points(p)), else the collapsed grid
template <bool X3, bool SYM>
int dispatch_tc(const dg_mesh *m, const double *c, const double *u0, double *out, float *trace_out,
                const float *fhat, const double *fmean, const StageUpdate &su, int mode, cudaStream_t s) {
#define CALL(P, NE)                                                                                      \
  (su.out2 && mode == 1                                                                                  \
       ? run_tc<P, NE, X3, true, SYM ? sym_points(P) : 0>(m, c, u0, out, trace_out, fhat, fmean, su, mode, s) \
       : run_tc<P, NE, X3, false, SYM ? sym_points(P) : 0>(m, c, u0, out, trace_out, fhat, fmean, su, mode, s))
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaErrorInvalidValue;
}


}  // namespace
}  // namespace dg
