/*
 * dg_mixed_tc.cuh -- the mixed-precision element kernel k_element_tc and its
 * launcher, included by the translation units that instantiate it: dg_mixed.cu
 * for the collapsed volume grid, dg_mixed_sym.cu for the symmetric rules (two
 * units, so that the two sets of instantiations compile in parallel).
 *
 * A tile is 32 elements = 128 accumulator rows, row r = 4 e + m (element e,
 * variable m); thread r of the CTA owns row r.  Per tile:
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
 *
 * Operands.  The A operands of the three GEMMs live in tensor memory: row r of A
 * is TMEM lane r, so the thread that owns a row writes it with tcgen05.st straight
 * from its registers (TF32 planes hi and, for 3xTF32, lo; one column per
 * element along K).  The B operands (the tables, split likewise) sit in shared
 * memory, K-major without swizzle, written once per CTA.  The accumulator D takes
 * the first columns of the CTA's TMEM allocation and the A planes the next ones;
 * GEMM 1's operand shares columns with GEMM 2's (its result has been read back by
 * the time GEMM 2's operand is written), and GEMM 3's with both.
 *
 * Only the flux step moves data between the threads of an element (its four
 * rows are four lanes of one warp): the interpolated state goes through shared
 * memory from the row layout [variable][point] to the point layout, and the
 * reference fluxes back, with warp-level synchronisation only.  The CTA
 * synchronises three times per tile, before each GEMM is issued.
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
constexpr int imax(int a, int b) { return a > b ? a : b; }
// TMEM is allocated in powers of two of at least 32 columns
constexpr int tmem_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }
constexpr int kTcThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s per MMA batch before giving up
constexpr uint32_t kSuspendNs = 2000;         // suspend-time hint of one mbarrier try

template <int P, int NE, bool X3, int Q>
struct Tc {
  using C = Cfg<P, NE, Q>;
  static constexpr int NP = C::NP, NQ = C::NQ, NF = C::NF;
  static constexpr int EB = 32, ROWS = 128;
  static constexpr int K1 = pad8(NP), N1 = pad16(NQ), K2 = pad8(2 * NQ + NF), N2 = pad16(NP), N4 = pad16(NF);
  static constexpr int NS = X3 ? 2 : 1;                     // TF32 planes: hi (, lo)
  static constexpr int ND = imax(imax(N1, N2), N4);
  // GEMM 2 as one batch over [G_r | G_s | lifted fluxes] (K2 columns of A), or,
  // where that takes fewer TMEM columns (SPLIT: p = 4 in 3xTF32), as two batches
  // into the same accumulator that reuse the operand columns: [G_r | lifted
  // fluxes] (KG + KL columns, B = [Dr; Lf]), then G_s (KG columns, B = Ds)
  static constexpr int KG = pad8(NQ), KL = pad8(NF);
  static constexpr bool SPLIT = tmem_cols(ND + NS * (KG + KL)) < tmem_cols(ND + NS * K2);
  static constexpr int KA = SPLIT ? KG + KL : K2;            // A columns per plane
  // TMEM columns: D [0, ND), A hi [ND, ND + KA), A lo [ND + KA, ND + 2 KA)
  static constexpr int COLS = tmem_cols(ND + NS * KA);
  static constexpr int PER_SM = 512 / COLS;                   // CTAs whose TMEM fits on one SM
  // shared memory: B operands (split), then per-warp staging
  static constexpr int B1P = N1 * K1 * 4, B4P = N4 * K1 * 4;
  static constexpr int B2P = N2 * (SPLIT ? KG + KL : K2) * 4, B2bP = SPLIT ? N2 * KG * 4 : 0;
  static constexpr int oB1 = 0;
  static constexpr int oB2 = align1k(oB1 + B1P * NS);
  static constexpr int oB2b = align1k(oB2 + B2P * NS);
  static constexpr int oB4 = align1k(oB2b + B2bP * NS);
  static constexpr int endB = align1k(oB4 + B4P * NS);
  // U staging [EB][SE] floats, point k of element e at e SE + 4 k (its four
  // variables); SE / 4 is odd, so the row threads' scalar writes hit 32 banks.
  // The edge traces [NF][4] are staged in the same place.
  static constexpr int SE4 = imax((NQ & 1) ? NQ : NQ + 1, (NF & 1) ? NF : NF + 1);
  static constexpr int SE = 4 * SE4;
  // reference-flux staging [EB][M][RG] floats (row 4 e + m, column k of G_r,
  // NQ + k of G_s); RG odd.  Each warp (8 elements) has a region of WS floats
  // holding its U staging and, in the same place, its G staging: a thread has
  // read its points' U before the warp writes G.
  static constexpr int RG = (2 * NQ) | 1;
  static constexpr int WS = imax(8 * SE, 8 * M * RG);
  static constexpr int oW = endB;
  static constexpr int oJ = oW + 4 * WS * 4;                         // float [EB][4]  J^tau
  static constexpr int oBar = (oJ + EB * 16 + 15) / 16 * 16;        // 2 mbarriers, TMEM slot
  static constexpr int SMEM_NOPF = oBar + 32;
  // the next tile's stage input, u^n [EB][M][NP] and geometry [EB][GEO] (bulk
  // copies one tile ahead), where the shared memory of the CTAs an SM holds allows
  static constexpr int PC = EB * M * NP * 8, PG = EB * GEO * 8;
  static constexpr int oPC = (SMEM_NOPF + 127) / 128 * 128, oPU = oPC + PC, oPG = oPU + PC;
  static constexpr int SMEM_PF = oPG + PG;
  static constexpr int CTAS = PER_SM < 4 ? PER_SM : 4;              // the launch bound
  static constexpr bool PF = SMEM_PF + 1024 <= 233472 / CTAS;
  static constexpr int SMEM = PF ? SMEM_PF : SMEM_NOPF;
  static_assert(K1 <= KA, "GEMM 1's operand shares GEMM 2's columns");
  static_assert(N1 <= 256 && N2 <= 256 && N4 <= 256, "MMA N");
  static_assert(ND + NS * KA <= 512, "TMEM columns");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// writes v (rounded to TF32, and its TF32 remainder for the split product) at
// (row, k) of a K-major shared-memory operand with ktot columns (the B tables)
template <bool X3>
__device__ __forceinline__ void put(unsigned char *base, int plane_bytes, int row, int k, int ktot, float v) {
  const int off = tc::kmaj(row, k, ktot);
  const float hi = tc::to_tf32(v);
  *reinterpret_cast<float *>(base + off) = hi;
  if (X3) *reinterpret_cast<float *>(base + plane_bytes + off) = tc::to_tf32(v - hi);
}

// this thread's TMEM lane, columns [c0, c0 + N) (N a multiple of 8) <- v split
// into TF32 planes: hi = v rounded to TF32 at tHi, and (3xTF32) the remainder
// lo = v - hi at tLo, exact in float32; the tensor core takes lo's leading TF32
// bits, so hi + lo carries v to within 2^-22 of |v|.
template <bool X3, int N>
__device__ __forceinline__ void st_split(uint32_t tHi, uint32_t tLo, const float *v) {
#pragma unroll
  for (int c = 0; c < N; c += 8) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      hi[i] = tc::tf32_bits(__float_as_uint(v[c + i]));
      if (X3) lo[i] = __float_as_uint(v[c + i] - __uint_as_float(hi[i]));
    }
    tc::st8(tHi + (uint32_t)c, hi);
    if (X3) tc::st8(tLo + (uint32_t)c, lo);
  }
}

// D (TMEM) = sum over k-steps of A B^T with A in TMEM (columns aHi, aLo) and B in
// shared memory; split products a_lo b_hi + a_hi b_lo + a_hi b_hi when X3
// ACC: accumulate onto D from the first k-step on (the second batch of a split GEMM 2)
template <bool X3, int KT, bool ACC = false>
__device__ __forceinline__ void gemm_ts(uint32_t d, uint32_t aHi, uint32_t aLo, uint32_t b, int b_plane,
                                        uint32_t idesc) {
#pragma unroll
  for (int s = 0; s < KT / 8; ++s) {
    const uint32_t off = (uint32_t)s * 256u, ac = (uint32_t)s * 8u;
    const uint32_t first = (ACC || s > 0) ? 1u : 0u;
    if (X3) {
      tc::mma_tf32_ts(d, aLo + ac, tc::desc(b + off, KT), idesc, first);
      tc::mma_tf32_ts(d, aHi + ac, tc::desc(b + b_plane + off, KT), idesc, 1u);
      tc::mma_tf32_ts(d, aHi + ac, tc::desc(b + off, KT), idesc, 1u);
    } else {
      tc::mma_tf32_ts(d, aHi + ac, tc::desc(b + off, KT), idesc, first);
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
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(U[0]));
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
__global__ void __launch_bounds__(kTcThreads, Tc<P, NE, X3, Q>::CTAS)
k_element_tc(const double *c, const double *u0, double *out, float *__restrict__ trace_out,
             const float *__restrict__ fhat, const double *__restrict__ fmean, const double *__restrict__ geo,
             const int32_t *__restrict__ elem_face, const unsigned char *__restrict__ bimg, int N, int64_t F,
             StageUpdate su, int mode, double gamma, int bulk, int *err) {
  using T = Tc<P, NE, X3, Q>;
  constexpr int NP = T::NP, NQ = T::NQ, NF = T::NF, EB = T::EB, SE = T::SE, RG = T::RG;
  constexpr int K1 = T::K1, N1 = T::N1, K2 = T::K2, N2 = T::N2, N4 = T::N4;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *B1 = sm + T::oB1, *B2 = sm + T::oB2, *B2b = sm + T::oB2b, *B4 = sm + T::oB4;
  // this warp's staging region: element e (its e & 7) at sU + (e & 7) SE, sG + (e & 7) M RG
  float *sU = reinterpret_cast<float *>(sm + T::oW) + (threadIdx.x >> 5) * T::WS;
  float *sG = sU;
  float *sJ = reinterpret_cast<float *>(sm + T::oJ);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + T::oBar);         // [0] MMAs, [1] bulk copies
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + T::oBar + 16);
  const double *sPC = reinterpret_cast<const double *>(sm + T::oPC);
  const double *sPU = reinterpret_cast<const double *>(sm + T::oPU);
  const double *sPG = reinterpret_cast<const double *>(sm + T::oPG);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t mbar = tc::smem_u32(bar), mbar_in = tc::smem_u32(bar + 1);
  const bool pf = T::PF && bulk;

  // ---- once per CTA: TMEM, mbarriers; the B operands (split, in their shared-
  // memory layout: the mesh's image, k_tc_tables) arrive by a bulk copy, with
  // the first tile's inputs ----
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(slot), T::COLS);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(mbar_in, 1);
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t tD = tmem + ((uint32_t)(warp * 32) << 16);          // this warp's 32 lanes
  const uint32_t tHi = tD + (uint32_t)T::ND, tLo = tHi + (uint32_t)T::KA;
  const uint32_t aHi = tmem + (uint32_t)T::ND, aLo = aHi + (uint32_t)T::KA;
  const uint32_t uB1 = tc::smem_u32(B1), uB2 = tc::smem_u32(B2), uB2b = tc::smem_u32(B2b), uB4 = tc::smem_u32(B4);
  const float g32 = (float)gamma;
  const int row = tid, rel = row >> 2, rm = row & 3;                 // accumulator row = 4 e + m
  const int le = rel & 7;                                            // element within the warp
  uint32_t phase = 0, phase_in = 0;
  // failed: a bounded wait expired; mma_lost: it was an MMA batch's; copies: a
  // bulk copy is in flight (its phase is phase_in)
  bool failed = false, mma_lost = false, copies = false;

  // the rows' tcgen05.st complete and are ordered before the MMA issue
  auto sync_operands = [&]() {
    tc::wait_st();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  // waits for the issued MMAs; false if the bounded wait expired (recorded)
  auto mma_done = [&]() -> bool {
    const bool done = tc::mbar_wait_sleep(mbar, phase, kWaitNs, kSuspendNs);
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicOr(err, kErrTimeout);
      failed = true;
      mma_lost = true;
      return false;
    }
    tc::fence_after_sync();
    return true;
  };
  // GEMM 3 has completed: edge traces of the state in the A columns [0, K1) ->
  // trace_out, staged through this warp's part of sU for float4 stores
  auto store_traces = [&](int e0, bool live) {
    float v[N4];
    tmem_row<N4>(tD, v);
    float *t = sU + le * SE + rm;
#pragma unroll
    for (int qk = 0; qk < NF; ++qk) t[4 * qk] = v[qk];
    __syncwarp();
    float4 *dst = reinterpret_cast<float4 *>(trace_out + (size_t)(e0 + rel) * NF * M);
#pragma unroll
    for (int i = 0; i < (NF + 3) / 4; ++i) {
      const int qk = rm + 4 * i;
      if (qk < NF && live) dst[qk] = *reinterpret_cast<const float4 *>(sU + le * SE + 4 * qk);
    }
    __syncwarp();
  };

  const int ntiles = (N + EB - 1) / EB;
  const bool need_u0 = mode == 1 && su.a0 != 0.0;
  // one thread: bulk copies of tile t's stage input, u^n and geometry into the
  // prefetch buffers (the CTA has finished reading them)
  auto prefetch = [&](int t) {
    const int e0 = t * EB, ec = min(EB, N - e0);
    const uint32_t bc = (uint32_t)ec * M * NP * 8, bg = (uint32_t)ec * GEO * 8;
    tc::fence_proxy_async();
    tc::mbar_arrive_expect_tx(mbar_in, bc + (need_u0 ? bc : 0u) + (mode != 2 ? bg : 0u));
    tc::bulk_g2s(tc::smem_u32(sPC), c + (size_t)e0 * M * NP, bc, mbar_in);
    if (need_u0) tc::bulk_g2s(tc::smem_u32(sPU), u0 + (size_t)e0 * M * NP, bc, mbar_in);
    if (mode != 2) tc::bulk_g2s(tc::smem_u32(sPG), geo + (size_t)e0 * GEO, bg, mbar_in);
  };
  // the prologue's copies: the B image, and the first tile's inputs
  if (tid == 0) {
    const int e0 = blockIdx.x * EB, ec = min(EB, N - e0);
    const uint32_t bc = (uint32_t)ec * M * NP * 8, bg = (uint32_t)ec * GEO * 8;
    const bool first = pf && blockIdx.x < ntiles;
    tc::mbar_arrive_expect_tx(mbar_in, (uint32_t)T::endB +
                                           (first ? bc + (need_u0 ? bc : 0u) + (mode != 2 ? bg : 0u) : 0u));
    tc::bulk_g2s(tc::smem_u32(sm), bimg, (uint32_t)T::endB, mbar_in);
    if (first) {
      tc::bulk_g2s(tc::smem_u32(sPC), c + (size_t)e0 * M * NP, bc, mbar_in);
      if (need_u0) tc::bulk_g2s(tc::smem_u32(sPU), u0 + (size_t)e0 * M * NP, bc, mbar_in);
      if (mode != 2) tc::bulk_g2s(tc::smem_u32(sPG), geo + (size_t)e0 * GEO, bg, mbar_in);
    }
  }
  {
    const bool ok = tc::mbar_wait_sleep(mbar_in, phase_in, kWaitNs, kSuspendNs);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(err, kErrTimeout);
      failed = true;
      copies = true;                    // the teardown waits on phase_in again
    } else {
      phase_in ^= 1u;
    }
  }
  // the element's three edges (2 f + side), loaded one tile ahead
  auto load_ef = [&](int t, int *ef) {
    const int r = t * EB + rel;
#pragma unroll
    for (int q = 0; q < 3; ++q) ef[q] = mode != 2 && t < ntiles && r < N ? elem_face[(size_t)r * 3 + q] : 0;
  };
  int ef[3];
  load_ef(blockIdx.x, ef);
  for (int tile = failed ? ntiles : blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * EB;
    const int ecount = min(EB, N - e0);
    const bool live = rel < ecount;
    const size_t o = ((size_t)(e0 + rel) * M + rm) * NP;
    const int tnext = tile + gridDim.x;
    // ---- the row's edge fluxes in the element's point order (the lift columns
    // of GEMM 2) and their float64 mean-mode integrals; the loads stay in flight
    // until GEMM 2's operand is written, where the sign of the element's
    // orientation is applied (on the bit patterns) ----
    float fl[NF];
    double sq[3];
    uint32_t sgn[3];
    if (mode != 2) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int64_t f = checked(ef[q] >> 1, F, err);
        const int side = ef[q] & 1;
        sgn[q] = side ? 0u : 0x80000000u;
        sq[q] = live ? fmean[(size_t)f * M + rm] : 0.0;
        const float *fp = fhat + (size_t)f * NE * M + rm;
#pragma unroll
        for (int k = 0; k < NE; ++k) fl[q * NE + k] = live ? fp[(side ? NE - 1 - k : k) * M] : 0.0f;
      }
      load_ef(tnext, ef);
    }
    if (pf && tile != (int)blockIdx.x) {
      const bool ok = tc::mbar_wait_sleep(mbar_in, phase_in, kWaitNs, kSuspendNs);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(err, kErrTimeout);
        failed = true;                  // copies stays true: the teardown waits on phase_in again
        break;
      }
      phase_in ^= 1u;
      copies = false;
    }
    // ---- the stage input: GEMM 1's operand (A columns [0, K1)) ----
    // (without the bulk copies: scalar loads of the caller's array, which then
    // needs only the alignment of a double; a warp's rows are contiguous)
    double cv[NP];
    if (pf && NP % 2 == 0) {
      const double2 *r2 = reinterpret_cast<const double2 *>(sPC + row * NP);
#pragma unroll
      for (int j = 0; j < NP / 2; ++j) {
        const double2 x = r2[j];
        cv[2 * j] = live ? x.x : 0.0;
        cv[2 * j + 1] = live ? x.y : 0.0;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NP; ++j) cv[j] = live ? (pf ? sPC[row * NP + j] : c[o + j]) : 0.0;
    }
    // the part of the stage update that does not depend on the RHS, b0 c + a0 u0,
    // in float64 among the integer work of the operand conversion:
    // a0 u0 + b0 c + g dt R with R = D / det J is b0 c + a0 u0 + (g dt / det J) D
    double tb[NP];
    if (mode == 1) {
      if (need_u0) {
        double uv[NP];
        if (pf && NP % 2 == 0) {
          const double2 *r2 = reinterpret_cast<const double2 *>(sPU + row * NP);
#pragma unroll
          for (int j = 0; j < NP / 2; ++j) {
            const double2 x = r2[j];
            uv[2 * j] = live ? x.x : 0.0;
            uv[2 * j + 1] = live ? x.y : 0.0;
          }
        } else {
#pragma unroll
          for (int j = 0; j < NP; ++j) uv[j] = live ? (pf ? sPU[row * NP + j] : u0[o + j]) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < NP; ++j) tb[j] = fma(su.a0, uv[j], su.b0 * cv[j]);
      } else if (su.b0 == 1.0) {
#pragma unroll
        for (int j = 0; j < NP; ++j) tb[j] = cv[j];
      } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) tb[j] = su.b0 * cv[j];
      }
    }
    {
      float v[K1];
#pragma unroll
      for (int k = 0; k < K1; ++k) v[k] = k < NP ? __uint_as_float(tc::f64_to_f32_rz_bits(cv[k])) : 0.0f;
      st_split<X3, K1>(tHi, tLo, v);
    }
    if (mode == 2) {
      // ---- traces only: GEMM 3 on the stage input ----
      sync_operands();
      if (tid == 0) {
        gemm_ts<X3, K1>(tmem, aHi, aLo, uB4, T::B4P, tc::idesc_tf32(128, N4));
        tc::commit(mbar);
      }
      if (!mma_done()) break;
      if (pf && tnext < ntiles) {
        if (tid == 0) prefetch(tnext);
        copies = true;
      }
      store_traces(e0, live);
      continue;
    }
    double inv = 0.0;
    {
      const double *ge = pf ? sPG + rel * GEO : geo + (size_t)(e0 + rel) * GEO;
      inv = live ? ge[4] : 0.0;
      sJ[row] = __uint_as_float(tc::f64_to_f32_rz_bits(live ? ge[rm] : 0.0));
    }
    const double kap = su.g * su.dt * inv;
    sync_operands();
    // ---- GEMM 1: interpolation to the volume points ----
    if (tid == 0) {
      gemm_ts<X3, K1>(tmem, aHi, aLo, uB1, T::B1P, tc::idesc_tf32(128, N1));
      tc::commit(mbar);
    }
    if (!mma_done()) break;
    // every thread has read the prefetch buffers: the next tile's copies
    if (pf && tnext < ntiles) {
      if (tid == 0) prefetch(tnext);
      copies = true;
    }
    // ---- U (this row: variable rm at the NQ points) -> point layout ----
    {
      float v[N1];
      tmem_row<N1>(tD, v);
      float *u = sU + le * SE + rm;
#pragma unroll
      for (int k = 0; k < NQ; ++k) u[4 * k] = v[k];
    }
    __syncwarp();
    // ---- float32 flux at the points k = rm + 4 i of element rel ----
    {
      const float4 J = *reinterpret_cast<const float4 *>(sJ + rel * 4);
      const float jt[4] = {J.x, J.y, J.z, J.w};
      float4 Up[(NQ + 3) / 4];
#pragma unroll
      for (int i = 0; i < (NQ + 3) / 4; ++i) {
        const int k = rm + 4 * i;
        Up[i] = k < NQ ? *reinterpret_cast<const float4 *>(sU + le * SE + 4 * k) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();          // the G staging below overwrites the U staging
      float *g = sG + le * (M * RG);
      bool phys = true;
#pragma unroll
      for (int i = 0; i < (NQ + 3) / 4; ++i) {
        const int k = rm + 4 * i;
        if (k < NQ) {
          const float U[M] = {Up[i].x, Up[i].y, Up[i].z, Up[i].w};
          float Gr[M], Gs[M];
          if (live) {
            phys &= ref_flux_f32(U, jt, g32, Gr, Gs);
          } else {
#pragma unroll
            for (int m = 0; m < M; ++m) { Gr[m] = 0.0f; Gs[m] = 0.0f; }
          }
#pragma unroll
          for (int m = 0; m < M; ++m) {
            g[m * RG + k] = Gr[m];
            g[m * RG + NQ + k] = Gs[m];
          }
        }
      }
      if (!phys) atomicOr(err, kErrNonPhysical);
    }
    __syncwarp();
    const float *g = sG + (row & 31) * RG;
    if constexpr (!T::SPLIT) {
      // ---- GEMM 2's operand: [G_r | G_s | lifted fluxes | 0] in A columns [0, K2) ----
#pragma unroll
      for (int c0 = 0; c0 < K2; c0 += 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int col = c0 + i;
          const int li = col - 2 * NQ >= 0 && col - 2 * NQ < NF ? col - 2 * NQ : 0;
          v[i] = col < 2 * NQ ? g[col]
                              : (col < 2 * NQ + NF ? __uint_as_float(__float_as_uint(fl[li]) ^ sgn[li / NE]) : 0.0f);
        }
        st_split<X3, 8>(tHi + (uint32_t)c0, tLo + (uint32_t)c0, v);
      }
      sync_operands();
      // ---- GEMM 2: volume projection + lift ----
      if (tid == 0) {
        gemm_ts<X3, K2>(tmem, aHi, aLo, uB2, T::B2P, tc::idesc_tf32(128, N2));
        tc::commit(mbar);
      }
      if (!mma_done()) break;
    } else {
      // ---- GEMM 2 in two batches: [G_r | 0 | lifted fluxes | 0] in A columns
      // [0, KG + KL) against [Dr; Lf], then G_s in columns [0, KG) against Ds ----
      constexpr int KG = T::KG, KL = T::KL;
#pragma unroll
      for (int c0 = 0; c0 < KG + KL; c0 += 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int col = c0 + i;
          const int li = col - KG >= 0 && col - KG < NF ? col - KG : 0;
          v[i] = col < KG ? (col < NQ ? g[col] : 0.0f)
                          : (col - KG < NF ? __uint_as_float(__float_as_uint(fl[li]) ^ sgn[li / NE]) : 0.0f);
        }
        st_split<X3, 8>(tHi + (uint32_t)c0, tLo + (uint32_t)c0, v);
      }
      sync_operands();
      if (tid == 0) {
        gemm_ts<X3, KG + KL>(tmem, aHi, aLo, uB2, T::B2P, tc::idesc_tf32(128, N2));
        tc::commit(mbar);
      }
      if (!mma_done()) break;
#pragma unroll
      for (int c0 = 0; c0 < KG; c0 += 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = c0 + i < NQ ? g[NQ + c0 + i] : 0.0f;
        st_split<X3, 8>(tHi + (uint32_t)c0, tLo + (uint32_t)c0, v);
      }
      sync_operands();
      if (tid == 0) {
        gemm_ts<X3, KG, true>(tmem, aHi, aLo, uB2b, T::B2bP, tc::idesc_tf32(128, N2));
        tc::commit(mbar);
      }
      if (!mma_done()) break;
    }
    double cr[NP];
    {
      // the mean mode's lift: the three edges' float64 integrals, signed by the
      // element's orientation
      double sqs[3];
#pragma unroll
      for (int q = 0; q < 3; ++q)
        sqs[q] = __hiloint2double(__double2hiint(sq[q]) ^ (int)sgn[q], __double2loint(sq[q]));
      const double s0 = (sqs[0] + sqs[1]) + sqs[2];
      float v[N2];
      tmem_row<N2>(tD, v);
      if (mode == 0) {
#pragma unroll
        for (int j = 0; j < NP; ++j) cr[j] = (j == 0 ? s0 : tc::f32_to_f64_fast(v[j])) * inv;
      } else {
        // with the second output (the classical RK4's running sum)
        // x acc + y out + (w dt / det J) D beside it
        const double kw = su.w * su.dt * inv;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const double D = j == 0 ? s0 : tc::f32_to_f64_fast(v[j]);
          cr[j] = fma(kap, D, tb[j]);
          if (OUT2 && live) {
            double t2 = su.y * cr[j];
            if (su.x != 0.0) t2 = fma(su.x, su.acc[o + j], t2);
            su.out2[o + j] = fma(kw, D, t2);
          }
        }
      }
      if (live) {
#pragma unroll
        for (int j = 0; j < NP; ++j) out[o + j] = cr[j];
      }
    }
    if (trace_out) {
      // ---- GEMM 3: edge traces of the new state ----
      float v[K1];
#pragma unroll
      for (int k = 0; k < K1; ++k) v[k] = k < NP ? __uint_as_float(tc::f64_to_f32_rz_bits(cr[k])) : 0.0f;
      st_split<X3, K1>(tHi, tLo, v);
      sync_operands();
      if (tid == 0) {
        gemm_ts<X3, K1>(tmem, aHi, aLo, uB4, T::B4P, tc::idesc_tf32(128, N4));
        tc::commit(mbar);
      }
      if (!mma_done()) break;
      store_traces(e0, live);
    }
  }
  if (failed) {
    // a bounded wait expired: wait (bounded again) for the MMAs of that batch, so
    // that the columns freed below are no longer written, and for a bulk copy
    // still in flight, so that no copy lands after the CTA has left
    if (mma_lost) tc::mbar_wait_sleep(mbar, phase ^ 1u, kWaitNs, kSuspendNs);
    if (copies) tc::mbar_wait_sleep(mbar_in, phase_in, kWaitNs, kSuspendNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, T::COLS);
}

// The B operands of the three GEMMs, split into TF32 planes, in the byte layout
// k_element_tc keeps them in shared memory: one image per mesh and precision
// mode (T::endB bytes), which every CTA of every launch bulk-copies.
template <int P, int NE, bool X3, int Q>
__global__ void __launch_bounds__(kTcThreads) k_tc_tables(DevTables tab, unsigned char *img) {
  using T = Tc<P, NE, X3, Q>;
  constexpr int NP = T::NP, NQ = T::NQ, NF = T::NF, K1 = T::K1, K2 = T::K2, N2 = T::N2, N4 = T::N4;
  unsigned char *B1 = img + T::oB1, *B2 = img + T::oB2, *B2b = img + T::oB2b, *B4 = img + T::oB4;
  for (int i = threadIdx.x; i < T::endB / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(img)[i] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < T::N1 * K1; i += blockDim.x) {
    const int n = i / K1, k = i - n * K1;
    const double v = (n < NQ && k < NP) ? tab.BvT[k * NQ + n] : 0.0;
    put<X3>(B1, T::B1P, n, k, K1, (float)v);
  }
  if constexpr (!T::SPLIT) {
    for (int i = threadIdx.x; i < N2 * K2; i += blockDim.x) {
      const int n = i / K2, k = i - n * K2;
      double v = 0.0;
      if (n < NP) {
        if (k < NQ) v = tab.Dr[k * NP + n];
        else if (k < 2 * NQ) v = tab.Ds[(k - NQ) * NP + n];
        else if (k < 2 * NQ + NF) v = tab.Lf[(k - 2 * NQ) * NP + n];
      }
      put<X3>(B2, T::B2P, n, k, K2, (float)v);
    }
  } else {
    constexpr int KG = T::KG, KA = T::KG + T::KL;
    for (int i = threadIdx.x; i < N2 * KA; i += blockDim.x) {   // [Dr; Lf]
      const int n = i / KA, k = i - n * KA;
      double v = 0.0;
      if (n < NP) {
        if (k < NQ) v = tab.Dr[k * NP + n];
        else if (k >= KG && k < KG + NF) v = tab.Lf[(k - KG) * NP + n];
      }
      put<X3>(B2, T::B2P, n, k, KA, (float)v);
    }
    for (int i = threadIdx.x; i < N2 * KG; i += blockDim.x) {   // Ds
      const int n = i / KG, k = i - n * KG;
      const double v = (n < NP && k < NQ) ? tab.Ds[k * NP + n] : 0.0;
      put<X3>(B2b, T::B2bP, n, k, KG, (float)v);
    }
  }
  for (int i = threadIdx.x; i < N4 * K1; i += blockDim.x) {
    const int n = i / K1, k = i - n * K1;
    const double v = (n < NF && k < NP) ? tab.BfT[k * NF + n] : 0.0;
    put<X3>(B4, T::B4P, n, k, K1, (float)v);
  }
}

// builds the mesh's two images (1xTF32, 3xTF32) for its p, n_e and volume rule
template <int P, int NE, int Q>
int tc_tables_pq(dg_mesh *m) {
  const size_t bytes[2] = {(size_t)Tc<P, NE, false, Q>::endB, (size_t)Tc<P, NE, true, Q>::endB};
  for (int x = 0; x < 2; ++x) {
    cudaError_t e = cudaMalloc((void **)&m->tc_img[x], bytes[x]);
    if (e != cudaSuccess) return (int)e;
  }
  k_tc_tables<P, NE, false, Q><<<1, kTcThreads>>>(m->tab, m->tc_img[0]);
  k_tc_tables<P, NE, true, Q><<<1, kTcThreads>>>(m->tab, m->tc_img[1]);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}

template <bool SYM>
int tc_tables_rule(dg_mesh *m) {
#define CALL(P, NE) tc_tables_pq<P, NE, SYM ? sym_points(P) : 0>(m)
  if (m->p == 1 && m->ne == 2) return CALL(1, 2);
  if (m->p == 2 && m->ne == 3) return CALL(2, 3);
  if (m->p == 3 && m->ne == 4) return CALL(3, 4);
  if (m->p == 3 && m->ne == 3) return CALL(3, 3);
  if (m->p == 4 && m->ne == 5) return CALL(4, 5);
  if (m->p == 5 && m->ne == 6) return CALL(5, 6);
#undef CALL
  return (int)cudaSuccess;           // no tensor-core kernel for this (p, n_e): nothing to build
}

template <int P, int NE, bool X3, bool OUT2, int Q>
int run_tc(const dg_mesh *m, const double *c, const double *u0, double *out, float *trace_out, const float *fhat,
           const double *fmean, const StageUpdate &su, int mode, cudaStream_t s) {
  using T = Tc<P, NE, X3, Q>;
  auto kern = k_element_tc<P, NE, X3, OUT2, Q>;
  // per device: CTAs per SM from TMEM (512 columns per SM), shared memory and
  // registers, and the dynamic shared memory that keeps the SM at that count
  struct Launch { int per_sm, smem; };
  static Launch cfg[64];
  static PerDevice ready;
  const int dev = m->device;
  Launch L{0, 0};
  if (dev >= 0 && dev < 64 && ready.test(dev)) {
    L = cfg[dev];
  } else {
    int smem_sm = 0, reserved = 0, regs_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return (int)e;
    int per_sm = T::PER_SM;
    const int by_smem = smem_sm / (T::SMEM + reserved);
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs_sm / (warp_regs * (kTcThreads / 32));
    if (per_sm > by_smem) per_sm = by_smem;
    if (per_sm > by_regs) per_sm = by_regs;
    if (per_sm < 1) per_sm = 1;
    // ask for as much shared memory as leaves room for per_sm CTAs only, so that
    // no more CTAs than their TMEM allows share an SM
    int smem = smem_sm / per_sm - reserved;
    smem = smem / 128 * 128;
    if (smem > 227 * 1024) smem = 227 * 1024;
    if (smem < T::SMEM) smem = T::SMEM;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    L = Launch{per_sm, smem};
    if (dev >= 0 && dev < 64) {
      cfg[dev] = L;
      ready.set(dev);
    }
  }
  const int ntiles = (int)((m->N + T::EB - 1) / T::EB);
  const int grid = ntiles < m->num_sms * L.per_sm ? ntiles : m->num_sms * L.per_sm;
  // the bulk copies need 16-byte aligned sources (the mesh's arrays are; the
  // caller's state arrays usually are, else the kernel loads them directly)
  const bool need_u0 = mode == 1 && su.a0 != 0.0;
  const int bulk = ((uintptr_t)c % 16 == 0 && (!need_u0 || (uintptr_t)u0 % 16 == 0)) ? 1 : 0;
  if (!m->tc_img[X3 ? 1 : 0]) return (int)cudaErrorNotReady;
  kern<<<grid, kTcThreads, L.smem, s>>>(c, u0, out, trace_out, fhat, fmean, m->geo, m->elem_face,
                                        m->tc_img[X3 ? 1 : 0], (int)m->N, m->F, su, mode, m->gamma, bulk,
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
