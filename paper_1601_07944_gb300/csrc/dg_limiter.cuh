/*
 * dg_limiter.cuh -- the p = 1 Barth-Jespersen limiter's device code, shared by
 * its own kernel (k_limit_p1) and the limiter phase of the fused small-mesh
 * stepper, so that both produce the same bits.
 */
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dg_device.cuh"
#include "dg_internal.h"

namespace dg {
namespace {

// ---------------------------------------------------------------------------
// Barth-Jespersen limiter for p = 1 (Section 4.3.5), one thread per element and
// variable, in place on c.
// Per variable: Ubar = phi_1 c_1 is the centroid value (the linear modes vanish at
// the centroid), U^max / U^min the extremes of the centroid values of the element
// and its three neighbours; at each edge integration point, with
// d = U(r_qk) - Ubar, alpha_k = min(1, (U^max - Ubar)/d) for d > 0 and
// min(1, (U^min - Ubar)/d) for d < 0; the linear modes are scaled by min_k alpha_k.
// Threads read only the constant mode of their neighbours and write only the
// linear modes of their own element, so the in-place update has no race.
//
// HAVE_TRACES: trace holds the edge traces of c on entry (the element kernel
// wrote them, with the same per-point sums, edge_traces_unit); they are read
// instead of recomputed, and rewritten, for the limited state, only where an
// element is limited.  Otherwise the traces are formed here, and written to
// trace when it is not null.
// The float64 pipe is spared where the decisions allow it: extremes are found on
// order-preserving integer keys of the bit patterns, and every choice between
// two doubles is an integer select of their bit patterns (a conditional move of
// a double may take a float64-pipe instruction, which on this part costs as much
// as an FMA); the smallest ratio over the points is the smaller of
// (U^max - Ubar) / d+ and (U^min - Ubar) / d- with d+ the largest positive and
// |d-| the largest negative deviation (again integer compares, the deviations'
// magnitudes being non-negative), compared by their cross products; a ratio
// limits only when its numerator is below its denominator; the one reciprocal
// is formed only when the element is limited.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// the double whose order_key is k
__device__ __forceinline__ double key_value(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}
__device__ __forceinline__ unsigned long long nonneg_bits(double x) {
  return (unsigned long long)__double_as_longlong(x);   // x >= 0: bits order like values
}
__device__ __forceinline__ double bits_value(unsigned long long b) { return __longlong_as_double((long long)b); }

// The items (element, variable) of block `block` of `nblocks` (a grid-stride
// loop over the blocks' threads): one item per (element, variable), four
// independent chains per element, and a warp's loads and trace stores cover
// contiguous runs.  Every thread of the block calls it (it stages the p = 1 edge
// tables in shared memory behind a block barrier).
template <bool HAVE_TRACES>
__device__ __forceinline__ void limit_p1_items(double *c, double *__restrict__ trace,
                                               const int32_t *__restrict__ elem_nbr, const double *__restrict__ EPa,
                                               const double *__restrict__ EChiM1, const double *__restrict__ EChi,
                                               double phi1, int64_t N, int *err, int block, int nblocks) {
  constexpr int P = 1, NE = 2, ND = 2, NP = 3, NF = 6;
  __shared__ double sPa[ND * NE], sChiM1[NP], sChi[NP * NE];
  if (threadIdx.x < NP * NE) sChi[threadIdx.x] = EChi[threadIdx.x];
  if (threadIdx.x < ND * NE) sPa[threadIdx.x] = EPa[threadIdx.x];
  if (threadIdx.x < NP) sChiM1[threadIdx.x] = EChiM1[threadIdx.x];
  __syncthreads();
  for (int64_t it = (int64_t)block * blockDim.x + threadIdx.x; it < N * M; it += (int64_t)nblocks * blockDim.x) {
    const int64_t e = it >> 2;
    const int m = (int)(it & 3);
    const int64_t nb0 = checked(elem_nbr[e * 3], N, err), nb1 = checked(elem_nbr[e * 3 + 1], N, err),
                  nb2 = checked(elem_nbr[e * 3 + 2], N, err);
    double *ce = c + (e * M + m) * NP;
    double cj[NP] = {ce[0], ce[1], ce[2]};
    const double cn[3] = {c[(nb0 * M + m) * NP], c[(nb1 * M + m) * NP], c[(nb2 * M + m) * NP]};
    double *dst = trace ? trace + (size_t)e * NF * M + m : nullptr;
    double t[NF], z[ND + 1];
    if (HAVE_TRACES) {
#pragma unroll
      for (int x = 0; x < NF; ++x) t[x] = dst[x * M];
    } else {
      face_sums<P>(cj, sChiM1, sChi[0], z);
#pragma unroll
      for (int k = 0; k < NE; ++k) edge_traces_unit<P, NE>(cj, z, sPa, sChi, k, t[k], t[NE + k], t[3 * NE - 1 - k]);
    }
    // extremes of the constant modes (phi_1 > 0 keeps the order)
    unsigned long long kmax = order_key(cj[0]), kmin = kmax;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const unsigned long long kq = order_key(cn[q]);
      kmax = kq > kmax ? kq : kmax;
      kmin = kq < kmin ? kq : kmin;
    }
    const double ub = phi1 * cj[0];
    // U^max - Ubar and Ubar - U^min, formed so that they are exactly >= 0 (an
    // FMA-contracted phi1 cmax - ub would leave the product's rounding error,
    // of either sign, where the difference is 0; the comparisons below read
    // these as non-negative bit patterns)
    const double up = phi1 * (key_value(kmax) - cj[0]), dn = phi1 * (cj[0] - key_value(kmin));
    // the largest deviation above and below the centroid value: the extremes of
    // the edge values less Ubar (a rounded subtraction of Ubar is monotone, so
    // this is the largest of the rounded deviations t - Ubar); 0 where none lies
    // on that side
    unsigned long long tkmax = order_key(t[0]), tkmin = tkmax;
#pragma unroll
    for (int x = 1; x < NF; ++x) {
      const unsigned long long kx = order_key(t[x]);
      tkmax = kx > tkmax ? kx : tkmax;
      tkmin = kx < tkmin ? kx : tkmin;
    }
    const unsigned long long bp = nonneg_bits(key_value(tkmax) - ub), bn = nonneg_bits(ub - key_value(tkmin));
    const unsigned long long dpos = (bp >> 63) ? 0ull : bp, dneg = (bn >> 63) ? 0ull : bn;
    // numerator and denominator of the smallest ratio as bit patterns of
    // non-negative doubles; 1 / 1: no limiting
    constexpr unsigned long long kOne = 0x3FF0000000000000ull;
    const bool above = dpos != 0ull && nonneg_bits(up) < dpos;
    unsigned long long nbest = above ? nonneg_bits(up) : kOne, dbest = above ? dpos : kOne;
    if (dneg != 0ull && nonneg_bits(dn) < dneg) {
      const bool below = nonneg_bits(dn * bits_value(dbest)) < nonneg_bits(bits_value(nbest) * bits_value(dneg));
      nbest = below ? nonneg_bits(dn) : nbest;
      dbest = below ? dneg : dbest;
    }
    if (nbest < dbest) {
      // alpha = nbest / dbest by the Newton-refined reciprocal (within 1.5 ulp of
      // the quotient); the traces of the scaled coefficients by the same sums
      // every kernel uses, so that they agree bit for bit with k_traces'
      const double alpha = bits_value(nbest) * recip(bits_value(dbest));
      cj[1] *= alpha;
      cj[2] *= alpha;
      ce[1] = cj[1];
      ce[2] = cj[2];
      if (dst) {
        double u[NF];
        face_sums<P>(cj, sChiM1, sChi[0], z);
#pragma unroll
        for (int k = 0; k < NE; ++k) edge_traces_unit<P, NE>(cj, z, sPa, sChi, k, u[k], u[NE + k], u[3 * NE - 1 - k]);
#pragma unroll
        for (int x = 0; x < NF; ++x) dst[x * M] = u[x];
      }
    } else if (!HAVE_TRACES && dst) {
#pragma unroll
      for (int x = 0; x < NF; ++x) dst[x * M] = t[x];
    }
  }
}

}  // namespace
}  // namespace dg
