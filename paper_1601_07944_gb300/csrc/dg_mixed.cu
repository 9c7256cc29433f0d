/*
 * dg_mixed.cu -- mixed-precision element kernel: the three dense contractions of
 * a stage run on the Blackwell tensor cores (tcgen05.mma kind::tf32, FP32
 * accumulation in TMEM), as one TF32 product (DG_TF32X1) or as the split
 * product a_hi b_hi + a_hi b_lo + a_lo b_hi (DG_TF32X3, a = a_hi + a_lo with
 * both parts rounded to TF32).
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
 *
 * The traces are results of float32 accumulation, so they are stored as float32
 * (exactly).  The edge flux (k_face_mixed) widens them exactly and evaluates the
 * Lax-Friedrichs flux in float64, once per edge; it stores the flux rounded to
 * float32 for the lift columns of GEMM 2 and, in float64, the flux's integral
 * against the constant mode.  The mean mode, which carries the conserved totals,
 * is lifted from those float64 integrals: each edge's value enters its two
 * elements with opposite signs.
 */
#include "dg_mixed_tc.cuh"

namespace dg {
namespace {

// Edge flux of the mixed-precision modes, one thread per edge.  The two traces
// are float32 (exact results of the tensor-core contraction) and are widened
// exactly; the local Lax-Friedrichs flux is evaluated in float64 at the NE edge
// points (lax_friedrichs_edge_f32: the flux of k_face, alpha included, with two
// float64 operations fewer for float32 inputs), with the right element's trace
// at the reversed point (Eq. edgeint).  Written per
// edge: l F_hat at the points rounded to float32 (the lift columns of GEMM 2), and
// the float64 integral of l F_hat against the constant mode,
// fmean_m = sum_k omega_k phi_1 l F_hat_{k,m} (Algorithm 2 for j = 1; the
// Gauss-Legendre weights are symmetric, so it is the same from both sides).
// BND: the launch covers the boundary faces [f0, f1) = [0, Fb) (a ghost state on
// the right, Algorithm 2); otherwise the interior faces [Fb, F), in a separate
// instantiation so that the common case carries no boundary code.
template <int NE, bool BND>
__global__ void __launch_bounds__(256)
k_face_mixed(const float *__restrict__ trace, float *__restrict__ fhat, double *__restrict__ fmean,
             const FaceConn *__restrict__ conn, const FaceGeo *__restrict__ fg, const double *__restrict__ Lf,
             const double *__restrict__ bstate, int np, int64_t N, int64_t f0, int64_t f1, double gamma,
             int *err) {
  constexpr int NF = 3 * NE;
  bool ok = true;
  // the grid is what is resident at once; block b takes the b-th of gridDim.x
  // equal slices of the edges
  const int64_t F = f1 - f0;
  const int64_t lo = f0 + F * blockIdx.x / gridDim.x, hi = f0 + F * (blockIdx.x + 1) / gridDim.x;
  for (int64_t f = lo + threadIdx.x; f < hi; f += blockDim.x) {
    const FaceConn cn = conn[f];
    const FaceGeo g = fg[f];
    // [N][NF][M] float32: one point's four values are one aligned float4
    constexpr bool bnd = BND;
    const int64_t el = checked(cn.l, N, err);
    const float4 *tl = reinterpret_cast<const float4 *>(trace) + (size_t)el * NF + checked(cn.L, 3, err) * NE;
    const float4 *tr = reinterpret_cast<const float4 *>(trace) + (size_t)(bnd ? el : checked(cn.r, N, err)) * NF +
                       (bnd ? 0 : checked(cn.R, 3, err) * NE);
    float4 *dst = reinterpret_cast<float4 *>(fhat) + (size_t)f * NE;
    double sm[M] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NE; ++k) {
      const float4 a = tl[k];
      double Fh[M];
      if (bnd) {
        const double ul[M] = {tc::f32_to_f64(a.x), tc::f32_to_f64(a.y), tc::f32_to_f64(a.z), tc::f32_to_f64(a.w)};
        double ur[M];
        ghost_state(cn.r, ul, g.nx, g.ny, bstate + ((size_t)f * NE + k) * M, ur);
        ok &= lax_friedrichs_edge(ul, ur, g, gamma, Fh);
      } else {
        ok &= lax_friedrichs_edge_f32(a, tr[NE - 1 - k], g, gamma, Fh);
      }
      const double w = Lf[k * np];           // omega_k phi_1, the same on the three faces
#pragma unroll
      for (int m = 0; m < M; ++m) sm[m] = fma(w, Fh[m], sm[m]);
      dst[k] = make_float4(tc::f64_to_f32(Fh[0]), tc::f64_to_f32(Fh[1]), tc::f64_to_f32(Fh[2]),
                           tc::f64_to_f32(Fh[3]));
    }
    double2 *dm = reinterpret_cast<double2 *>(fmean + (size_t)f * M);
    dm[0] = make_double2(sm[0], sm[1]);
    dm[1] = make_double2(sm[2], sm[3]);
  }
  if (!ok) atomicOr(err, kErrNonPhysical);
}

// Self-check of the integer float64 <-> float32 conversions against the hardware
// conversions on n values spread over the float32 normal range (both signs, with
// rounding ties and exact zeros among them).
__global__ void k_convert_check(int n, unsigned long long *bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // a deterministic spread of bit patterns: exponent in [-120, 120], random mantissa
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z ^= z >> 31; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 29;
  const int ex = (int)((z >> 52) % 241) - 120;
  unsigned long long mant = z & 0xFFFFFFFFFFFFFull;
  if ((i & 15) == 3) mant = (mant & ~0x1FFFFFFFull) | 0x10000000ull;   // exact float32 rounding tie
  unsigned long long bits = ((unsigned long long)(ex + 1023) << 52) | mant;
  if (i & 1) bits |= 0x8000000000000000ull;
  double x = __longlong_as_double((long long)bits);
  if ((i & 255) == 7) x = (i & 512) ? -0.0 : 0.0;
  const float f_hw = (float)x, f_int = tc::f64_to_f32(x);
  const double d_hw = (double)f_hw, d_int = tc::f32_to_f64(f_hw);
  if (__float_as_uint(f_hw) != __float_as_uint(f_int)) atomicAdd(bad, 1ull);
  if (__double_as_longlong(d_hw) != __double_as_longlong(d_int)) atomicAdd(bad + 1, 1ull);
  // Newton-refined reciprocal and square root against the correctly rounded 1/x
  // and sqrt(x): at most 1 ulp apart; the reciprocal square root against
  // 1/sqrt(x), itself rounded twice: at most 2 ulp apart
  const double ax = fabs(x);
  if (ax != 0.0) {
    const long long q = __double_as_longlong(1.0 / ax), r = __double_as_longlong(recip(ax));
    const long long d = q > r ? q - r : r - q;
    if (d > 1) atomicAdd(bad + 2, 1ull);
    const long long qs = __double_as_longlong(sqrt(ax)), rs = __double_as_longlong(sqrt_nr(ax));
    const long long ds = qs > rs ? qs - rs : rs - qs;
    const long long qr = __double_as_longlong(1.0 / sqrt(ax)), rr = __double_as_longlong(rsqrt_nr(ax));
    const long long dr = qr > rr ? qr - rr : rr - qr;
    if (ds > 1 || dr > 2) atomicAdd(bad + 3, 1ull);
  }
}

}  // namespace

int launch_convert_check(int n, unsigned long long *bad, void *stream) {
  k_convert_check<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, bad);
  return (int)cudaGetLastError();
}

int tc_tables(dg_mesh *m) {
  return m->rule == DG_RULE_SYMMETRIC ? tc_tables_sym(m) : tc_tables_rule<false>(m);
}

int launch_element_tc(const dg_mesh *m, int split3, const double *c, const double *u0, double *out,
                      float *trace_out, const float *fhat, const double *fmean, const StageUpdate &su,
                      int mode, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (m->rule == DG_RULE_SYMMETRIC)
    return launch_element_tc_sym(m, split3, c, u0, out, trace_out, fhat, fmean, su, mode, stream);
  return split3 ? dispatch_tc<true, false>(m, c, u0, out, trace_out, fhat, fmean, su, mode, s)
                : dispatch_tc<false, false>(m, c, u0, out, trace_out, fhat, fmean, su, mode, s);
}

MixedBuffers mixed_buffers(const dg_mesh *m, double *trace, double *fhat) {
  MixedBuffers b;
  b.trace = reinterpret_cast<float *>(trace);
  b.fhat = reinterpret_cast<float *>(fhat);
  b.fmean = reinterpret_cast<double *>(b.fhat + (size_t)m->F * m->ne * M);   // byte offset F ne 16
  return b;
}

int launch_face_flux_mixed(const dg_mesh *m, const MixedBuffers &b, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
#define FACE(NE)                                                                                          \
  do {                                                                                                    \
    static int per_sm = 0, per_sm_b = 0;                                                                  \
    k_face_mixed<NE, false><<<resident_grid(m, (const void *)k_face_mixed<NE, false>, 256, m->F - m->Fb,   \
                                            &per_sm), 256, 0, s>>>(                                       \
        b.trace, b.fhat, b.fmean, m->face_conn, m->face_geo, m->tab.Lf, m->bstate, m->np, m->N, m->Fb, m->F, \
        m->gamma, m->err_flag);                                                                           \
    if (m->Fb > 0)                                                                                        \
      k_face_mixed<NE, true><<<resident_grid(m, (const void *)k_face_mixed<NE, true>, 256, m->Fb,         \
                                             &per_sm_b), 256, 0, s>>>(                                    \
          b.trace, b.fhat, b.fmean, m->face_conn, m->face_geo, m->tab.Lf, m->bstate, m->np, m->N, 0, m->Fb, \
          m->gamma, m->err_flag);                                                                         \
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

}  // namespace dg

