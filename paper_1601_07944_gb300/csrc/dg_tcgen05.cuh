/*
 * dg_tcgen05.cuh -- the small set of Blackwell (sm_100a/sm_103a) tensor-core
 * primitives the mixed-precision kernels use, as inline PTX:
 *
 *   tcgen05.alloc / dealloc        tensor-memory (TMEM) columns for the accumulator
 *   tcgen05.mma.cta_group::1.kind::tf32
 *                                  D[128 x N] (+)= A[128 x 8] B[8 x N], A and B in
 *                                  shared memory, D in TMEM, FP32 accumulation
 *   tcgen05.mma ... [a-tmem]       the same with A read from TMEM (lane = row of
 *                                  A, one column per TF32 element along K)
 *   tcgen05.commit -> mbarrier     completion of the issued MMAs
 *   tcgen05.ld.32x32b              TMEM -> registers (each warp reads its own
 *                                  32-lane quarter; lane = accumulator row)
 *   tcgen05.st.32x32b              registers -> TMEM (the same lane mapping)
 *
 * Operand layout: K-major without swizzle.  The tile is made of core matrices of
 * 8 rows x 16 bytes (8 rows x 4 TF32 values) stored as 128 contiguous bytes; the
 * core matrix holding K elements 4c..4c+3 of rows 8g..8g+7 starts at byte
 * g * (Ktot * 32) + c * 128.  In the shared-memory descriptor the leading byte
 * offset (LBO, next core matrix along K) is 128 and the stride byte offset (SBO,
 * next 8-row group) is Ktot * 32.  One MMA consumes K = 8, i.e. two core
 * matrices along K, so the descriptor of k-step s starts s * 256 bytes in.
 */
#pragma once

#include <cstdint>

namespace dg {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) of a K-major tile with ktot columns
__host__ __device__ constexpr int kmaj(int row, int k, int ktot) {
  return (row >> 3) * (ktot * 32) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: no swizzle, LBO = 128, SBO = ktot * 32
__device__ __forceinline__ uint64_t desc(uint32_t addr, int ktot) {
  const uint32_t sbo = (uint32_t)ktot * 32u;
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                       // descriptor version (fixed 0b001)
  return d;
}

// instruction descriptor: D f32, A and B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// A operand in tensor memory: A[row][k] at lane row, column a_tmem + k (K-major;
// one K = 8 step reads eight consecutive columns)
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Waits for the mbarrier phase `parity` to complete; gives up after limit_ns
// nanoseconds and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint64_t limit_ns) {
  uint32_t done = 0;
  const uint64_t t0 = global_ns();
  while (true) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// The same, with the waiting threads suspended (up to suspend_ns per try) instead
// of polling, so that they take fewer issue slots from the other warps of the
// SM; the clock is read on every eighth try.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t mbar, uint32_t parity, uint64_t limit_ns,
                                                uint32_t suspend_ns) {
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity), "r"(suspend_ns));
    if (done) return true;
    if ((it & 7u) == 0u) {
      const uint64_t t = global_ns();
      if (it == 0u) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

// the calling thread arrives on the mbarrier and adds tx_bytes to the bytes the
// current phase waits for (the bulk copies below complete them)
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t tx_bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(tx_bytes) : "memory");
}

// bulk copy (TMA, not tiled) of `bytes` bytes global -> shared memory, completing
// on the mbarrier; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst_smem, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   dst_smem),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;"); }

// one warp: allocates ncols TMEM columns, writes the base address to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_smem), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective)
__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;"); }

// 8 consecutive 32-bit columns of this thread's TMEM lane from v (warp-collective)
__device__ __forceinline__ void st8(uint32_t taddr, const uint32_t *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// TF32 rounding of a float32 bit pattern, to nearest with ties away from zero
// (an add on the magnitude bits, then the 13 low bits cleared)
__device__ __forceinline__ uint32_t tf32_bits(uint32_t b) { return (b + 0x1000u) & 0xFFFFE000u; }

// float64 -> float32 truncated toward zero, branchless, on the bit patterns:
// magnitudes below the float32 normal range give signed zero, magnitudes of 2^128
// and above (and non-finite values) give signed infinity.  (The tensor-core
// operands round this value to TF32 again, so truncation costs nothing there.)
__device__ __forceinline__ uint32_t f64_to_f32_rz_bits(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t ah = hi & 0x7FFFFFFFu;
  uint32_t f = __funnelshift_l(lo, ah - 0x38000000u, 3);   // exponent rebias, 23 mantissa bits
  f = ah < 0x38100000u ? 0u : f;
  f = ah >= 0x47F00000u ? 0x7F800000u : f;
  return f | (hi & 0x80000000u);
}

// float32 -> float64, exact for zeros and normal values, branchless; float32
// subnormals (below 2^-126) come out within 2^-126 of their value, non-finite
// values as finite values of magnitude 2^128 or more.
__device__ __forceinline__ double f32_to_f64_fast(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ab = b & 0x7FFFFFFFu;
  uint32_t hi = (ab >> 3) + 0x38000000u;
  hi = ab == 0u ? 0u : hi;
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(b << 29));
}

// round an FP32 value to TF32 (10 mantissa bits, round to nearest, ties away)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float32 -> float64 from the bit pattern (exact), with integer instructions only.
// Zeros and float32 subnormals map to signed zero; non-finite values keep their
// class.  (The float64 pipe of this GPU is narrow; conversions through it would
// compete with the stage update.)
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t sign = b & 0x80000000u;
  uint32_t hi = sign, lo = 0u;
  if (e != 0u) {
    const uint32_t e64 = e == 0xFFu ? 0x7FFu : e + 896u;
    hi = sign | (e64 << 20) | ((b & 0x7FFFFFu) >> 3);
    lo = b << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// float64 -> float32, round to nearest even, from the bit pattern with integer
// instructions only.  Magnitudes below the float32 normal range flush to signed
// zero; above it, to infinity.
__device__ __forceinline__ float f64_to_f32(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 896;        // float32 biased exponent
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  uint32_t f = ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rnd = (lo >> 28) & 1u, sticky = (lo & 0x0FFFFFFFu) != 0u, lsb = f & 1u;
  f += rnd & (sticky | lsb);                              // a carry rolls into the exponent
  return __uint_as_float(sign | f);
}

// -x for a float64 by flipping the sign bit (integer instruction)
__device__ __forceinline__ double neg_bits(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

}  // namespace tc
}  // namespace dg
