// Blackwell tensor-core building blocks (tcgen05, sm_100a / sm_103a) for the tensor-core
// form of the corner sweep: TMEM allocation, shared-memory matrix descriptors, the
// kind::tf32 MMA with its completion through an mbarrier, and TMEM loads.
//
// Operand layout (both operands K-major, no swizzle).  A matrix of R rows and C columns
// (C a multiple of 4, R a multiple of 8) is stored as "core matrices" of 8 rows x 4 FP32
// values (16 bytes per row, 128 bytes each), the core matrix of row group r8 and column
// group k4 at ((k4 * R / 8) + r8) * 128 bytes.  For one MMA over 8 columns of K (two core
// matrices along K), the descriptor's leading-dimension byte offset is the distance
// between the two column groups (R / 8 * 128) and the stride byte offset the distance
// between row groups (128).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pdgdev {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Offset (in floats) of element (row, k) of an R-row operand in the core-matrix layout.
__host__ __device__ __forceinline__ int op_index(int row, int k, int R) {
  return (((k >> 2) * (R >> 3) + (row >> 3)) << 5) + ((row & 7) << 2) + (k & 3);
}

// TF32 rounding of an FP32 value (10 explicit mantissa bits, to nearest, ties away).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// ---- exact conversions by integer operations on the IEEE bit patterns ----
// GB300's FP64 pipe runs 1/62 of its FP32 rate, and conversions between FP64 and FP32 use
// it too; these replace them with integer arithmetic.  Magnitudes below 2^-126 (and zero)
// map to zero (the scheme's values are O(1): that absolute error, < 2^-126, is far below
// its rounding); infinities and NaNs are not expected and not handled.

// FP32 value from its parts; a biased exponent <= 0 (below the normal range) gives zero.
__device__ __forceinline__ float f32_from_parts(unsigned sign, int ebiased, unsigned mant23) {
  if (ebiased <= 0) return 0.0f;
  return __uint_as_float((sign << 31) | ((unsigned)ebiased << 23) | mant23);
}

// Round the nonzero magnitude a (leading bit p < 63) to `bits` significant bits, to nearest
// with ties away from zero: returns the significand (leading one at bit bits - 1) and adds
// the carry of a round-up past a power of two to *p.
template <int bits>
__device__ __forceinline__ unsigned round_sig(unsigned long long a, int* p) {
  unsigned long long m;
  if (*p >= bits) {
    const int sh = *p - (bits - 1);
    m = (a + (1ull << (sh - 1))) >> sh;
    if (m == (1ull << bits)) {
      m >>= 1;
      ++*p;
    }
  } else {
    m = a << ((bits - 1) - *p);
  }
  return (unsigned)m;
}

// x = hi + lo exactly, hi = x rounded to `bits` significant bits (nearest, ties away), lo =
// the remainder rounded to `bits` significant bits the same way (so |x - hi - lo| is about
// 2^(-2 bits) |x|).  bits = 11: the two TF32 parts of a tensor-core operand; bits = 24: a
// double-float pair.
template <int bits>
__device__ __forceinline__ void split_f64_bits(double x, float* hi, float* lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 63);
  const int e = (int)((u >> 52) & 0x7ff);   // biased FP64 exponent
  if (e <= 1023 - 126) {
    *hi = 0.0f;
    *lo = 0.0f;
    return;
  }
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // x = M 2^(e - 1075)
  constexpr int sh = 53 - bits;
  unsigned long long Mh = (M + (1ull << (sh - 1))) >> sh;
  const long long R = (long long)M - (long long)(Mh << sh);               // |R| <= 2^(sh - 1)
  int eh = e;
  if (Mh == (1ull << bits)) {
    Mh >>= 1;
    ++eh;
  }
  *hi = f32_from_parts(sign, eh - 1023 + 127, (unsigned)(Mh & ((1ull << (bits - 1)) - 1)) << (24 - bits));
  if (R == 0) {
    *lo = 0.0f;
    return;
  }
  const unsigned long long a = (unsigned long long)(R < 0 ? -R : R);
  int p = 63 - __clzll((long long)a);                                      // a = 1.f 2^p
  const unsigned ml = round_sig<bits>(a, &p);
  *lo = f32_from_parts(sign ^ (R < 0 ? 1u : 0u), e - 1075 + p + 127, (ml & ((1u << (bits - 1)) - 1)) << (24 - bits));
}

// x truncated to 24 significant bits, as an FP32 value built from the FP64 bit pattern (sign,
// rebiased exponent, the top 23 mantissa bits); *e gets the FP64 biased exponent and *lw the
// low 32 bits of the pattern.  Returns false (value 0) outside the normal FP32 range.
__device__ __forceinline__ bool f32_trunc_bits(double x, float* t, int* e, unsigned* lw) {
  const unsigned hw = (unsigned)__double2hiint(x);
  *lw = (unsigned)__double2loint(x);
  *e = (int)((hw >> 20) & 0x7ffu);
  if (*e <= 1023 - 127 || *e >= 1023 + 128) {
    *t = 0.0f;
    return false;
  }
  *t = __uint_as_float((hw & 0x80000000u) | ((unsigned)(*e - 1023 + 127) << 23) | ((hw & 0xfffffu) << 3) |
                       (*lw >> 29));
  return true;
}

// The two TF32 parts of an FP64 value, |x - hi - lo| <= 2^-22 |x| (the precision of
// split_f64_bits<11>, with far fewer operations): hi = the 24-bit truncation rounded to TF32,
// lo = the exact FP32 remainder of that truncation rounded to TF32.
__device__ __forceinline__ void split_tf32_fast(double x, float* hi, float* lo) {
  float t;
  int e;
  unsigned lw;
  f32_trunc_bits(x, &t, &e, &lw);
  *hi = tf32_rna(t);
  *lo = tf32_rna(__fsub_rn(t, *hi));
}

// An FP64 value as an unevaluated FP32 pair, |x - hi - lo| <= 2^-48 |x| for |x| >= 2^-74
// (absolute error below 2^-98 under it): hi = the 24-bit truncation, lo = the remaining 29
// mantissa bits (an integer below 2^29, rounded to FP32) times 2^(e - 1075), the scale an
// exact power of two.
__device__ __forceinline__ void split_dd_fast(double x, float* hi, float* lo) {
  float t;
  int e;
  unsigned lw;
  if (!f32_trunc_bits(x, &t, &e, &lw)) {
    *hi = 0.0f;
    *lo = 0.0f;
    return;
  }
  *hi = t;
  const int se = e - 1075 + 127;
  if (se <= 0) {
    *lo = 0.0f;
    return;
  }
  const float m = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)se << 23));
  *lo = __double2hiint(x) < 0 ? -m : m;
}

// The FP64 value of an FP32 value (exact).
__device__ __forceinline__ double f64_from_f32_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0) return 0.0;
  const unsigned long long u = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)(e + 896) << 52) |
                               ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)u);
}

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (all
// multiples of 16 bytes), descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in FP32, A and B in TF32, both K-major, dense,
// no negation; N at bits 17-22 (N / 8), M at bits 24-28 (M / 16).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on the mbarrier when every MMA this thread issued so far has completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete, for at most `max_cycles` SM clock
// cycles; returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, long long max_cycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}

// TMEM allocation (a whole warp): the base address is written to shared memory.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make this thread's generic-proxy shared-memory writes visible to the tensor cores.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Load X consecutive 32-bit columns of this thread's TMEM lane (the warp's 32-lane
// quarter, shape 32x32b) and wait for the load, in one asm block, so that the values are
// complete where they are defined.
template <int X>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_ld<4>(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace pdgdev
