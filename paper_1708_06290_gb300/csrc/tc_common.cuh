// tcgen05 / mbarrier / bulk-copy helpers (inline PTX) and the error-free BF16
// digit splitting shared by the tensor-core residual (residual_tc.cu) and the
// tensor-core sweep (solve_tc.cu).
#pragma once
#include <stdint.h>

#include "ssv_internal.cuh"

namespace ssv {
namespace tcg {

constexpr int kDigits = 8;               // 7-bit digits per value (56 bits)
constexpr int kBadExp = 0x40000000;      // exponent marker of a non-finite row / column
constexpr long long kWaitLimit = 1LL << 26;

// 2^E > |x| for the largest |x| of a row / column: E from the exponent field
static __device__ __forceinline__ int scale_exp(double maxabs) {
  if (!(maxabs <= 1.7976931348623157e308)) return kBadExp;  // Inf or NaN
  const unsigned long long b = (unsigned long long)__double_as_longlong(maxabs);
  const int ef = (int)((b >> 52) & 0x7ff);
  return ef == 0 ? -1022 : ef - 1022;
}

// the eight 7-bit digits of x relative to 2^E, as BF16 bit patterns
static __device__ __forceinline__ void digits8(double x, int E, unsigned short (&d)[kDigits]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned short sgn = (unsigned short)((b >> 63) << 15);
  const int ef = (int)((b >> 52) & 0x7ff);
  unsigned long long mant = b & ((1ull << 52) - 1);
  int ex = ef;
  if (ef == 0) ex = 1;
  else mant |= 1ull << 52;
  // M = |x| 2^{56 - E} = mant 2^{ex - 1019 - E} < 2^56
  const int sh = ex - 1019 - E;
  unsigned long long M = 0;
  if (E != kBadExp) {
    if (sh >= 0) M = mant << sh;  // sh <= 3 because |x| < 2^E
    else if (sh > -64) M = mant >> (-sh);
  }
#pragma unroll
  for (int l = 0; l < kDigits; ++l) {
    const unsigned int dig = (unsigned int)(M >> (49 - 7 * l)) & 127u;
    // dig is exact in FP32 (magic-number conversion) and, having at most 7
    // significant bits, in BF16 (the top half of the FP32 pattern)
    const float f = __uint_as_float(0x4B000000u | dig) - 8388608.0f;
    d[l] = (unsigned short)(__float_as_uint(f) >> 16) | sgn;
  }
}

// 2^E > |x| for the largest |x| of a row of FP32 high words (a double-float row:
// |hi + lo| < 2^E as well, since |lo| <= ulp(hi) / 2), from the exponent field
static __device__ __forceinline__ int scale_exp_f(float maxabs) {
  const unsigned b = __float_as_uint(maxabs);
  if ((b & 0x7f800000u) == 0x7f800000u) return kBadExp;  // Inf or NaN
  const int eb = (int)((b >> 23) & 0xffu);
  return eb == 0 ? -126 : eb - 126;
}

// the seven 7-bit digits of x = hi + lo (a double-float value, |x| < 2^E)
// relative to 2^E, as BF16 bit patterns: each word's 24-bit significand is
// shifted to units of 2^{E - 56} (truncated toward zero) from its bit fields,
// the low word with its own sign, so no FP64 arithmetic is involved
static __device__ __forceinline__ void digits7_pair(float hi, float lo, int E, unsigned short (&d)[7]) {
  auto part = [E](float f) -> long long {
    const unsigned b = __float_as_uint(f);
    const int eb = (int)((b >> 23) & 0xffu);
    const long long mi = (long long)(b & 0x7fffffu) | (eb ? (1ll << 23) : 0ll);
    const int sh = (eb ? eb : 1) - 94 - E;
    const long long v = sh >= 0 ? (mi << sh) : (sh > -64 ? (mi >> (-sh)) : 0ll);
    return (b >> 31) ? -v : v;
  };
  const long long M = (E == kBadExp) ? 0ll : part(hi) + part(lo);
  const unsigned short sgn = M < 0 ? (unsigned short)0x8000u : (unsigned short)0u;
  const unsigned long long U = (unsigned long long)(M < 0 ? -M : M);
#pragma unroll
  for (int l = 0; l < 7; ++l) {
    const unsigned int dig = (unsigned int)(U >> (49 - 7 * l)) & 127u;
    const float f = __uint_as_float(0x4B000000u | dig) - 8388608.0f;
    d[l] = (unsigned short)(__float_as_uint(f) >> 16) | sgn;
  }
}

// element offset in a K-major core-matrix tile with kg core matrices along K
// (8 rows x 8 K elements per 128 bytes; byte strides 128 along K, kg * 128
// along rows)
__host__ __device__ __forceinline__ int tile_off_kg(int row, int k, int kg) {
  return (((row >> 3) * kg + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7);
}

static __device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte stride of
// core matrices along K, sbo = along M / N
static __device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, N, M
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

static __device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                                uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
static __device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
static __device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase,
                                                 long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}
static __device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
static __device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 1-D bulk copy global -> shared (TMA), completing `bytes` on the mbarrier
static __device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
static __device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
static __device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
static __device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tcg
}  // namespace ssv
