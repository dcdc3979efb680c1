// Double-word and double-float arithmetic on the FP32 pipe, shared by the
// double-float sweeps (solve_fp64.cu) and the tensor-core sweep (solve_tc.cu).
#pragma once
#include "ssv_internal.cuh"

namespace ssv {

// Double-word scalars (hi + lo, |lo| <= ulp(hi) / 2) on the FP32 pipe, for the
// few per-row reflector quantities of the double-float panel: Knuth's two-sum,
// Dekker's fast two-sum, FMA-exact products, one correction step for the
// quotient and for the square root (Newton on s^2 = x).  About 44 bits each.
struct dw {
  float hi, lo;
};
static __device__ __forceinline__ dw dw_fast(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return dw{s, b - (s - a)};
}
static __device__ __forceinline__ dw dw_add(dw x, dw y) {
  const float s = x.hi + y.hi;
  const float bb = s - x.hi;
  const float e = (x.hi - (s - bb)) + (y.hi - bb);
  return dw_fast(s, e + (x.lo + y.lo));
}
static __device__ __forceinline__ dw dw_mul(dw x, dw y) {
  const float p = x.hi * y.hi;
  const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
  return dw_fast(p, e);
}
static __device__ __forceinline__ dw dw_div(dw x, dw y) {
  const float q1 = x.hi / y.hi;
  // x - q1 y: the leading part is exact by FMA
  const float r = fmaf(-q1, y.hi, x.hi) + fmaf(-q1, y.lo, x.lo);
  return dw_fast(q1, r / y.hi);
}
static __device__ __forceinline__ dw dw_sqrt(dw x) {
  if (!(x.hi > 0.f)) return dw{0.f, 0.f};
  const float s = sqrtf(x.hi);
  const float e = fmaf(-s, s, x.hi) + x.lo;
  return dw_fast(s, e / (2.f * s));
}
// complex128 <-> double-float (re_hi, re_lo, im_hi, im_lo)
static __device__ __forceinline__ float4 df_split(cd z) {
  const float rh = (float)z.x, ih = (float)z.y;
  return make_float4(rh, (float)(z.x - (double)rh), ih, (float)(z.y - (double)ih));
}
static __device__ __forceinline__ cd df_join(float4 w) {
  return mkcd((double)w.x + (double)w.y, (double)w.z + (double)w.w);
}

}  // namespace ssv
