// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two floats (~48 significant bits), computed on the float32 pipes, which on
// GB300 run ~64x faster than its float64 units.
//
// Error-free transformations used (published methods):
//   TwoSum   -- Knuth, TAOCP Vol. 2, Sec. 4.2.2: s + e = a + b exactly;
//   Fast2Sum -- Dekker, Numer. Math. 18 (1971): same, for |a| >= |b|;
//   TwoProd  -- with a fused multiply-add (Ogita, Rump, Oishi, SISC 2005):
//               p + e = a * b exactly.
// The explicit __f*_rn intrinsics keep the compiler from contracting or
// reassociating the compensated operations.
#pragma once

namespace rr {

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// (a.h + a.l) * (b.h + b.l), dropping the a.l * b.l term (< 2^-48 relative)
__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.h, b.h);
  p.l = __fmaf_rn(a.h, b.l, p.l);
  p.l = __fmaf_rn(a.l, b.h, p.l);
  return fast_two_sum(p.h, p.l);
}

// acc += a (a, acc df); result renormalised
__device__ __forceinline__ df df_add(df acc, df a) {
  df s = two_sum(acc.h, a.h);
  s.l = __fadd_rn(s.l, __fadd_rn(acc.l, a.l));
  return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ df df_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

}  // namespace rr
