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

// ---------------------------------------------------------------- pairs
// The same transformations on two independent lanes at once with the packed
// float32 pair instructions (add/sub/mul/fma .rn.f32x2): each lane is an
// ordinary round-to-nearest float32 operation, so every identity above holds
// lane by lane.
struct p2 {
  unsigned long long v;
};
__device__ __forceinline__ p2 mk2(float a, float b) {
  p2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 un2(p2 x) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(x.v));
  return r;
}
__device__ __forceinline__ p2 add2(p2 a, p2 b) {
  p2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ p2 sub2(p2 a, p2 b) {
  p2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ p2 mul2(p2 a, p2 b) {
  p2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ p2 fma2(p2 a, p2 b, p2 c) {
  p2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ p2 neg2(p2 a) {
  p2 r;
  r.v = a.v ^ 0x8000000080000000ull;
  return r;
}

struct df2 {
  p2 h, l;
};
__device__ __forceinline__ df2 two_sum2(p2 a, p2 b) {
  const p2 s = add2(a, b);
  const p2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ df2 fast_two_sum2(p2 a, p2 b) {
  const p2 s = add2(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ df2 two_prod2(p2 a, p2 b) {
  const p2 p = mul2(a, b);
  return {p, fma2(a, b, neg2(p))};
}
__device__ __forceinline__ df2 df_mul2(df2 a, df2 b) {
  df2 p = two_prod2(a.h, b.h);
  p.l = fma2(a.h, b.l, p.l);
  p.l = fma2(a.l, b.h, p.l);
  return fast_two_sum2(p.h, p.l);
}

}  // namespace rr
