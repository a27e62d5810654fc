// Packed single-precision pairs for sm_100+ (FADD2 / FMUL2 / FFMA2): one
// instruction operates on the two radially adjacent nodes a thread owns.
// Also the float-float (hi + lo) error-free transformations on pairs.
#pragma once

#include <cuda_runtime.h>

namespace pclb {

typedef float2 f2;

__device__ __forceinline__ f2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 bc2(float a) { return make_float2(a, a); }

__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

// a - b, exactly the rounded difference (the negation is exact)
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ f2 abs2(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }

// Error-free transformations (Knuth two-sum, fma two-product) on pairs.
__device__ __forceinline__ void two_sum2(f2 a, f2 b, f2& s, f2& e) {
  s = add2(a, b);
  const f2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ void two_prod2(f2 a, f2 b, f2& p, f2& e) {
  p = mul2(a, b);
  e = fma2(a, b, neg2(p));
}

// Float-float pairs: value = hi + lo for each of the two nodes.
struct ff2 {
  f2 hi, lo;
};

__device__ __forceinline__ ff2 ff2_of(f2 x) { return ff2{x, bc2(0.f)}; }

__device__ __forceinline__ ff2 ff2_renorm(f2 s, f2 lo) {
  ff2 r;
  r.hi = add2(s, lo);
  r.lo = sub2(lo, sub2(r.hi, s));
  return r;
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b) {
  f2 s, se;
  two_sum2(a.hi, b.hi, s, se);
  return ff2_renorm(s, add2(se, add2(a.lo, b.lo)));
}
__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b) {
  f2 p, e;
  two_prod2(a.hi, b.hi, p, e);
  e = fma2(a.hi, b.lo, fma2(a.lo, b.hi, e));
  return ff2_renorm(p, e);
}
// a * b + c
__device__ __forceinline__ ff2 ff2_mul_add(ff2 a, ff2 b, ff2 c) {
  f2 p, pe, s, se;
  two_prod2(a.hi, b.hi, p, pe);
  pe = fma2(a.hi, b.lo, fma2(a.lo, b.hi, pe));
  two_sum2(p, c.hi, s, se);
  return ff2_renorm(s, add2(se, add2(pe, c.lo)));
}
__device__ __forceinline__ ff2 ff2_scale(ff2 a, float s) { return ff2{mul2(a.hi, bc2(s)), mul2(a.lo, bc2(s))}; }
__device__ __forceinline__ ff2 ff2_recip(ff2 a) {
  const f2 r0 = make_float2(__frcp_rn(a.hi.x), __frcp_rn(a.hi.y));
  const f2 e = sub2(fma2(neg2(a.hi), r0, bc2(1.f)), mul2(a.lo, r0));   // 1 - a r0
  return ff2_renorm(r0, mul2(r0, e));
}
__device__ __forceinline__ f2 ff2_round(ff2 a) { return add2(a.hi, a.lo); }

}  // namespace pclb
