// Float-float ("double-float") arithmetic: a value is the unevaluated sum hi + lo of two
// binary32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  Built from the
// error-free transformations
//   two_sum      (Knuth, TAOCP vol. 2, 4.2.2):  a + b = s + e exactly, any a, b;
//   fast_two_sum (Dekker 1971):                  the same for |a| >= |b|, three operations;
//   two_prod     (with a fused multiply-add):    a b = p + e exactly, e = fma(a, b, -p).
// The explicitly rounded intrinsics keep the compiler from contracting a product and a
// sum into one FMA, which would break the exactness of the transformations.
//
// On this GPU a binary64 FMA costs as much issue time on its pipe as 64 binary32
// instructions, so a float-float multiply-add (~17 binary32 instructions) is several
// times cheaper than binary64 where ~46 bits suffice.
#pragma once

#include <cuda_runtime.h>

namespace ez {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff{p, __fmaf_rn(a, b, -p)};
}

// a + b; the error is bounded relative to |a| + |b| (no cancellation analysis needed
// where the sum is well conditioned, as in Horner steps and sums of positive terms)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = ff_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, s.lo);
}

// a + b with a binary32 b
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = ff_two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return ff_fast_two_sum(s.hi, s.lo);
}

// a b (the lo * lo product, below 2^-48 relative, is dropped)
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = ff_two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return ff_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_sqr(ff a) {
  ff p = ff_two_prod(a.hi, a.hi);
  p.lo = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
  return ff_fast_two_sum(p.hi, p.lo);
}

// (a_hi + a_lo) + (b_hi + b_lo) from four binary32 parts
__device__ __forceinline__ ff ff_add4(float a_hi, float a_lo, float b_hi, float b_lo) {
  ff s = ff_two_sum(a_hi, b_hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a_lo, b_lo));
  return ff_fast_two_sum(s.hi, s.lo);
}

// 1 / a: binary32 reciprocal refined by one Newton step with the residual 1 - a y
// computed exactly by fma
__device__ __forceinline__ ff ff_rcp(ff a) {
  const float y = __frcp_rn(a.hi);
  float e = __fmaf_rn(-a.hi, y, 1.0f);
  e = __fmaf_rn(-a.lo, y, e);
  return ff_fast_two_sum(y, __fmul_rn(y, e));
}

// sqrt(a), a > 0: binary32 root refined by one Newton step, a - y^2 from two_prod
__device__ __forceinline__ ff ff_sqrt(ff a) {
  const float y = sqrtf(a.hi);
  const ff p = ff_two_prod(y, y);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
  return ff_fast_two_sum(y, __fdividef(r, __fmul_rn(2.0f, y)));
}

// split of a binary64 value (setup and per-node code; not for inner loops)
__host__ __device__ __forceinline__ void ff_split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

// the same split with two binary64-pipe operations instead of four: hi = x truncated to 24
// significant bits, assembled by integer operations from the bits of x (binary32 normal
// range; else the rounded split), lo = x - hi (exact in binary64) rounded to binary32.
// |lo| <= ulp(hi): a float-float value of ~47 bits.
__device__ __forceinline__ void ff_split_trunc(double x, float& hi, float& lo) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e > 896 && e < 1151) {
    hi = __int_as_float((int)((b >> 32) & 0x80000000LL) | ((e - 896) << 23) | (int)((b >> 29) & 0x7fffff));
    lo = (float)(x - __longlong_as_double(b & ~0x1fffffffLL));
  } else {
    ff_split(x, hi, lo);
  }
}

}  // namespace ez
