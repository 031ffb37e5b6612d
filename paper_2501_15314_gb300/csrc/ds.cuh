// Double-single arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits).  GB300 runs FP64 arithmetic, and
// conversions between FP64 and FP32, at about 1/58 of its FP32 rate, so the
// FP64-accurate parts of the hot path that would otherwise be bound by the
// FP64 pipe are written with these error-free transformations on the FP32
// pipes:
//   two_sum(a, b):  s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a
//                   (Knuth), exact: a + b = s + e;
//   two_prod(a, b): p = a b, e = fma(a, b, -p), exact: a b = p + e.
// Explicit __f*_rn intrinsics keep the compiler from contracting or
// re-associating them.
#pragma once

#include <cstdint>

namespace ibm {

struct dsf {
  float hi, lo;
};

__device__ __forceinline__ dsf two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dsf fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dsf two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// (a.hi + a.lo) + (b.hi + b.lo)
__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
  dsf s = two_sum(a.hi, b.hi);
  const dsf t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
// The same sum with one two_sum (Dekker's addition): the error is within a
// few units of 2^-46 (|a| + |b|) instead of 2^-46 |a + b|, for 11 FP32
// operations instead of 20; enough where the operands' own representation
// error (2^-46 of each) already bounds the result's.
__device__ __forceinline__ dsf ds_add_d(dsf a, dsf b) {
  const dsf s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dsf ds_neg(dsf a) { return {-a.hi, -a.lo}; }
// (a.hi + a.lo) + b for an FP32 b
__device__ __forceinline__ dsf ds_add_f(dsf a, float b) {
  dsf s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}
// (a.hi + a.lo) * (b.hi + b.lo), dropping lo*lo
__device__ __forceinline__ dsf ds_mul(dsf a, dsf b) {
  dsf p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// (a.hi + a.lo) * b for an FP32 b
__device__ __forceinline__ dsf ds_mul_f(dsf a, float b) {
  dsf p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// x = hi + lo to within 2^-46 |x| without FP64 arithmetic or conversions
// (which run on the slow FP64 pipe): hi takes the sign, the exponent and the
// top 23 fraction bits of x, lo the next 23 fraction bits, read as an integer
// (exactly, through the FP32 significand of 2^23 + m) and scaled by a power
// of two; the lowest 6 fraction bits are dropped.  Integer operations only,
// also on the edge cases: |x| < 2^-80 (zero, subnormal or far below the
// values of the flow) gives (0, 0), |x| >= 2^101 (and inf, NaN) gives
// (+-inf, 0), which the callers' finiteness checks report.
__device__ __forceinline__ dsf split_exact(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ffu) - 1023;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (E < -80) return {0.f, 0.f};
  if (E > 100) return {__uint_as_float(sign | 0x7f800000u), 0.f};
  const float hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) |
                                   (unsigned)((b >> 29) & 0x7fffffu));
  const unsigned m23 = (unsigned)((b >> 6) & 0x7fffffu);
  const float mf = __fsub_rn(__uint_as_float(0x4b000000u | m23), 8388608.0f);
  const float lo = __fmul_rn(mf, __uint_as_float((unsigned)(E - 46 + 127) << 23));
  return {hi, __uint_as_float(__float_as_uint(lo) | sign)};
}

// Exact FP64 value of an FP32 number without the FP64 pipe: sign, re-biased
// exponent and the 23 fraction bits moved into place (integer operations
// only); subnormal x, far below the values of the flow, give +-0, inf and
// NaN keep their class.
__device__ __forceinline__ double f2d_exact(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned long long frac = (unsigned long long)(u & 0x7fffffu) << 29;
  const unsigned long long e64 = ex == 0u ? 0ull
                                          : (ex == 0xffu ? 0x7ffull
                                                         : (unsigned long long)(ex + (1023u - 127u)));
  return __longlong_as_double((long long)(sign | (e64 << 52) | (ex == 0u ? 0ull : frac)));
}

// The same transformations on two independent values at once, with the
// paired FP32 instructions of sm_100 and later (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: each component rounds exactly as the scalar instruction, so a
// pair computes bit for bit what two scalar chains would, in half the
// instructions).  dsf2 holds two double-single values: (hi.x, lo.x) and
// (hi.y, lo.y).
struct dsf2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ dsf2 two_sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 bb = fsub2(s, a);
  const float2 e = __fadd2_rn(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
  return {s, e};
}
__device__ __forceinline__ dsf2 fast_two_sum2(float2 a, float2 b) {   // |a| >= |b| per component
  const float2 s = __fadd2_rn(a, b);
  return {s, fsub2(b, fsub2(s, a))};
}
__device__ __forceinline__ dsf2 two_prod2(float2 a, float2 b) {
  const float2 p = __fmul2_rn(a, b);
  return {p, __ffma2_rn(a, b, neg2(p))};
}
// each component of a times the double-single b (dropping lo*lo), as ds_mul
__device__ __forceinline__ dsf2 ds_mul2(dsf2 a, dsf b) {
  const float2 bh = make_float2(b.hi, b.hi), bl = make_float2(b.lo, b.lo);
  dsf2 p = two_prod2(a.hi, bh);
  p.lo = __ffma2_rn(a.hi, bl, p.lo);
  p.lo = __ffma2_rn(a.lo, bh, p.lo);
  return fast_two_sum2(p.hi, p.lo);
}

}  // namespace ibm
