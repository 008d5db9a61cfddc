// Float-float arithmetic on the FP32 pipes (device only).
//
// A real value is the unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi) / 2, which carries 48 significand bits (Dekker 1971, "A
// floating-point technique for extending the available precision"): unit
// roundoff about 2^-48 = 3.6e-15 against 2^-53 for binary64, with binary32's
// exponent range (values above 2^127 overflow; below about 2^-102 the lo part
// is subnormal and the relative precision drops towards binary32's).
//
// The two error-free transformations used:
//   - the sum a + b = s + t exactly, with s = fl(a + b) (Knuth's TwoSum, six
//     additions, no condition on the magnitudes);
//   - the product a b = p + e exactly, with p = fl(a b) and e = fma(a, b, -p).
// Products of two float-float numbers drop the lo x lo term (below 2^-48
// relatively).  Sums are kept unnormalised in an accumulator (s, e): each
// product's high part enters s through TwoSum and every rounding error and
// low-order term is added into e, which is renormalised once, when the value
// is stored.  All operations are the correctly rounded intrinsics, so the
// compiler neither contracts nor reorders them.
//
// Complex float-float values are float4 {re.hi, re.lo, im.hi, im.lo}: the same
// 16 bytes as a complex binary64 value, so buffers keep their sizes.
#pragma once

#include <cuda_runtime.h>

namespace rexi {
namespace ff {

// a + b = s + t exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// unnormalised real accumulator: value s + e
struct Acc {
  float s, e;
};

// acc += (ah + al) (bh + bl)
__device__ __forceinline__ void mac(Acc &acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);  // exact error of p
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  float s, t;
  two_sum(acc.s, p, s, t);
  acc.s = s;
  acc.e = __fadd_rn(acc.e, __fadd_rn(t, pe));
}

// acc += (xh + xl)
__device__ __forceinline__ void add(Acc &acc, float xh, float xl) {
  float s, t;
  two_sum(acc.s, xh, s, t);
  acc.s = s;
  acc.e = __fadd_rn(acc.e, __fadd_rn(t, xl));
}

// (ah + al)(bh + bl) as an unevaluated pair: the rounded product and its error terms
__device__ __forceinline__ Acc prod(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);  // exact error of p
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  return Acc{p, e};
}

// real r times complex z (both float-float), as an unnormalised pair per component
__device__ __forceinline__ float4 rscale(float2 r, float4 z) {
  const Acc a = prod(r.x, r.y, z.x, z.y), b = prod(r.x, r.y, z.z, z.w);
  return make_float4(a.s, a.e, b.s, b.e);
}

// complex accumulator
struct CAcc {
  Acc re, im;
};

__device__ __forceinline__ CAcc cacc(float4 v) { return CAcc{{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ CAcc czero() { return CAcc{{0.f, 0.f}, {0.f, 0.f}}; }

// acc += a b
__device__ __forceinline__ void cmac(CAcc &acc, float4 a, float4 b) {
  mac(acc.re, a.x, a.y, b.x, b.y);
  mac(acc.re, -a.z, -a.w, b.z, b.w);
  mac(acc.im, a.x, a.y, b.z, b.w);
  mac(acc.im, a.z, a.w, b.x, b.y);
}

// acc -= a b
__device__ __forceinline__ void cmsub(CAcc &acc, float4 a, float4 b) {
  mac(acc.re, -a.x, -a.y, b.x, b.y);
  mac(acc.re, a.z, a.w, b.z, b.w);
  mac(acc.im, -a.x, -a.y, b.z, b.w);
  mac(acc.im, -a.z, -a.w, b.x, b.y);
}

// acc += v
__device__ __forceinline__ void cadd(CAcc &acc, float4 v) {
  add(acc.re, v.x, v.y);
  add(acc.im, v.z, v.w);
}

// An accumulator as a value without renormalising: the pair (s, e) still represents s + e
// exactly, and |e| stays within a few 2^-24 of the summed magnitudes |p| that formed it.
// As a factor of mac, e enters through FP32 cross products (relative error 2^-24), so the
// error stays at the float-float level of those magnitudes; as the start of another
// accumulator or a summand of add it is exact.  Values that are stored and read back
// within a sweep skip the six-operation TwoSum this way.
__device__ __forceinline__ float4 raw(const CAcc &a) { return make_float4(a.re.s, a.re.e, a.im.s, a.im.e); }

// complex a b, unnormalised
__device__ __forceinline__ float4 cmul(float4 a, float4 b) {
  CAcc r{prod(a.x, a.y, b.x, b.y), prod(a.x, a.y, b.z, b.w)};
  mac(r.re, -a.z, -a.w, b.z, b.w);
  mac(r.im, a.z, a.w, b.x, b.y);
  return raw(r);
}

__device__ __forceinline__ float4 cconj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }

// normalised value of an accumulator (TwoSum: no condition on |s| against |e|)
__device__ __forceinline__ float4 norm(const CAcc &a) {
  float4 r;
  two_sum(a.re.s, a.re.e, r.x, r.y);
  two_sum(a.im.s, a.im.e, r.z, r.w);
  return r;
}

// binary64 -> float-float: hi = fl32(x), lo = fl32(x - hi); x - hi is exact in binary64
__device__ __forceinline__ float2 split(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return make_float2(hi, lo);
}
__device__ __forceinline__ float4 csplit(double2 z) {
  const float2 r = split(z.x), i = split(z.y);
  return make_float4(r.x, r.y, i.x, i.y);
}

// true when a finite binary64 component of z became infinite in the split (|x| above
// binary32's largest finite value)
__device__ __forceinline__ bool split_overflow(double2 z, float4 v) {
  return (isinf(v.x) && isfinite(z.x)) || (isinf(v.z) && isfinite(z.y));
}

// float-float -> binary64 (hi + lo rounded once)
__device__ __forceinline__ double join(float hi, float lo) { return (double)hi + (double)lo; }
__device__ __forceinline__ double2 cjoin(float4 v) { return make_double2(join(v.x, v.y), join(v.z, v.w)); }

}  // namespace ff
}  // namespace rexi
