// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits.  On GB300 an FP32 operation issues at 64x
// the FP64 rate, so a float-float add (~10 FP32 operations) or multiply (~7) is several
// times cheaper than the FP64 one it replaces.
//
// The operations are built from the classical error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = a + b, e = (a - (s - bb)) + (b - bb) with
//     bb = s - a, gives a + b = s + e exactly;
//   FastTwoSum (Dekker 1971): for |a| >= |b|, s = a + b, e = b - (s - a);
//   TwoProduct with a fused multiply-add: p = a b, e = fma(a, b, -p), a b = p + e exactly.
// Addition adds the low parts to the TwoSum error before renormalising (the "sloppy" sum):
// its error is bounded by a few units of 2^-48 times |a| + |b|, which is the absolute
// accuracy an FFT needs.  Nothing here may be reassociated: the file is compiled without
// fast-math options, and every FMA is written out.
#pragma once
#include <cuda_runtime.h>

namespace pcf {

using ::fma;  // keep the FP64/FP32 overloads visible next to the float-float one below

struct ff {
  float hi, lo;
  ff() = default;
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
  // nearest float-float of a double: hi = fl(d), lo = fl(d - hi) (d - hi is exact in FP64)
  __device__ __forceinline__ ff(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
};

__device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(double a) { return a; }

__device__ __forceinline__ ff ff_renorm(float s, float e) {
  const float hi = __fadd_rn(s, e);
  return ff(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_renorm(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_renorm(p, e);
}

// a b + c: the product's exact high part and error enter one TwoSum with c
__device__ __forceinline__ ff fma(ff a, ff b, ff c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const float s = __fadd_rn(p, c.hi);
  const float bb = __fsub_rn(s, p);
  float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  return ff_renorm(s, e);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }

struct ff2 {
  ff x, y;
};

}  // namespace pcf
