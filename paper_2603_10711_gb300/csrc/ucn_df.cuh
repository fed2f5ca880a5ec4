// Double-float ("DF") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// Why.  GB300 runs FP64 at 1/64 of its FP32 rate, so the FP32 path's
// per-SCP-iteration work that needs more than float precision (the RK4
// rollout of the candidate, defects, merits, the nominal trajectory itself)
// costs more issue slots in FP64 than all of an SCP iteration's ADMM work.
// The same arithmetic on float pairs runs on the FP32 pipes at a few FP32
// instructions per operation.
//
// Methods (written from the published algorithms):
//  - two_sum: Knuth's error-free sum (TAOCP Vol. 2, Sec. 4.2.2, Theorem B);
//  - quick_two_sum: Dekker's Fast2Sum (Dekker 1971), valid for |a| >= |b|;
//  - two_prod: the error-free product from one fused multiply-add;
//  - add / mul: Dekker's double-length operations built on those;
//  - div / sqrt: one correction of the float quotient or root by the exact
//    residual (the Karp-Markstein form of a Newton step, 1997).
// Every float operation below is an explicit round-to-nearest intrinsic, so
// the compiler neither contracts nor reorders them.
#pragma once
#include <cuda_runtime.h>

namespace ucn {

struct __align__(8) DF {
  float hi, lo;
  __device__ __forceinline__ DF() : hi(0.0f), lo(0.0f) {}
  __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  // exact for the small constants the models use (folded at compile time)
  __device__ __forceinline__ explicit DF(int a) : hi((float)a), lo(0.0f) {}
  __device__ __forceinline__ explicit DF(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ DF df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// conversions
__device__ __forceinline__ DF df_from(float a) { return {a, 0.0f}; }
__device__ __forceinline__ DF df_from(double a) {
  const float h = __double2float_rn(a);
  return {h, __double2float_rn(a - (double)h)};
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float df_to_float(DF a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  const DF t = df_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
// DF + float
__device__ __forceinline__ DF df_add(DF a, float b) {
  DF s = df_two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF p = df_two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return df_quick_two_sum(p.hi, p.lo);
}
// DF * float
__device__ __forceinline__ DF df_mul(DF a, float b) {
  DF p = df_two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return df_quick_two_sum(p.hi, p.lo);
}
// a + b c: the product exact in its high parts plus the cross terms, then one
// sum of the pair (Dekker's add without the separate low-part sum); the error
// is a few units of 2^-48 relative to |a| + |b c| -- what an RK4 update
// x + h k needs -- at about half the instructions of a product and a sum.
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) {
  DF p = df_two_prod(b.hi, c.hi);
  p.lo = __fmaf_rn(b.hi, c.lo, __fmaf_rn(b.lo, c.hi, p.lo));
  DF s = df_two_sum(a.hi, p.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, p.lo));
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF r = df_sub(a, df_mul(b, q1));   // exact-enough residual a - q1 b
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return df_quick_two_sum(q1, q2);
}
__device__ __forceinline__ DF df_sqrt(DF a) {
  if (!(a.hi > 0.0f)) return {a.hi == 0.0f ? 0.0f : __fsqrt_rn(a.hi), 0.0f};   // 0, or NaN below 0
  const float s = __fsqrt_rn(a.hi);
  const DF r = df_sub(a, df_two_prod(s, s));   // a - s^2, s^2 exactly
  return df_quick_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.0f, s)));
}

__device__ __forceinline__ DF operator+(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return df_sub(a, b); }
__device__ __forceinline__ DF operator-(DF a) { return df_neg(a); }
__device__ __forceinline__ DF operator*(DF a, DF b) { return df_mul(a, b); }
__device__ __forceinline__ DF operator/(DF a, DF b) { return df_div(a, b); }

// Residual norms of Step 4 (Sec. III-B) are accumulated in the wide type of
// the path: FP64 on the plain path; double-float on the FP32 path, where each
// term is the square of the EXACT difference of two FP32 iterates (Knuth's
// error-free sum) and every sum is a double-float sum of non-negative terms
// (relative error below 2^-44 each), so a CTA total of t terms per node over a
// tree of <= 256 nodes is within (t + 8) 2^-44 < 1e-11 of the exact sum of the
// iterates' squared differences -- FP64-grade, without the FP64 pipe (1/64 of
// the FP32 rate on this GPU).
__device__ __forceinline__ void acc_sq_diff(double& acc, double a, double b) {
  const double d = a - b;
  acc += d * d;
}
__device__ __forceinline__ void acc_sq_diff(DF& acc, float a, float b) {
  const DF d = df_two_sum(a, -b);
  acc = df_add(acc, df_mul(d, d));
}
__device__ __forceinline__ void acc_sq(double& acc, double v) { acc += v * v; }
__device__ __forceinline__ void acc_sq(DF& acc, float v) { acc = df_add(acc, df_two_prod(v, v)); }

// The wide type of a compute precision: FP64 for the FP64 path; double-float
// for the FP32 path (no FP64 instruction in its per-iteration work).
template <class T> struct WideOf { typedef double type; };
template <> struct WideOf<float> { typedef DF type; };

// Conversions between a wide value and double / the compute type.
__device__ __forceinline__ double wide_to_double(double a) { return a; }
__device__ __forceinline__ double wide_to_double(DF a) { return df_to_double(a); }
template <class W> __device__ __forceinline__ W wide_from_double(double a);
template <> __device__ __forceinline__ double wide_from_double<double>(double a) { return a; }
template <> __device__ __forceinline__ DF wide_from_double<DF>(double a) { return df_from(a); }
template <class T> __device__ __forceinline__ T wide_to(double a) { return (T)a; }
template <class T> __device__ __forceinline__ T wide_to(DF a) { return (T)df_to_float(a); }
// wide + compute-type value, wide - wide rounded to the compute type
__device__ __forceinline__ double wide_add(double a, double b) { return a + b; }
__device__ __forceinline__ double wide_add(double a, float b) { return a + (double)b; }
__device__ __forceinline__ DF wide_add(DF a, float b) { return df_add(a, b); }
template <class T> __device__ __forceinline__ T wide_diff(double a, double b) { return (T)(a - b); }
template <class T> __device__ __forceinline__ T wide_diff(DF a, DF b) { return (T)df_to_float(df_sub(a, b)); }

}  // namespace ucn
