// Double-float ("float-float") arithmetic on the FP32 pipe: a value is an
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48
// significant bits.  The building blocks are the error-free transformations
// of Knuth (TwoSum), Dekker (Fast2Sum) and the FMA-based TwoProduct; see
// Muller et al., "Handbook of Floating-Point Arithmetic", ch. 4 and 14.
//
// GB300 runs FP32 at 62x the FP64 rate, so work that needs more than FP32
// but is not itself a triangular solve (combinations and normalisations of
// FP64 solutions) is cheaper here than on the FP64 pipe.
#pragma once

namespace stap {
namespace ff {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // needs |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// acc + a * b with a, b double-floats (the a.lo * b.lo term is below the result's precision)
__device__ __forceinline__ F2 fma(F2 acc, F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const F2 s = two_sum(acc.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, e), acc.lo));
}

// acc - a * b
__device__ __forceinline__ F2 fms(F2 acc, F2 a, F2 b) { return fma(acc, {-a.hi, -a.lo}, b); }

// a + b with a a double-float and b a float
__device__ __forceinline__ F2 add(F2 a, float b) {
  const F2 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// Split a double into hi = nearest float, lo = nearest float to the rest.
__device__ __forceinline__ F2 from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double to_double(F2 a) { return (double)a.hi + (double)a.lo; }

}  // namespace ff
}  // namespace stap
