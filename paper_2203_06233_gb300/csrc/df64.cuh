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

#include <cstdint>

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

// a + b and a - b with a, b double-floats (the sloppy sum: about 2^-48 of |a| + |b|)
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return add2(a, {-b.hi, -b.lo}); }

// a + b with a a double-float and b a float
__device__ __forceinline__ F2 add(F2 a, float b) {
  const F2 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// ---- conversions on the integer pipe -------------------------------------
// On this GPU every float <-> double conversion instruction occupies the FP64
// pipe, the one the solve is bound by.  Both directions are exact or
// correctly rounded re-encodings of IEEE-754 fields, done here with integer
// operations.

// Exact float -> double: the binary32 fields re-encoded as binary64 (exponent
// rebiased by 1023 - 127, fraction moved up 29 bits; subnormals normalised;
// zeros, infinities and NaNs carried over).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint64_t bits;
  if (e == 0xFFu) {                       // infinity or NaN
    bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
  } else if (e != 0) {                    // normal
    bits = sign | ((uint64_t)(e + 896) << 52) | ((uint64_t)m << 29);
  } else if (m == 0) {                    // zero
    bits = sign;
  } else {                                // subnormal: m 2^-149, leading bit at p
    const int p = 31 - __clz(m);
    bits = sign | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)bits);
}

// -x by flipping the sign bit
__device__ __forceinline__ double dneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// Round the integer magnitude n (< 2^62) times 2^e2 to a float, to nearest with
// ties to even, assuming the result is a normal float (the caller checks the
// exponent range); sign in bit 31 of `sign`.
__device__ __forceinline__ float round_to_float(uint64_t n, int e2, uint32_t sign) {
  if (n == 0) return __uint_as_float(sign);
  const int p = 63 - __clzll((long long)n);           // leading bit
  uint64_t sig;
  int ex = p + e2;                                     // value = 1.f * 2^ex
  if (p > 23) {
    const int sh = p - 23;
    const uint64_t rem = n & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    sig = n >> sh;
    if (rem > half || (rem == half && (sig & 1))) ++sig;
    if (sig == (1ull << 24)) {                         // carried into a new binade
      sig >>= 1;
      ++ex;
    }
  } else {
    sig = n << (23 - p);
  }
  return __uint_as_float(sign | ((uint32_t)(ex + 127) << 23) | ((uint32_t)sig & 0x7FFFFFu));
}

// Split a double into hi = nearest float, lo = nearest float to the rest
// (x - hi is exact in double), with the conversion instructions: for kernels
// bound by the FP32 or integer issue rather than by the FP64 pipe.
__device__ __forceinline__ F2 from_double_cvt(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

// The same split on the integer pipe (bit-identical), for kernels bound by the
// FP64 pipe: |x| in [2^-70, 2^126), where hi and a nonzero lo are normal
// floats; the conversion instructions elsewhere (zero, tiny, huge,
// non-finite).
__device__ __forceinline__ F2 from_double(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  if (E < -70 || E >= 126) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
  }
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t S = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // x = S 2^(E-52)
  // hi: S rounded to 24 bits
  const uint64_t rem = S & ((1ull << 29) - 1);
  uint64_t H = S >> 29;
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (H & 1))) ++H;
  const float hi = round_to_float(H, E - 23, sign);      // exact: H has <= 25 bits, H 2^(E-23)
  // lo = x - hi = (S - H 2^29) 2^(E-52), |S - H 2^29| <= 2^28
  const long long d = (long long)S - (long long)(H << 29);
  const uint32_t lsign = d < 0 ? (sign ^ 0x80000000u) : sign;
  const float lo = round_to_float((uint64_t)(d < 0 ? -d : d), E - 52, lsign);
  return {hi, lo};
}

__device__ __forceinline__ double to_double(F2 a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

}  // namespace ff
}  // namespace stap
