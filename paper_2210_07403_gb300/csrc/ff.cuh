// Float-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| ≤ ulp(hi)/2, about 48 significand bits. It gives the 2-D operator an application accurate
// to about 1e-13 at FP32-pipe speed, for the refinement residual of mixed-precision solves (the
// FP64 pipe of this GPU runs at about 1/58 of the FP32 rate).
//
// The operations are built from error-free transformations: TwoSum (Knuth, TAOCP vol. 2,
// §4.2.2: s + e = a + b exactly), FastTwoSum (Dekker 1971, for |a| ≥ |b|) and TwoProd with a fused
// multiply-add (p + e = a·b exactly). Addition adds the low parts into the TwoSum error before
// renormalising: its error is bounded by a few units of 2^−48 times |a| + |b| (a normwise bound,
// which is what an FFT's accuracy rests on). Products add the cross terms a.hi·b.lo + a.lo·b.hi
// into the TwoProd error. Division refines an FP32 quotient by one float-float correction step.
// None of these may be rewritten by the compiler: only explicit fmaf calls fuse, and the
// sums are kept in their written order (no fast-math flags are used).
#pragma once

#include <cuda_runtime.h>

namespace ibdl {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest float-float to a double: hi = fl32(d), lo = fl32(d − hi) (d − hi is exact in FP64)
  __host__ __device__ constexpr explicit ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr explicit ff(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff(s, e);
}
// s + e = a + b exactly, given |a| ≥ |b| (or a = 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff(s, b - (s - a));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);  // p + e = a.hi·b.hi exactly
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
// a / b: q1 = fl32(a.hi / b.hi), then q2 = (a − q1·b)/b.hi with the remainder in float-float
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  const ff r = a - ff(q1, 0.0f) * b;
  const float q2 = r.hi / b.hi;
  return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }

// The float-float value of a double by integer arithmetic on its bits, so the conversion does not
// use the FP64 pipe. With d = ±M·2^(e−1075) (e the biased exponent, M the 53-bit significand):
// Mh = ⌊(M + 2^28)/2^29⌋ ≤ 2^24 (the leading 24 bits, rounded; converts to FP32 exactly) gives
// hi = ±Mh·2^(e−1046), and r = M − 2^29·Mh (|r| ≤ 2^28) gives lo = ±fl32(r)·2^(e−1075), so
// |d − hi − lo| ≤ 2^−24·|lo| ≤ 2^−48·|d|. Both scales are normal floats and hi does not overflow
// for 949 ≤ e ≤ 1149 (2^−74 ≤ |d| < 2^127). Zero (most nodes of a spread grid) and subnormal
// doubles (below 2^−1022) give (0, 0); the remaining values outside that range are converted
// through FP64.
__device__ __forceinline__ ff ff_from_double(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return ff(0.0f, 0.0f);
  if (e < 949 || e > 1149) return ff(d);
  const long long M = (b & 0xfffffffffffffLL) | (1LL << 52);
  const long long Mh = (M + (1LL << 28)) >> 29;
  const int r = (int)(M - (Mh << 29));
  const float s_hi = __int_as_float((e - 1046 + 127) << 23);  // 2^(e − 1046)
  const float s_lo = __int_as_float((e - 1075 + 127) << 23);  // 2^(e − 1075)
  const float hi = __int2float_rn((int)Mh) * s_hi;
  const float lo = __int2float_rn(r) * s_lo;
  return b < 0 ? ff(-hi, -lo) : ff(hi, lo);
}
__device__ __forceinline__ bool operator==(ff a, ff b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(ff a, ff b) { return !(a == b); }
// comparisons of normalised values: the high parts decide unless they are equal
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

}  // namespace ibdl
