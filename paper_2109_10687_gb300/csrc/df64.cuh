// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two float32 numbers, |lo| <= ulp(hi)/2, about 48 significant bits.  The
// float64 residual of the defect-correction loop (Algorithm 4) runs in this
// format on the float32 pipes, which on this GPU are far wider than the
// float64 ones.
//
// Building blocks (error-free transformations, Dekker/Knuth, with fused
// multiply-add for the exact product error):
//   two_sum(a, b)       = (s, e) with s = fl(a + b), s + e = a + b exactly
//   quick_two_sum(a, b) = the same when |a| >= |b|
//   two_prod(a, b)      = (p, e) with p = fl(a b), e = fma(a, b, -p)
// Addition and multiplication renormalise once ("sloppy" variants): relative
// error a few units of 2^-48.
#pragma once

#include <cuda_runtime.h>

namespace qcd {

struct df64 {
  float hi, lo;
  __host__ __device__ df64() : hi(0.f), lo(0.f) {}
  __host__ __device__ df64(float h) : hi(h), lo(0.f) {}
  __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df64(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
};

// fused multiply-add for every real type the kernels use, visible to
// unqualified calls inside namespace qcd
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

__device__ __forceinline__ double to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
// a * b + c with one final renormalisation
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  df64 s = two_sum(p, c.hi);
  s.lo += e + c.lo;
  return quick_two_sum(s.hi, s.lo);
}

// The exponent k of the power of two 2^k that brings a field with |b|^2 =
// b2 over n2 complex components to components of order one: the
// double-float paths hold b, x and r scaled by it, since a double-float
// number has the exponent range of float32 (k = 0 for a zero field).
__device__ __forceinline__ int df_scale_exp(double b2, size_t n2) {
  int e = 0;
  const double m = b2 / (double)n2;
  if (m > 0.0) frexp(m, &e);
  return max(-120, min(120, -e / 2));
}

// Conversions between float64 and double-float with a power-of-two scale
// 2^k folded in, by integer operations on the IEEE-754 bit fields (sign,
// biased exponent, significand) instead of float64 arithmetic: the
// float64 pipe of this GPU is a small fraction of its integer and float32
// width.  For a value whose scaled magnitude lies in float32's normal
// range the result equals the float64 computation exactly: hi is d 2^k
// rounded to nearest-even float32, lo is d 2^k - hi rounded to float32.
// Zero and float64 subnormals give zero; scaled values below the normal
// range give zero, above it infinity (with d's sign).
__device__ __forceinline__ df64 df64_from_double_scaled(double d, int k) {
  const unsigned long long D = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(D >> 32) & 0x80000000u;
  const int e = (int)((D >> 52) & 0x7FF);
  const int E = e - 1023 + 127 + k;  // biased float32 exponent of hi
  if (e == 0 || E <= 0) return df64(__uint_as_float(sign), 0.f);
  if (E >= 255) return df64(__uint_as_float(sign | 0x7F800000u), 0.f);
  const unsigned long long m = D & 0xFFFFFFFFFFFFFull;  // 52 significand bits
  const unsigned top = (unsigned)(m >> 29);              // the 23 that hi keeps
  const unsigned rest = (unsigned)(m & 0x1FFFFFFFu);     // the 29 it drops
  const bool up = rest > (1u << 28) || (rest == (1u << 28) && (top & 1u));
  // a carry out of the significand moves into the exponent, as rounding requires
  const float hi = __uint_as_float(sign | (((unsigned)E << 23) + top + (up ? 1u : 0u)));
  // lo = (rest - 2^29 [if rounded up]) 2^(E - 127 - 52), with d's sign
  const int r = (int)rest - (up ? (1 << 29) : 0);
  float lo = 0.f;
  if (E > 52) lo = (float)r * __uint_as_float((unsigned)(E - 52) << 23);
  return df64(hi, sign ? -lo : lo);
}

// the exact float64 value of a float32 (zero and float32 subnormals give
// zero, below 1.2e-38 of the order-one scaled values; infinities and NaNs
// keep their class)
__device__ __forceinline__ double exact_double(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned E = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if (E == 0) return __longlong_as_double((long long)s);
  const unsigned long long Ed = E == 0xFFu ? 0x7FFull : (unsigned long long)(E - 127 + 1023);
  return __longlong_as_double((long long)(s | (Ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// (hi + lo) 2^-k as float64: the exact float64 values of hi and lo summed
// by one float64 addition (the rounding of the plain float64 sum), then the
// scale on the exponent field (zero stays zero; a result outside the
// float64 normal range becomes zero or infinity)
__device__ __forceinline__ double df64_to_double_scaled(df64 a, int k) {
  const double v = exact_double(a.hi) + exact_double(a.lo);
  const unsigned long long V = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((V >> 52) & 0x7FF);
  if (e == 0 || e == 0x7FF) return v;
  const int e2 = e - k;
  const unsigned long long s = V & 0x8000000000000000ull;
  if (e2 <= 0) return __longlong_as_double((long long)s);
  if (e2 >= 0x7FF) return __longlong_as_double((long long)(s | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)((V & ~0x7FF0000000000000ull) | ((unsigned long long)e2 << 52)));
}

}  // namespace qcd
