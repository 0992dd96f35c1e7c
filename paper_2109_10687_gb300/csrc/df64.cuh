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

}  // namespace qcd
