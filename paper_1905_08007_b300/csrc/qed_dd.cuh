// Double-double arithmetic for the re-evaluation of flagged points
// (Sec. 3: round-off of the numerical subtraction is controlled by
// arithmetics of different precisions).  A value is hi + lo with
// |lo| <= ulp(hi)/2; the error-free transformations are Knuth's two-sum and
// the FMA-based two-product (Dekker's algorithm with a fused multiply-add).
// Intrinsics with explicit rounding keep the compiler from contracting the
// compensation terms.
#pragma once
#include <cuda_runtime.h>

struct dd {
  double hi, lo;
  __host__ __device__ dd() : hi(0.0), lo(0.0) {}
  __host__ __device__ dd(double h, double l) : hi(h), lo(l) {}
  __host__ __device__ explicit dd(double h) : hi(h), lo(0.0) {}
};

__device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return dd(s, e);
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  return dd(s, __dsub_rn(b, __dsub_rn(s, a)));
}
__device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = __dmul_rn(a, b);
  return dd(p, __fma_rn(a, b, -p));
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = __fma_rn(a.hi, b.lo, p.lo);
  p.lo = __fma_rn(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd operator/(dd a, dd b) {
  const double q1 = __ddiv_rn(a.hi, b.hi);
  dd r = a - b * dd(q1);
  const double q2 = __ddiv_rn(r.hi, b.hi);
  r = r - b * dd(q2);
  const double q3 = __ddiv_rn(r.hi, b.hi);
  dd q = quick_two_sum(q1, q2);
  return q + dd(q3);
}

__host__ __device__ __forceinline__ double to_double(double x) { return x; }
__host__ __device__ __forceinline__ double to_double(dd x) { return x.hi + x.lo; }

// (sum, Neumaier compensation) -> normalised double-double
__device__ __forceinline__ dd dd_from_sum(double s, double c) { return two_sum(s, c); }
