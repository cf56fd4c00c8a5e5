// Double-FP32 ("df64") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits (unit roundoff ~2^-47). The operations are built from
// the classical error-free transformations: Knuth's TwoSum, the fast TwoSum for ordered operands,
// and the product error through a fused multiply-add (Dekker's TwoProduct with an FMA); division,
// reciprocal and square roots refine an FP32 first approximation by one Newton step carried out in
// df64. On GB300 an FP64 instruction occupies the FP64 pipe for 64 FP32 issue slots, so a df64
// add (about 20 FP32 instructions) or multiply (about 6) is several times cheaper than its FP64
// counterpart while still resolving tolerances far below FP32's.
#pragma once
#include <cuda_runtime.h>

namespace gs {

struct F2 {
  float hi, lo;
  F2() = default;
  // exact split of an FP64 value into the nearest FP32 and the FP32 rounding of the remainder
  __host__ __device__ constexpr F2(double x) : hi(float(x)), lo(float(x - double(float(x)))) {}
  __host__ __device__ constexpr F2(float x) : hi(x), lo(0.0f) {}
  __host__ __device__ constexpr F2(int x) : hi(float(x)), lo(0.0f) {}
  __host__ __device__ static constexpr F2 pair(float h, float l) {
    F2 r(0.0f);
    r.hi = h;
    r.lo = l;
    return r;
  }
};

// s + e = a + b exactly, for |a| >= |b|
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return F2::pair(s, b - (s - a));
}
// s + e = a + b exactly
__device__ __forceinline__ F2 two_sum_f(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return F2::pair(s, (a - (s - bb)) + (b - bb));
}
// p + e = a * b exactly
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = a * b;
  return F2::pair(p, fmaf(a, b, -p));
}

__device__ __forceinline__ F2 operator-(const F2& a) { return F2::pair(-a.hi, -a.lo); }
__device__ __forceinline__ F2 operator+(const F2& a, const F2& b) {
  // both parts summed error-free, then renormalised twice (accurate also under cancellation)
  const F2 s = two_sum_f(a.hi, b.hi);
  const F2 t = two_sum_f(a.lo, b.lo);
  const F2 u = fast_two_sum(s.hi, s.lo + t.hi);
  return fast_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ F2 operator-(const F2& a, const F2& b) { return a + (-b); }
__device__ __forceinline__ F2 operator*(const F2& a, const F2& b) {
  const F2 p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ F2 mul_f(const F2& a, float b) {
  const F2 p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
// q1 = a/b in FP32, then one correction with the df64 residual a - q1 b
__device__ __forceinline__ F2 operator/(const F2& a, const F2& b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = a.hi * rb;
  const F2 r = a - mul_f(b, q1);
  const float q2 = r.hi * rb;
  const F2 r2 = r - mul_f(b, q2);
  return fast_two_sum(q1, q2 + r2.hi * rb);
}
__device__ __forceinline__ F2& operator+=(F2& a, const F2& b) { a = a + b; return a; }
__device__ __forceinline__ F2& operator-=(F2& a, const F2& b) { a = a - b; return a; }
__device__ __forceinline__ F2& operator*=(F2& a, const F2& b) { a = a * b; return a; }

// elementary functions used by the right-hand sides
__device__ __forceinline__ F2 grcp(const F2& a) { return F2(1.0f) / a; }
__device__ __forceinline__ F2 gdiv(const F2& a, const F2& b) { return a / b; }
__device__ __forceinline__ F2 gsqrt(const F2& a) {
  const float s = sqrtf(a.hi);
  if (!(a.hi > 0.0f)) return F2::pair(s, 0.0f);
  const F2 p = two_prod(s, s);
  const float r = ((a.hi - p.hi) - p.lo) + a.lo;  // a - s^2, the leading terms cancel exactly
  return fast_two_sum(s, r / (2.0f * s));
}
__device__ __forceinline__ F2 grsqrt(const F2& a) {
  const float y = rsqrtf(a.hi);
  const F2 e = F2(1.0f) - a * two_prod(y, y);  // 1 - a y^2
  return fast_two_sum(y, 0.5f * y * e.hi);
}

__device__ __forceinline__ float val(const F2& x) { return x.hi; }
__device__ __forceinline__ double to_f64(const F2& x) { return double(x.hi) + double(x.lo); }
__device__ __forceinline__ double to_f64(float x) { return double(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

}  // namespace gs
