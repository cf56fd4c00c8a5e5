// FP64 <-> FP32 conversions, FP64 comparisons and tests written with integer instructions on the
// numbers' bit patterns.
//
// On GB300 one FP64 warp instruction occupies a scheduler's FP64 unit for about as long as 64 FP32
// instructions, and conversions between FP32 and FP64 and FP64 comparisons run on that unit too.
// The FP32-stage precision mode keeps only the FP64 arithmetic the precision split asks for (the
// error-norm accumulation, the compensated time, the step size) on the FP64 pipe; the conversions
// and tests around it go through these helpers. The same helpers serve trajectory start-up, where a
// lane of a persistent warp starts alone and every FP64-pipe instruction costs the whole warp's
// share of the pipe.
//
// Each helper gives exactly the result of the operation it replaces for every input (conversions
// as this library is built, with FP32 flush-to-zero: -ftz=true); gs_selftest() checks them on the
// device against the hardware instructions.
//
// Sign masks work on the 32-bit high word: the compiler recognises a 64-bit "bits & 0x7fff...ffff"
// of a double as fabs and issues it as an FP64 add with an absolute-value operand (measured: two
// such masks per accepted step were two FP64 instructions per step).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

// An FP32 number widened to FP64 exactly (sign; exponent rebiased by 1023 - 127; mantissa shifted
// up by 29). Zero and, with flush-to-zero, a subnormal give a signed zero; infinities and NaNs keep
// their class.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sgn = u & 0x80000000u, ex = (u >> 23) & 0xffu, man = u & 0x7fffffu;
  uint32_t hi = sgn | ((ex + 896u) << 20) | (man >> 3), lo = man << 29;
  if (ex == 0u) { hi = sgn; lo = 0u; }
  if (ex == 0xffu) hi = sgn | 0x7ff00000u | (man >> 3) | (man ? 0x80000u : 0u);
  return __hiloint2double(int(hi), int(lo));
}

// An FP64 number rounded to FP32, to nearest with ties to even (IEEE 754 roundTiesToEven). The
// 24-bit significand is the hidden bit and the top 23 mantissa bits; the 29 bits below decide the
// rounding; a carry out of the significand raises the exponent (and past the largest finite FP32
// gives infinity). A result below the normal range flushes to a signed zero, as the conversion
// instruction does with flush-to-zero; the one exception is the band just below the smallest normal
// number 2^-126 whose rounding reaches it. |x| >= 2^128 gives infinity; NaN stays NaN.
__device__ __forceinline__ float narrow_f64(double x) {
  const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x));
  const uint32_t sgn = hi & 0x80000000u;
  const int ex = int((hi >> 20) & 0x7ffu);
  const uint32_t q = 0x800000u | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t r = lo & 0x1fffffffu;
  const uint32_t up = (r > 0x10000000u || (r == 0x10000000u && (q & 1u))) ? 1u : 0u;
  uint32_t bits = (uint32_t(ex - 897) << 23) + q + up;  // FP32 biased exponent ex - 896 >= 1
  // ex = 896: x in [2^-127, 2^-126); on the subnormal grid (unit 2^-149) it rounds up to 2^-126
  // exactly when its top 24 significand bits are all ones (any remainder then reaches the half)
  if (ex == 896) bits = (q == 0xffffffu) ? 0x800000u : 0u;
  if (ex < 896) bits = 0u;
  if (ex >= 1151) bits = 0x7f800000u;
  if (ex == 0x7ff) bits = 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u);
  return __uint_as_float(sgn | bits);
}

// x in the stage precision R: FP32 through narrow_f64; FP64 and double-FP32 as constructed
template <class R> __device__ __forceinline__ R to_r(double x) { return R(x); }
template <> __device__ __forceinline__ float to_r<float>(double x) { return narrow_f64(x); }

// Order, NaN test and log2 of a non-negative FP64 number (a sum of squares) from its bits with
// integer and FP32 instructions: for x, y >= 0 the bit patterns order as the values do, and every
// NaN pattern lies above that of +inf.
__device__ __forceinline__ bool le_nonneg_f64(double x, double y) { return __double_as_longlong(x) <= __double_as_longlong(y); }
__device__ __forceinline__ bool isnan_f64_bits(double x) {
  const uint32_t hi = uint32_t(__double2hiint(x)) & 0x7fffffffu;
  return hi > 0x7ff00000u || (hi == 0x7ff00000u && __double2loint(x) != 0);
}
__device__ __forceinline__ bool isfinite_f64_bits(double x) {
  return (uint32_t(__double2hiint(x)) & 0x7ff00000u) != 0x7ff00000u;
}
// log2 x to FP32 accuracy: the unbiased exponent plus log2 of the mantissa truncated to 24 bits
__device__ __forceinline__ float log2_f64_f32(double x) {
  const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x));
  const int ex = int((hi >> 20) & 0x7ffu) - 1023;
  const float m = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));
  return float(ex) + __log2f(m);
}

// A signed 64-bit key that orders non-NaN FP64 numbers as their values (-0 and +0 get the same key):
// non-negative numbers keep their bit pattern, negative ones get minus their magnitude's pattern.
__device__ __forceinline__ long long key_f64(double x) {
  const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x));
  const long long mag = (long long)(((unsigned long long)(hi & 0x7fffffffu) << 32) | lo);
  return (hi & 0x80000000u) ? -mag : mag;
}
// x <= y and x == y as the FP64 comparisons give them; both false when either is NaN
__device__ __forceinline__ bool le_f64_bits(double x, double y) {
  return !isnan_f64_bits(x) && !isnan_f64_bits(y) && key_f64(x) <= key_f64(y);
}
__device__ __forceinline__ bool eq_f64_bits(double x, double y) {
  return !isnan_f64_bits(x) && key_f64(x) == key_f64(y);
}
// -x and |x| by the sign bit of the high word
__device__ __forceinline__ double neg_f64_bits(double x) {
  return __hiloint2double(int(uint32_t(__double2hiint(x)) ^ 0x80000000u), __double2loint(x));
}
__device__ __forceinline__ double abs_f64_bits(double x) {
  return __hiloint2double(int(uint32_t(__double2hiint(x)) & 0x7fffffffu), __double2loint(x));
}
__device__ __forceinline__ bool signbit_f64_bits(double x) { return __double2hiint(x) < 0; }
// max(|a|, |b|) * 2^-48 (16 eps max(|a|, |b|) in FP64) of finite a, b, flushed to zero below the
// normal range: the larger magnitude by its (high, low) words, then 48 off its exponent field
__device__ __forceinline__ double max_abs_2m48_bits(double a, double b) {
  const uint32_t ha = uint32_t(__double2hiint(a)) & 0x7fffffffu, la = uint32_t(__double2loint(a));
  const uint32_t hb = uint32_t(__double2hiint(b)) & 0x7fffffffu, lb = uint32_t(__double2loint(b));
  const bool a_big = ha > hb || (ha == hb && la >= lb);
  const uint32_t hm = a_big ? ha : hb, lm = a_big ? la : lb;
  const uint32_t e48 = 48u << 20;
  const bool keep = hm > e48 || (hm == e48 && lm != 0u);
  return keep ? __hiloint2double(int(hm - e48), int(lm)) : 0.0;
}

}  // namespace gs
