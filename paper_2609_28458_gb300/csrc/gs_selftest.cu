// gs_selftest: the bit-level FP64 helpers of gs_bits.cuh checked on the device against the
// instructions they replace (conversions, comparisons, sign operations), built with this library's
// own compiler flags. The kernels use the helpers wherever the FP64 pipe is not needed, on the
// premise that each gives exactly the instruction's result; this test is that premise's evidence.
//
// Inputs come from SplitMix64 (Steele, Lea & Flood 2014: x += 0x9e3779b97f4a7c15, then two
// xor-shift-multiply rounds) on the counter seed + i, shaped into: raw 64-bit patterns (every
// exponent, subnormals, infinities, NaNs); FP64 numbers in and around the FP32 range; exact
// rounding ties of the FP64 -> FP32 conversion and their neighbours; and a fixed list of edge cases.
#include <cstdint>
#include <cuda_runtime.h>

#include "gs.h"
#include "gs_bits.cuh"

namespace gs {
int set_error(int code, const char* msg);  // defined in gs_api.cu
}

namespace {
using gs::narrow_f64;
using gs::widen_f32;

__device__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

__device__ const uint64_t kEdge[] = {
    0x0000000000000000ULL, 0x8000000000000000ULL,  // +-0
    0x7ff0000000000000ULL, 0xfff0000000000000ULL,  // +-inf
    0x7ff8000000000000ULL, 0x7ff0000000000001ULL,  // quiet, signalling NaN
    0xfff8000000000001ULL, 0x0000000000000001ULL,  // negative NaN, smallest FP64 subnormal
    0x000fffffffffffffULL, 0x0010000000000000ULL,  // largest FP64 subnormal, smallest normal
    0x7fefffffffffffffULL, 0x3ff0000000000000ULL,  // largest FP64, 1
    0x47efffffe0000000ULL, 0x47efffffefffffffULL,  // FP32 max, just below its rounding to inf
    0x47effffff0000000ULL, 0x47f0000000000000ULL,  // rounds to inf (tie to even), 2^128
    0x3810000000000000ULL, 0x380fffffffffffffULL,  // 2^-126, just below it
    0x380ffffff0000000ULL, 0x380fffffdfffffffULL,  // rounds up to 2^-126; rounds below it (flushed)
    0x3800000000000000ULL, 0x36a0000000000000ULL,  // 2^-127, 2^-149
    0x3690000000000000ULL, 0x3ff0000010000000ULL,  // 2^-150, 1 + half an FP32 ulp (tie, even: 1)
    0x3ff0000030000000ULL, 0xbff0000010000001ULL,  // tie up to the even neighbour, -(just above a tie)
};
constexpr int kNumEdge = sizeof(kEdge) / sizeof(kEdge[0]);

__device__ uint64_t draw_f64(uint64_t r, uint64_t r2) {
  const int mode = int(r >> 61);
  const uint64_t sgn = r2 & 0x8000000000000000ULL;
  const uint64_t man = r & 0xfffffffffffffULL;
  switch (mode) {
    case 0: case 1: return r;  // any pattern
    case 2: case 3: {          // exponents 860 .. 1159: around the FP32 range, both boundaries
      const uint64_t ex = 860 + (r2 >> 8) % 300;
      return sgn | (ex << 52) | man;
    }
    case 4: {  // exact ties of the rounding to FP32 (the 29 dropped bits 1000...0)
      const uint64_t ex = 890 + (r2 >> 8) % 265;
      return sgn | (ex << 52) | (man & ~0x1fffffffULL) | 0x10000000ULL;
    }
    case 5: {  // one unit above or below a tie
      const uint64_t ex = 890 + (r2 >> 8) % 265;
      const uint64_t t = (man & ~0x1fffffffULL) | 0x10000000ULL;
      return sgn | (ex << 52) | ((r2 & 1) ? t + 1 : t - 1);
    }
    case 6: return kEdge[(r2 >> 8) % kNumEdge];
    default: {  // ordinary magnitudes
      const uint64_t ex = 1000 + (r2 >> 8) % 48;
      return sgn | (ex << 52) | man;
    }
  }
}

__device__ bool nan32(float f) { return (__float_as_uint(f) & 0x7fffffffu) > 0x7f800000u; }
__device__ bool nan64(double d) { return (__double_as_longlong(d) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL; }

__device__ void bad(unsigned long long* counts, int check, uint64_t input) {
  atomicAdd(counts + check, 1ULL);
  atomicExch(counts + GS_SELFTEST_CHECKS + check, (unsigned long long)input);
}

__global__ void k_selftest(long long n, unsigned long long seed, unsigned long long* counts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint64_t c = seed + 4ULL * uint64_t(i);
    const uint64_t r1 = splitmix64(c), r2 = splitmix64(c + 1ULL), r3 = splitmix64(c + 2ULL), r4 = splitmix64(c + 3ULL);
    const uint64_t xb = draw_f64(r1, r2);
    const double x = __longlong_as_double((long long)xb);
    // y: x itself, -x, a neighbour of x, or an independent draw
    uint64_t yb;
    switch (int(r3 >> 62)) {
      case 0: yb = xb; break;
      case 1: yb = xb ^ 0x8000000000000000ULL; break;
      case 2: yb = xb + ((r3 & 1) ? 1ULL : ~0ULL); break;
      default: yb = draw_f64(r3, r4); break;
    }
    const double y = __longlong_as_double((long long)yb);
    // 0: FP64 -> FP32 rounding
    const float nf = narrow_f64(x), cf = float(x);
    if (!(nan32(nf) && nan32(cf)) && __float_as_uint(nf) != __float_as_uint(cf)) bad(counts, 0, xb);
    // 1: FP32 -> FP64 widening (every FP32 pattern: the low word of r4)
    const float f = __uint_as_float(uint32_t(r4));
    const double wd = widen_f32(f), cd = double(f);
    if (!(nan64(wd) && nan64(cd)) && __double_as_longlong(wd) != __double_as_longlong(cd)) bad(counts, 1, uint32_t(r4));
    // 2, 3: x <= y and x == y
    if (gs::le_f64_bits(x, y) != (x <= y)) bad(counts, 2, xb);
    if (gs::eq_f64_bits(x, y) != (x == y)) bad(counts, 3, xb);
    // 4: NaN and finiteness tests
    if (gs::isnan_f64_bits(x) != bool(isnan(x)) || gs::isfinite_f64_bits(x) != bool(isfinite(x))) bad(counts, 4, xb);
    // 5: sign operations, bit for bit on numbers (the instructions may return another NaN for a
    // NaN; the helpers, like them, return a NaN)
    const double ng = gs::neg_f64_bits(x), ab = gs::abs_f64_bits(x);
    const bool sign_ok = nan64(x) ? (nan64(ng) && nan64(ab))
                                  : (__double_as_longlong(ng) == __double_as_longlong(-x) &&
                                     __double_as_longlong(ab) == __double_as_longlong(fabs(x)));
    if (!sign_ok || gs::signbit_f64_bits(x) != bool(signbit(x))) bad(counts, 5, xb);
    // 6: order of non-negative numbers (the norm's accept test): x, y >= 0, not NaN
    const double ax = fabs(x), ay = fabs(y);
    if (!nan64(ax) && !nan64(ay) && gs::le_nonneg_f64(ax, ay) != (ax <= ay)) bad(counts, 6, xb);
    // 8: 16 eps max(|x|, |y|) (the step-size floor) of finite x, y, where that product is normal
    if (isfinite(x) && isfinite(y)) {
      const double mx = fabs(x) > fabs(y) ? fabs(x) : fabs(y);
      const double ref = 16.0 * 2.220446049250313e-16 * mx;
      if (ref >= 2.2250738585072014e-308 &&
          __double_as_longlong(gs::max_abs_2m48_bits(x, y)) != __double_as_longlong(ref))
        bad(counts, 8, xb);
    }
    // 7: log2 of a positive normal number to FP32 accuracy: the mantissa truncated to 24 bits
    // (2^-24 relative: 8.6e-8 in log2), the fast FP32 log2 on [1, 2) and the rounding of the FP32
    // sum (half an ulp of |log2 x| < 1024): within 2^-20 + 2^-23 |log2 x|
    if (ax >= 2.2250738585072014e-308 && ax <= 1.7976931348623157e308) {
      const double ref = log2(ax), got = double(gs::log2_f64_f32(ax));
      if (!(fabs(got - ref) <= 9.5367431640625e-7 + 1.1920928955078125e-7 * fabs(ref))) bad(counts, 7, xb);
    }
  }
}
}  // namespace

extern "C" int gs_selftest(int64_t n, uint64_t seed, unsigned long long* counts, void* cuda_stream) {
  if (n < 1 || !counts) return gs::set_error(GS_ERR_INVALID, "gs_selftest: need n >= 1 and a counts array");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemsetAsync(counts, 0, 2 * GS_SELFTEST_CHECKS * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return gs::set_error(GS_ERR_CUDA, cudaGetErrorString(e));
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return gs::set_error(GS_ERR_CUDA, cudaGetErrorString(e));
  k_selftest<<<sms * 8, 256, 0, s>>>(n, seed, counts);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gs::set_error(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}
