// Forward-mode dual numbers for the device right-hand sides: a value and M directional derivatives.
// Instantiating a system on Dual<R, M> evaluates f and its Jacobian-vector products
// J_y v + J_theta w along M directions at once (Sec. 2.3, Eq. sens: the right-hand side of the
// sensitivity equations). Value parts use exactly the scalar operations, so a step taken on duals
// makes the same decisions as the scalar step.
#pragma once
#include <cuda_runtime.h>

#include "gs_systems.cuh"

namespace gs {

template <class R, int M>
struct Dual {
  R v;
  R d[M];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double x) : v(R(x)) {
#pragma unroll
    for (int i = 0; i < M; i++) d[i] = R(0);
  }
  __device__ __forceinline__ Dual(float x) : v(R(x)) {
#pragma unroll
    for (int i = 0; i < M; i++) d[i] = R(0);
  }
  __device__ __forceinline__ Dual(int x) : v(R(x)) {
#pragma unroll
    for (int i = 0; i < M; i++) d[i] = R(0);
  }
};

template <class T> struct DualTraits { using Base = T; static constexpr int M = 0; };
template <class R, int M_> struct DualTraits<Dual<R, M_>> { using Base = R; static constexpr int M = M_; };

__device__ __forceinline__ float val(float x) { return x; }
__device__ __forceinline__ double val(double x) { return x; }
template <class R, int M> __device__ __forceinline__ R val(const Dual<R, M>& x) { return x.v; }

#define GS_DUAL_LOOP(expr) _Pragma("unroll") for (int i = 0; i < M; i++) r.d[i] = (expr);

template <class R, int M> __device__ __forceinline__ Dual<R, M> operator+(const Dual<R, M>& a, const Dual<R, M>& b) {
  Dual<R, M> r; r.v = a.v + b.v; GS_DUAL_LOOP(a.d[i] + b.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator-(const Dual<R, M>& a, const Dual<R, M>& b) {
  Dual<R, M> r; r.v = a.v - b.v; GS_DUAL_LOOP(a.d[i] - b.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator-(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = -a.v; GS_DUAL_LOOP(-a.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator*(const Dual<R, M>& a, const Dual<R, M>& b) {
  Dual<R, M> r; r.v = a.v * b.v; GS_DUAL_LOOP(a.d[i] * b.v + a.v * b.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator/(const Dual<R, M>& a, const Dual<R, M>& b) {
  Dual<R, M> r; r.v = a.v / b.v; const R ib = R(1) / b.v; GS_DUAL_LOOP((a.d[i] - r.v * b.d[i]) * ib) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator+(const Dual<R, M>& a, R b) {
  Dual<R, M> r = a; r.v = a.v + b; return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator+(R a, const Dual<R, M>& b) {
  Dual<R, M> r = b; r.v = a + b.v; return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator-(const Dual<R, M>& a, R b) {
  Dual<R, M> r = a; r.v = a.v - b; return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator-(R a, const Dual<R, M>& b) {
  Dual<R, M> r; r.v = a - b.v; GS_DUAL_LOOP(-b.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator*(const Dual<R, M>& a, R b) {
  Dual<R, M> r; r.v = a.v * b; GS_DUAL_LOOP(a.d[i] * b) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator*(R a, const Dual<R, M>& b) {
  Dual<R, M> r; r.v = a * b.v; GS_DUAL_LOOP(a * b.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> operator/(const Dual<R, M>& a, R b) {
  Dual<R, M> r; r.v = a.v / b; const R ib = R(1) / b; GS_DUAL_LOOP(a.d[i] * ib) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M>& operator+=(Dual<R, M>& a, const Dual<R, M>& b) {
  a = a + b; return a;
}

// elementary functions used by the right-hand sides (chain rule on the derivative parts)
template <class R, int M> __device__ __forceinline__ Dual<R, M> gsqrt(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = gsqrt(a.v); const R c = R(0.5) * grcp(r.v); GS_DUAL_LOOP(c * a.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> grsqrt(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = grsqrt(a.v); const R c = R(-0.5) * r.v * r.v * r.v; GS_DUAL_LOOP(c * a.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> grcp(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = grcp(a.v); const R c = -r.v * r.v; GS_DUAL_LOOP(c * a.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> gdiv(const Dual<R, M>& a, const Dual<R, M>& b) {
  Dual<R, M> r; const R ib = grcp(b.v); r.v = gdiv(a.v, b.v); GS_DUAL_LOOP((a.d[i] - r.v * b.d[i]) * ib) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> gexp(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = gexp(a.v); GS_DUAL_LOOP(r.v * a.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> glog(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = glog(a.v); const R c = grcp(a.v); GS_DUAL_LOOP(c * a.d[i]) return r;
}
template <class R, int M> __device__ __forceinline__ Dual<R, M> glog1p(const Dual<R, M>& a) {
  Dual<R, M> r; r.v = glog1p(a.v); const R c = grcp(R(1) + a.v); GS_DUAL_LOOP(c * a.d[i]) return r;
}

#undef GS_DUAL_LOOP

}  // namespace gs
