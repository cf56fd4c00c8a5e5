// Oracle (test infrastructure only): forward-mode dual numbers. They supply the products
// J_y S + df/dtheta of the forward sensitivity equations (Sec. 2.3, Eq. sens; Appendix A,
// Eq. stage-sens) and, nested once, the gradient of a potential for the orbit systems.
// The value part of every operation is the same floating-point operation as on plain doubles,
// so a solve carried out in duals takes bit-for-bit the same steps as a solve in doubles.
#pragma once
#include <cmath>

namespace orc {

template <class S, int M>
struct Dual {
  S v;
  S d[M];
  Dual() : v(0.0) { for (int i = 0; i < M; i++) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < M; i++) d[i] = 0.0; }
};

inline double val(double x) { return x; }
template <class S, int M> inline double val(const Dual<S, M>& x) { return val(x.v); }

template <class S, int M> inline Dual<S, M> operator+(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v + b.v; for (int i = 0; i < M; i++) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <class S, int M> inline Dual<S, M> operator-(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v - b.v; for (int i = 0; i < M; i++) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <class S, int M> inline Dual<S, M> operator-(const Dual<S, M>& a) {
  Dual<S, M> r; r.v = -a.v; for (int i = 0; i < M; i++) r.d[i] = -a.d[i]; return r;
}
template <class S, int M> inline Dual<S, M> operator*(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v * b.v;
  for (int i = 0; i < M; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class S, int M> inline Dual<S, M> operator/(const Dual<S, M>& a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a.v / b.v;
  for (int i = 0; i < M; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
// mixed with plain doubles
template <class S, int M> inline Dual<S, M> operator+(const Dual<S, M>& a, double b) {
  Dual<S, M> r = a; r.v = a.v + b; return r;
}
template <class S, int M> inline Dual<S, M> operator+(double a, const Dual<S, M>& b) {
  Dual<S, M> r = b; r.v = a + b.v; return r;
}
template <class S, int M> inline Dual<S, M> operator-(const Dual<S, M>& a, double b) {
  Dual<S, M> r = a; r.v = a.v - b; return r;
}
template <class S, int M> inline Dual<S, M> operator-(double a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a - b.v; for (int i = 0; i < M; i++) r.d[i] = -b.d[i]; return r;
}
template <class S, int M> inline Dual<S, M> operator*(const Dual<S, M>& a, double b) {
  Dual<S, M> r; r.v = a.v * b; for (int i = 0; i < M; i++) r.d[i] = a.d[i] * b; return r;
}
template <class S, int M> inline Dual<S, M> operator*(double a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a * b.v; for (int i = 0; i < M; i++) r.d[i] = a * b.d[i]; return r;
}
template <class S, int M> inline Dual<S, M> operator/(const Dual<S, M>& a, double b) {
  Dual<S, M> r; r.v = a.v / b; for (int i = 0; i < M; i++) r.d[i] = a.d[i] / b; return r;
}
template <class S, int M> inline Dual<S, M> operator/(double a, const Dual<S, M>& b) {
  Dual<S, M> r; r.v = a / b.v;
  for (int i = 0; i < M; i++) r.d[i] = -(r.v * b.d[i]) / b.v;
  return r;
}
template <class S, int M> inline Dual<S, M>& operator+=(Dual<S, M>& a, const Dual<S, M>& b) { a = a + b; return a; }
template <class S, int M> inline Dual<S, M>& operator-=(Dual<S, M>& a, const Dual<S, M>& b) { a = a - b; return a; }

// elementary functions: chain rule on the derivative part
using std::sqrt; using std::log; using std::exp; using std::sin; using std::cos; using std::atan2;
template <class S, int M> inline Dual<S, M> sqrt(const Dual<S, M>& a) {
  Dual<S, M> r; r.v = sqrt(a.v);
  for (int i = 0; i < M; i++) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
template <class S, int M> inline Dual<S, M> log(const Dual<S, M>& a) {
  Dual<S, M> r; r.v = log(a.v);
  for (int i = 0; i < M; i++) r.d[i] = a.d[i] / a.v;
  return r;
}
template <class S, int M> inline Dual<S, M> exp(const Dual<S, M>& a) {
  Dual<S, M> r; r.v = exp(a.v);
  for (int i = 0; i < M; i++) r.d[i] = r.v * a.d[i];
  return r;
}

}  // namespace orc
