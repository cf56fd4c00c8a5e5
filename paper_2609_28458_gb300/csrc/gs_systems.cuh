// Device right-hand sides f(t, y, theta) of the ensemble problem (Sec. 2.1, Eq. ivp) and their
// hand-derived vector-Jacobian products, instantiated in FP64 and FP32 (template R).
//
//   f(t, y, p, out):          out = f
//   vjp(t, y, p, w, gy, gp):  gy = J_y^T w, gp = J_theta^T w   (both overwritten)
//
// Orbit systems: f = (v, -grad Phi(x; theta)); their VJP is gy = (-H w_v, w_x) with H the Hessian
// of Phi, and gp = -d(w_v . grad Phi)/d theta. Every Hessian-vector product below is written from
// the closed-form gradient of the potential it differentiates.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "gs_df64.cuh"

namespace gs {

// Gravitational constant in kpc^3 / (1e10 Msun Myr^2): IAU nominal GM_sun = 1.3271244e20 m^3/s^2,
// 1 kpc = 3.0856775814913673e19 m, 1 Myr = 3.15576e13 s.
constexpr double kGmw = 1e10 * 1.3271244e20 * 3.15576e13 * 3.15576e13 /
                        (3.0856775814913673e19 * 3.0856775814913673e19 * 3.0856775814913673e19);

// 16-byte shared-memory store and load at a shared-window byte address (volatile: kept in program
// order with each other)
__device__ __forceinline__ void st_shared4(unsigned a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w));
}
__device__ __forceinline__ void ld_shared4(unsigned a, float& x, float& y, float& z, float& w) {
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x), "=f"(y), "=f"(z), "=f"(w) : "r"(a));
}

template <class R> __device__ __forceinline__ R gsqrt(R x);
template <> __device__ __forceinline__ double gsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float gsqrt<float>(float x) { return sqrtf(x); }
template <class R> __device__ __forceinline__ R glog1p(R x);
template <> __device__ __forceinline__ double glog1p<double>(double x) { return log1p(x); }
template <> __device__ __forceinline__ float glog1p<float>(float x) { return log1pf(x); }
template <class R> __device__ __forceinline__ R glog(R x);
template <> __device__ __forceinline__ double glog<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float glog<float>(float x) { return logf(x); }
template <class R> __device__ __forceinline__ R gexp(R x);
template <> __device__ __forceinline__ double gexp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float gexp<float>(float x) { return __expf(x); }
// 1/sqrt(x), 1/x, a/b: IEEE FP64 operations in FP64; the SFU-based FP32 intrinsics in FP32 (a few
// ulp, far below the FP32 stage rounding the FP32 path already carries).
template <class R> __device__ __forceinline__ R grsqrt(R x);
template <> __device__ __forceinline__ double grsqrt<double>(double x) { return 1.0 / sqrt(x); }
template <> __device__ __forceinline__ float grsqrt<float>(float x) { return rsqrtf(x); }
template <class R> __device__ __forceinline__ R grcp(R x);
template <> __device__ __forceinline__ double grcp<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float grcp<float>(float x) { return __fdividef(1.0f, x); }
template <class R> __device__ __forceinline__ R gdiv(R a, R b);
template <> __device__ __forceinline__ double gdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float gdiv<float>(float a, float b) { return __fdividef(a, b); }

// ------------------------------------------------------------------------------------------------
// Isochrone, Phi = -1/(1 + s), s = sqrt(1 + r^2): grad Phi = g x with g = 1/(s (1+s)^2);
// H w = g w + 2 g_u (x.w) x with g_u = dg/d(r^2) = -(1 + 3s) / (2 s^3 (1+s)^3).
template <class R>
struct Isochrone {
  static constexpr int D = 6, P = 0;
  static constexpr bool AUTONOMOUS = true;
  static constexpr bool SECOND_ORDER = true;  // y = (x, v), f = (v, a(x))
  __device__ static void f(R, const R* y, const R*, R* out) {
    const R u = R(1) + (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    const R is = grsqrt(u);            // 1/s
    const R iop = grcp(R(1) + u * is);  // 1/(1+s)
    const R g = is * iop * iop;
    out[0] = y[3]; out[1] = y[4]; out[2] = y[5];
    out[3] = -g * y[0]; out[4] = -g * y[1]; out[5] = -g * y[2];
  }
  __device__ static void vjp(R, const R* y, const R*, const R* w, R* gy, R*) {
    const R u = R(1) + (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    const R is = grsqrt(u);
    const R s = u * is;
    const R iop = grcp(R(1) + s);
    const R g = is * iop * iop;
    const R gu = -(R(1) + R(3) * s) * R(0.5) * (is * is * is) * (iop * iop * iop);
    const R xw = y[0] * w[3] + y[1] * w[4] + y[2] * w[5];
    const R c2 = R(2) * gu * xw;
    gy[0] = -(g * w[3] + c2 * y[0]);
    gy[1] = -(g * w[4] + c2 * y[1]);
    gy[2] = -(g * w[5] + c2 * y[2]);
    gy[3] = w[0]; gy[4] = w[1]; gy[5] = w[2];
  }
};

// ------------------------------------------------------------------------------------------------
// Milky-Way-like potential. theta = (M_d, M_b, M_h, q) in 1e10 Msun; a = 3, b = 0.28, c = 1,
// r_s = 15.6 kpc.
//  disc (Miyamoto-Nagai)  Phi_d = -G M_d / D, D^2 = R^2 + A^2, A = a + zeta, zeta = sqrt(z^2+b^2):
//      grad Phi_d = c_d u, c_d = G M_d / D^3, u = (x, y, A z/zeta);
//      H_d w = c_d (w1, w2, u3' w3) - 3 c_d/D^2 (u.w) u, u3' = z^2/zeta^2 + A b^2/zeta^3.
//  bulge (Hernquist)      Phi_b = -G M_b / (r + c): grad = k_b x, k_b = G M_b / (r (r+c)^2);
//      H_b w = k_b w + k_b'/r (x.w) x, k_b'/r = -G M_b (3r + c) / (r^3 (r+c)^3).
//  halo (NFW, flattened)  Phi_h = -G M_h ln(1 + m/r_s)/m, m^2 = R^2 + z^2/q^2:
//      grad = k_h v, v = (x, y, z/q^2), k_h = G M_h psi / m^3, psi = ln(1+m/r_s) - m/(r_s+m);
//      H_h w = k_h (w1, w2, w3/q^2) + k_h'/m (v.w) v,
//      k_h'/m = G M_h [1/(m^3 (r_s+m)^2) - 3 psi/m^5];
//      d(grad Phi_h)/dq = k_h' dm/dq v + k_h (0, 0, -2z/q^3), dm/dq = -z^2/(q^3 m).
template <class R>
struct MilkyWay {
  static constexpr int D = 6, P = 4, PP = 6;  // prepared: p[0..2] = G M, p[4] = 1/q^2, p[5] = 1/q^3
  static constexpr bool AUTONOMOUS = true;
  static constexpr bool SECOND_ORDER = true;  // y = (x, v), f = (v, a(x))
  __device__ static void prep(R* p) {
    const R G = R(kGmw);
    p[0] = G * p[0];
    p[1] = G * p[1];
    p[2] = G * p[2];
    const R iq = grcp(p[3]);
    p[4] = iq * iq;
    p[5] = p[4] * iq;
  }
  // The position-dependent factors of the force and of its Jacobian. u = (x, y, u2) and
  // v = (x, y, vh2); FULL adds the Hessian and q-derivative factors the VJP needs.
  struct Parts {
    R cd0, u2, iD2, kb0, kh0, vh2, iq2;  // c_d / (G M_d), A z / zeta, 1/D^2, k_b / (G M_b), k_h / (G M_h), z/q^2, 1/q^2
    R u3p, kbr0, khm0, iq3;              // u3', k_b'/(r G M_b), k_h'/(m G M_h), 1/q^3
  };
  template <bool FULL>
  __device__ static void parts(const R* y, const R* p, Parts& s) {
    const R a = R(3.0), b = R(0.28), c = R(1.0), rs = R(15.6);
    const R x = y[0], yy = y[1], z = y[2];
    const R R2 = x * x + yy * yy, z2 = z * z;
    const R zq = z2 + b * b;
    const R izeta = grsqrt(zq);
    const R zeta = zq * izeta;
    const R A = a + zeta;
    // 1/sqrt(D2) with one Newton step on the hardware reciprocal square root (FP32: 2 ulp before
    // the step); cheaper than a division and an IEEE square root, as accurate for the gradients
    const R D2 = R2 + A * A;
    R iD = grsqrt(D2);
    iD = iD * (R(1.5) - R(0.5) * D2 * iD * iD);
    s.iD2 = iD * iD;
    s.cd0 = s.iD2 * iD;
    s.u2 = A * z * izeta;
    const R r2 = R2 + z2;
    const R ir = grsqrt(r2);
    const R r = r2 * ir;
    const R irc = grcp(r + c);
    s.kb0 = ir * irc * irc;
    s.iq2 = p[4];
    const R m2 = R2 + z2 * s.iq2;
    const R im = grsqrt(m2);
    const R m = m2 * im;
    const R irsm = grcp(rs + m);
    const R psi = glog1p(m * R(1.0 / 15.6)) - m * irsm;
    const R im2 = im * im;
    const R im3 = im2 * im;
    s.kh0 = psi * im3;
    s.vh2 = z * s.iq2;
    if constexpr (FULL) {
      s.u3p = izeta * izeta * (z2 + A * b * b * izeta);
      // k_b'/r = -(3r + c) / (r^3 (r + c)^3) and k_h'/m = (1/(r_s + m)^2 - 3 psi/m^2) / m^3, from the
      // force factors above
      s.kbr0 = -(R(3) * r + c) * s.kb0 * (ir * ir) * irc;
      s.khm0 = im3 * (irsm * irsm - R(3) * psi * im2);
      s.iq3 = p[5];
    }
  }
  __device__ static void f_from(const R* y, const R* p, const Parts& s, R* out) {
    const R cd = p[0] * s.cd0, kb = p[1] * s.kb0, kh = p[2] * s.kh0;
    const R sd = cd + kb + kh;  // the in-plane force is -(c_d + k_b + k_h) (x, y)
    out[0] = y[3]; out[1] = y[4]; out[2] = y[5];
    out[3] = -sd * y[0];
    out[4] = -sd * y[1];
    out[5] = -(cd * s.u2 + kb * y[2] + kh * s.vh2);
  }
  __device__ static void vjp_from(const R* y, const R* p, const R* w, const Parts& s, R* gy, R* gp) {
    const R x = y[0], yy = y[1], z = y[2];
    const R wv[3] = {w[3], w[4], w[5]};
    const R cd = p[0] * s.cd0, kb = p[1] * s.kb0, kh = p[2] * s.kh0;
    const R xy = x * wv[0] + yy * wv[1];
    const R uw = xy + s.u2 * wv[2];
    const R xw = xy + z * wv[2];
    const R vw = xy + s.vh2 * wv[2];
    // H w = (c_d + k_b + k_h) w (with c_d u3' and k_h/q^2 in the z row) plus the rank-one parts
    // k_b'/r (x.w) x + k_h'/m (v.w) v - 3 c_d/D^2 (u.w) u; the in-plane rows share x_i times one term
    const R bx = p[1] * s.kbr0 * xw, hv = p[2] * s.khm0 * vw, du = R(3) * cd * s.iD2 * uw;
    const R sd = cd + kb + kh;
    const R tp = bx + hv - du;
    R Hw[3];
    Hw[0] = sd * wv[0] + tp * x;
    Hw[1] = sd * wv[1] + tp * yy;
    Hw[2] = (cd * s.u3p + kb + kh * s.iq2) * wv[2] + bx * z + hv * s.vh2 - du * s.u2;
    gy[0] = -Hw[0]; gy[1] = -Hw[1]; gy[2] = -Hw[2];
    gy[3] = w[0]; gy[4] = w[1]; gy[5] = w[2];
    // the masses' cotangents per unit of the prepared G M (vjp_param_scale: the caller multiplies
    // by G once per trajectory)
    gp[0] = -s.cd0 * uw;
    gp[1] = -s.kb0 * xw;
    gp[2] = -s.kh0 * vw;
    // -(k_h' dm/dq (v.w) + k_h (-2 z/q^3) w_z), dm/dq = -z^2/(q^3 m)
    gp[3] = z * s.iq3 * (hv * z + R(2) * kh * wv[2]);
  }
  // the factor from gp[q] as vjp gives it to the cotangent of parameter q: G for the masses
  __device__ static double vjp_param_scale(int q) { return q < 3 ? kGmw : 1.0; }
  __device__ static void f(R, const R* y, const R* p, R* out) {
    Parts s;
    parts<false>(y, p, s);
    f_from(y, p, s, out);
  }
  __device__ static void vjp(R, const R* y, const R* p, const R* w, R* gy, R* gp) {
    Parts s;
    parts<true>(y, p, s);
    vjp_from(y, p, w, s, gy, gp);
  }
  // FP32 reverse pass: f at a recomputed stage also leaves the stage's Jacobian factors in shared
  // memory (two float4 at the shared-window byte addresses sl and sl + st), and the stage's VJP reads
  // them back instead of evaluating the potential again.
  static constexpr int kSaveQ = 2;
  __device__ static void f_save(R, const R* y, const R* p, R* out, unsigned sl, unsigned st) {
    static_assert(std::is_same<R, float>::value, "saved stage factors are FP32");
    Parts s;
    parts<true>(y, p, s);
    f_from(y, p, s, out);
    st_shared4(sl, s.cd0, s.u2, s.iD2, s.u3p);
    st_shared4(sl + st, s.kb0, s.kbr0, s.kh0, s.khm0);
  }
  __device__ static void vjp_saved(R, const R* y, const R* p, const R* w, R* gy, R* gp, unsigned sl, unsigned st) {
    static_assert(std::is_same<R, float>::value, "saved stage factors are FP32");
    Parts s;
    ld_shared4(sl, s.cd0, s.u2, s.iD2, s.u3p);
    ld_shared4(sl + st, s.kb0, s.kbr0, s.kh0, s.khm0);
    s.iq2 = p[4];
    s.iq3 = p[5];
    s.vh2 = y[2] * s.iq2;
    vjp_from(y, p, w, s, gy, gp);
  }
};

// ------------------------------------------------------------------------------------------------
// Flattened logarithmic halo, Eq. loghalo: Phi = (v_c^2/2) ln Q, Q = R_c^2 + R^2 + z^2/q^2;
// grad Phi = kappa v, kappa = v_c^2/Q, v = (x, y, z/q^2);
// H w = kappa (w1, w2, w3/q^2) - 2 v_c^2/Q^2 (v.w) v. theta = (v_c, R_c, q).
template <class R>
struct LogHalo {
  static constexpr int D = 6, P = 3, PP = 5;  // p[3] = 1/q^2, p[4] = 1/q^3
  static constexpr bool AUTONOMOUS = true;
  static constexpr bool SECOND_ORDER = true;  // y = (x, v), f = (v, a(x))
  __device__ static void prep(R* p) {
    const R iq = grcp(p[2]);
    p[3] = iq * iq;
    p[4] = p[3] * iq;
  }
  __device__ static void f(R, const R* y, const R* p, R* out) {
    const R iq2 = p[3];
    const R Q = p[1] * p[1] + y[0] * y[0] + y[1] * y[1] + y[2] * y[2] * iq2;
    const R k = p[0] * p[0] * grcp(Q);
    out[0] = y[3]; out[1] = y[4]; out[2] = y[5];
    out[3] = -k * y[0]; out[4] = -k * y[1]; out[5] = -k * y[2] * iq2;
  }
  __device__ static void vjp(R, const R* y, const R* p, const R* w, R* gy, R* gp) {
    const R vc = p[0], Rc = p[1];
    const R iq2 = p[3], iq3 = p[4];
    const R Q = Rc * Rc + y[0] * y[0] + y[1] * y[1] + y[2] * y[2] * iq2;
    const R iQ = grcp(Q);
    const R k = vc * vc * iQ;
    const R k2 = R(2) * vc * vc * iQ * iQ;
    const R v2 = y[2] * iq2;
    const R vw = y[0] * w[3] + y[1] * w[4] + v2 * w[5];
    gy[0] = -(k * w[3] - k2 * vw * y[0]);
    gy[1] = -(k * w[4] - k2 * vw * y[1]);
    gy[2] = -(k * iq2 * w[5] - k2 * vw * v2);
    gy[3] = w[0]; gy[4] = w[1]; gy[5] = w[2];
    const R z = y[2];
    gp[0] = -(R(2) * vc * iQ) * vw;
    gp[1] = Rc * k2 * vw;
    gp[2] = -k2 * z * z * iq3 * vw + R(2) * k * z * iq3 * w[5];
  }
};

// ------------------------------------------------------------------------------------------------
// Orbit-averaged spin precession in v (Sec. 5, Eqs. prec-spins, prec-L, prec-omega, prec-rr),
// G = c = M = 1, y = (Lhat, S1hat, S2hat), theta = (q, chi1, chi2). Radiation reaction
// dv/dt = 32/5 eta v^9 (1 + b2 v^2 + b3 v^3 + b4 v^4) with the 2PN coefficients of Kidder (1995):
// b2 = -(743 + 924 eta)/336, b3 = 4 pi - beta, b4 = 34103/18144 + 13661 eta/2016 + 59 eta^2/18
// - eta/48 chi1 chi2 (247 S1.S2 - 721 (L.S1)(L.S2)), beta = 1/12 sum_j chi_j (L.S_j)(113 m_j^2 + 75 eta).
// The VJP is the reverse sweep of the forward evaluation, statement by statement.
template <class R>
__device__ __forceinline__ void cross3(const R* a, const R* b, R* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
template <class R>
__device__ __forceinline__ R dot3(const R* a, const R* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

template <class R>
struct Precession {
  static constexpr int D = 9, P = 3, PP = 6;  // p[3] = m1 = 1/(1+q), p[4] = 1/q, p[5] = 1/eta
  static constexpr bool AUTONOMOUS = false;
  __device__ static void prep(R* p) {
    p[3] = R(1) / (R(1) + p[0]);
    p[4] = R(1) / p[0];
    p[5] = R(1) / (p[3] * (p[0] * p[3]));
  }
  struct Fwd {
    R m1, m2, eta, S1, S2, L, h, q, iq, ieta, iv;
    R Lv[3], S1v[3], S2v[3], a1[3], a2[3], pr1, pr2, w1[3], w2[3], ds1[3], ds2[3], U[3], dL[3];
    R ls1, ls2, s12, X, T1, T2, b2, b3, b4, poly, dvdt, inv, v2, v3, v9;
  };
  __device__ static void fwd(R v, const R* y, const R* p, Fwd& F) {
    const R pi = R(3.14159265358979323846);
    const R* Lh = y; const R* s1 = y + 3; const R* s2 = y + 6;
    F.q = p[0];
    const R chi1 = p[1], chi2 = p[2];
    F.m1 = p[3];
    F.iq = p[4];
    F.ieta = p[5];
    F.m2 = F.q * F.m1;
    F.eta = F.m1 * F.m2;
    F.S1 = chi1 * F.m1 * F.m1;
    F.S2 = chi2 * F.m2 * F.m2;
    F.iv = R(1) / v;
    F.L = F.eta * F.iv;
    F.v2 = v * v; F.v3 = F.v2 * v;
    const R v6 = F.v3 * F.v3;
    F.v9 = v6 * F.v3;
    F.h = R(0.5) * v6;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      F.Lv[i] = F.L * Lh[i]; F.S1v[i] = F.S1 * s1[i]; F.S2v[i] = F.S2 * s2[i];
      F.a1[i] = F.S2v[i] + F.q * F.S1v[i];
      F.a2[i] = F.S1v[i] + F.S2v[i] * F.iq;
    }
    F.pr1 = dot3(Lh, F.a1);
    F.pr2 = dot3(Lh, F.a2);
    const R c1 = R(4) + R(3) * F.q, c2 = R(4) + R(3) * F.iq;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      F.w1[i] = F.h * (c1 * F.Lv[i] + F.S2v[i] - R(3) * F.pr1 * Lh[i]);
      F.w2[i] = F.h * (c2 * F.Lv[i] + F.S1v[i] - R(3) * F.pr2 * Lh[i]);
    }
    cross3(F.w1, s1, F.ds1);
    cross3(F.w2, s2, F.ds2);
    const R k = -v * F.ieta;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      F.U[i] = F.S1 * F.ds1[i] + F.S2 * F.ds2[i];
      F.dL[i] = k * F.U[i];
    }
    F.ls1 = dot3(Lh, s1); F.ls2 = dot3(Lh, s2); F.s12 = dot3(s1, s2);
    F.b2 = -(R(743) + R(924) * F.eta) * R(1.0 / 336.0);
    F.T1 = R(113) * F.m1 * F.m1 + R(75) * F.eta;
    F.T2 = R(113) * F.m2 * F.m2 + R(75) * F.eta;
    const R beta = (chi1 * F.ls1 * F.T1 + chi2 * F.ls2 * F.T2) * R(1.0 / 12.0);
    F.b3 = R(4) * pi - beta;
    F.X = R(247) * F.s12 - R(721) * F.ls1 * F.ls2;
    F.b4 = R(34103.0 / 18144.0) + R(13661.0 / 2016.0) * F.eta + R(59.0 / 18.0) * F.eta * F.eta -
           (F.eta * R(1.0 / 48.0)) * chi1 * chi2 * F.X;
    F.poly = R(1) + F.b2 * F.v2 + F.b3 * F.v3 + F.b4 * F.v2 * F.v2;
    F.dvdt = R(32.0 / 5.0) * F.eta * F.v9 * F.poly;
    F.inv = R(1) / F.dvdt;
  }
  __device__ static void f(R v, const R* y, const R* p, R* out) {
    Fwd F;
    fwd(v, y, p, F);
#pragma unroll
    for (int i = 0; i < 3; i++) {
      out[i] = F.dL[i] * F.inv;
      out[3 + i] = F.ds1[i] * F.inv;
      out[6 + i] = F.ds2[i] * F.inv;
    }
  }
  __device__ static void vjp(R v, const R* y, const R* p, const R* g, R* gy, R* gp) {
    Fwd F;
    fwd(v, y, p, F);
    const R* Lh = y; const R* s1 = y + 3; const R* s2 = y + 6;
    const R chi1 = p[1], chi2 = p[2];
    R Lh_b[3] = {0, 0, 0}, s1_b[3] = {0, 0, 0}, s2_b[3] = {0, 0, 0};
    R q_b = 0, c1_b = 0, c2_b = 0, eta_b = 0, m1_b = 0, m2_b = 0, S1_b = 0, S2_b = 0, L_b = 0;
    // out = (dL, ds1, ds2) * inv
    const R inv_b = dot3(g, F.dL) + dot3(g + 3, F.ds1) + dot3(g + 6, F.ds2);
    R dL_b[3], ds1_b[3], ds2_b[3];
#pragma unroll
    for (int i = 0; i < 3; i++) { dL_b[i] = g[i] * F.inv; ds1_b[i] = g[3 + i] * F.inv; ds2_b[i] = g[6 + i] * F.inv; }
    // inv = 1/dvdt
    const R dvdt_b = -inv_b * F.inv * F.inv;
    // dvdt = 32/5 eta v9 poly
    const R poly_b = dvdt_b * R(32.0 / 5.0) * F.eta * F.v9;
    eta_b += dvdt_b * R(32.0 / 5.0) * F.v9 * F.poly;
    // poly = 1 + b2 v2 + b3 v3 + b4 v4
    const R b2_b = poly_b * F.v2, b3_b = poly_b * F.v3, b4_b = poly_b * F.v2 * F.v2;
    // b4
    const R e48 = F.eta * R(1.0 / 48.0);
    eta_b += b4_b * (R(13661.0 / 2016.0) + R(2.0 * 59.0 / 18.0) * F.eta - chi1 * chi2 * F.X * R(1.0 / 48.0));
    c1_b += b4_b * (-e48 * chi2 * F.X);
    c2_b += b4_b * (-e48 * chi1 * F.X);
    const R X_b = b4_b * (-e48 * chi1 * chi2);
    R s12_b = R(247) * X_b;
    R ls1_b = -R(721) * F.ls2 * X_b;
    R ls2_b = -R(721) * F.ls1 * X_b;
    // b3 = 4 pi - beta, beta = (chi1 ls1 T1 + chi2 ls2 T2)/12
    const R beta_b = -b3_b;
    const R beta12 = beta_b * R(1.0 / 12.0);
    c1_b += beta12 * F.ls1 * F.T1;
    ls1_b += beta12 * chi1 * F.T1;
    const R T1_b = beta12 * chi1 * F.ls1;
    c2_b += beta12 * F.ls2 * F.T2;
    ls2_b += beta12 * chi2 * F.T2;
    const R T2_b = beta12 * chi2 * F.ls2;
    m1_b += T1_b * R(226) * F.m1;
    m2_b += T2_b * R(226) * F.m2;
    eta_b += R(75) * (T1_b + T2_b);
    // b2 = -(743 + 924 eta)/336
    eta_b += b2_b * (-R(924) / R(336));
    // ls1, ls2, s12
#pragma unroll
    for (int i = 0; i < 3; i++) {
      Lh_b[i] += ls1_b * s1[i] + ls2_b * s2[i];
      s1_b[i] += ls1_b * Lh[i] + s12_b * s2[i];
      s2_b[i] += ls2_b * Lh[i] + s12_b * s1[i];
    }
    // dL = -(v/eta) U, U = S1 ds1 + S2 ds2
    R U_b[3];
    const R k = -v * F.ieta;
#pragma unroll
    for (int i = 0; i < 3; i++) U_b[i] = k * dL_b[i];
    eta_b += (v * F.ieta * F.ieta) * dot3(dL_b, F.U);
    S1_b += dot3(U_b, F.ds1);
    S2_b += dot3(U_b, F.ds2);
#pragma unroll
    for (int i = 0; i < 3; i++) { ds1_b[i] += F.S1 * U_b[i]; ds2_b[i] += F.S2 * U_b[i]; }
    // ds_j = w_j x s_j:  w_b = s x r_b,  s_b += r_b x w
    R w1_b[3], w2_b[3], tmp[3];
    cross3(s1, ds1_b, w1_b);
    cross3(s2, ds2_b, w2_b);
    cross3(ds1_b, F.w1, tmp);
#pragma unroll
    for (int i = 0; i < 3; i++) s1_b[i] += tmp[i];
    cross3(ds2_b, F.w2, tmp);
#pragma unroll
    for (int i = 0; i < 3; i++) s2_b[i] += tmp[i];
    // w1 = h ((4+3q) Lv + S2v - 3 pr1 Lh), w2 = h ((4+3/q) Lv + S1v - 3 pr2 Lh)
    const R c1 = R(4) + R(3) * F.q, c2 = R(4) + R(3) * F.iq;
    R Lv_b[3], S1v_b[3], S2v_b[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
      Lv_b[i] = F.h * (c1 * w1_b[i] + c2 * w2_b[i]);
      S2v_b[i] = F.h * w1_b[i];
      S1v_b[i] = F.h * w2_b[i];
    }
    q_b += F.h * (R(3) * dot3(F.Lv, w1_b) - (R(3) * F.iq * F.iq) * dot3(F.Lv, w2_b));
    const R pr1_b = -R(3) * F.h * dot3(Lh, w1_b);
    const R pr2_b = -R(3) * F.h * dot3(Lh, w2_b);
#pragma unroll
    for (int i = 0; i < 3; i++) Lh_b[i] += -R(3) * F.h * (F.pr1 * w1_b[i] + F.pr2 * w2_b[i]);
    // pr_j = Lh . a_j
    R a1_b[3], a2_b[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
      Lh_b[i] += pr1_b * F.a1[i] + pr2_b * F.a2[i];
      a1_b[i] = pr1_b * Lh[i];
      a2_b[i] = pr2_b * Lh[i];
    }
    // a1 = S2v + q S1v, a2 = S1v + S2v/q
#pragma unroll
    for (int i = 0; i < 3; i++) {
      S2v_b[i] += a1_b[i] + a2_b[i] * F.iq;
      S1v_b[i] += F.q * a1_b[i] + a2_b[i];
    }
    q_b += dot3(F.S1v, a1_b) - dot3(F.S2v, a2_b) * (F.iq * F.iq);
    // Lv = L Lh, S1v = S1 s1, S2v = S2 s2
    L_b += dot3(Lh, Lv_b);
    S1_b += dot3(s1, S1v_b);
    S2_b += dot3(s2, S2v_b);
#pragma unroll
    for (int i = 0; i < 3; i++) {
      Lh_b[i] += F.L * Lv_b[i];
      s1_b[i] += F.S1 * S1v_b[i];
      s2_b[i] += F.S2 * S2v_b[i];
    }
    // L = eta / v
    eta_b += L_b * F.iv;
    // S1 = chi1 m1^2, S2 = chi2 m2^2
    c1_b += S1_b * F.m1 * F.m1;
    m1_b += S1_b * R(2) * chi1 * F.m1;
    c2_b += S2_b * F.m2 * F.m2;
    m2_b += S2_b * R(2) * chi2 * F.m2;
    // eta = m1 m2
    m1_b += eta_b * F.m2;
    m2_b += eta_b * F.m1;
    // m2 = q m1
    q_b += m2_b * F.m1;
    m1_b += m2_b * F.q;
    // m1 = 1/(1+q)
    q_b += -m1_b * F.m1 * F.m1;
#pragma unroll
    for (int i = 0; i < 3; i++) { gy[i] = Lh_b[i]; gy[3 + i] = s1_b[i]; gy[6 + i] = s2_b[i]; }
    gp[0] = q_b; gp[1] = c1_b; gp[2] = c2_b;
  }
};

// ------------------------------------------------------------------------------------------------
// Thawing quintessence in N = ln a (Sec. 4.1, Eq. de-model; Appendix C, Eq. de-rhs):
// E^2 = (Om e^-3N + Or e^-4N + a0 e^-lam phi) / (1 - u^2/6),
// dlnE/dN = -(3 Om e^-3N + 4 Or e^-4N)/(2 E^2) - u^2/2,
// phi' = u, u' = -(3 + dlnE/dN) u + 3 lam a0 e^-lam phi / E^2, I' = e^-N / E.
template <class R>
struct Quintessence {
  static constexpr int D = 3, P = 4;
  static constexpr bool AUTONOMOUS = false;
  __device__ static void f(R N, const R* y, const R* p, R* out) {
    const R u = y[1];
    const R ev = gexp(-p[1] * y[0]);
    const R vphi = p[0] * ev;
    const R em3 = gexp(R(-3) * N), em4 = gexp(R(-4) * N);
    const R E2 = gdiv(p[2] * em3 + p[3] * em4 + vphi, R(1) - u * u * R(1.0 / 6.0));
    const R iE2 = grcp(E2);
    const R dlnE = -(R(3) * p[2] * em3 + R(4) * p[3] * em4) * R(0.5) * iE2 - u * u * R(0.5);
    out[0] = u;
    out[1] = -(R(3) + dlnE) * u + R(3) * p[1] * vphi * iE2;
    out[2] = gexp(-N) * grsqrt(E2);
  }
  __device__ static void vjp(R N, const R* y, const R* p, const R* g, R* gy, R* gp) {
    const R phi = y[0], u = y[1];
    const R a0 = p[0], lam = p[1], om = p[2], orad = p[3];
    const R ev = gexp(-lam * phi);
    const R vphi = a0 * ev;
    const R em3 = gexp(R(-3) * N), em4 = gexp(R(-4) * N);
    const R num = om * em3 + orad * em4 + vphi;
    const R den = R(1) - u * u / R(6);
    const R E2 = num / den;
    const R Mm = R(3) * om * em3 + R(4) * orad * em4;
    const R dlnE = -Mm / (R(2) * E2) - u * u / R(2);
    const R f2 = gexp(-N) / gsqrt(E2);
    R u_b = g[0];
    // f1 = -(3 + dlnE) u + 3 lam vphi / E2
    const R dlnE_b = -g[1] * u;
    u_b += -(R(3) + dlnE) * g[1];
    R lam_b = R(3) * vphi / E2 * g[1];
    R vphi_b = R(3) * lam / E2 * g[1];
    R E2_b = -R(3) * lam * vphi / (E2 * E2) * g[1];
    // f2 = e^-N E2^-1/2
    E2_b += -R(0.5) * f2 / E2 * g[2];
    // dlnE = -M/(2 E2) - u^2/2
    const R M_b = -dlnE_b / (R(2) * E2);
    E2_b += dlnE_b * Mm / (R(2) * E2 * E2);
    u_b += -u * dlnE_b;
    R om_b = R(3) * em3 * M_b;
    R or_b = R(4) * em4 * M_b;
    // E2 = num / den
    const R num_b = E2_b / den;
    const R den_b = -E2_b * E2 / den;
    u_b += -(u / R(3)) * den_b;
    om_b += em3 * num_b;
    or_b += em4 * num_b;
    vphi_b += num_b;
    // vphi = a0 ev, ev = exp(-lam phi)
    const R a0_b = ev * vphi_b;
    const R ev_b = a0 * vphi_b;
    lam_b += -phi * ev * ev_b;
    const R phi_b = -lam * ev * ev_b;
    gy[0] = phi_b; gy[1] = u_b; gy[2] = R(0);
    gp[0] = a0_b; gp[1] = lam_b; gp[2] = om_b; gp[3] = or_b;
  }
};

// Systems whose right-hand sides use only what df64 provides (+, -, *, /, square roots): they are
// instantiated in precision mode 3 as well.
template <template <class> class SysT> struct HasDF64 { static constexpr bool value = false; };
template <> struct HasDF64<Isochrone> { static constexpr bool value = true; };
template <> struct HasDF64<LogHalo> { static constexpr bool value = true; };
template <> struct HasDF64<Precession> { static constexpr bool value = true; };

// Per-trajectory constants: a system may declare PP > P and prep(p), which fills p[P .. PP-1] from
// theta = p[0 .. P-1] once per trajectory (reciprocals of parameters, mass ratios), so that f and
// its VJP read them instead of dividing at every stage. Gradients stay with respect to theta.
template <class Sys, class = void> struct PrepCount { static constexpr int value = Sys::P; };
template <class Sys> struct PrepCount<Sys, std::void_t<decltype(Sys::PP)>> { static constexpr int value = Sys::PP; };
template <class Sys, class Rp>
__device__ __forceinline__ void prep_params(Rp* p) {
  if constexpr (PrepCount<Sys>::value > Sys::P) Sys::prep(p);
}

// float4s per stage that a system's f_save leaves for its vjp_saved (0: the system has neither)
template <class Sys, class = void> struct SaveQ { static constexpr int value = 0; };
template <class Sys> struct SaveQ<Sys, std::void_t<decltype(Sys::kSaveQ)>> { static constexpr int value = Sys::kSaveQ; };
// second-order systems: y = (x, v) with f(y) = (v, a(x)), the acceleration independent of v (and of
// t); the FP32 modes take their stages in Nystrom form (gs_tableaux.cuh, Nystrom)
template <class Sys, class = void> struct SecondOrder { static constexpr bool value = false; };
template <class Sys> struct SecondOrder<Sys, std::void_t<decltype(Sys::SECOND_ORDER)>> {
  static constexpr bool value = Sys::SECOND_ORDER;
};
// The factor that turns a system's parameter cotangent, as its vjp returns it, into the cotangent of
// the parameter itself: 1, except where prep() rescales a parameter and vjp differentiates by the
// prepared value (the Milky-Way masses, prepared as G M). Callers apply it once per trajectory.
template <class Sys, class = void> struct VjpParamScale {
  __device__ static double of(int) { return 1.0; }
};
template <class Sys> struct VjpParamScale<Sys, std::void_t<decltype(Sys::vjp_param_scale(0))>> {
  __device__ static double of(int q) { return Sys::vjp_param_scale(q); }
};

}  // namespace gs
