// Oracle (test infrastructure only): right-hand sides f(t, y, theta) of the ensemble problem
// (Sec. 2.1, Eq. ivp), templated on the scalar so that the same code runs on doubles and on
// dual numbers. Every function cites the passage whose formula it writes out.
//
// Orbit systems are written as a potential Phi(x; theta); the acceleration -grad Phi is taken by
// forward-mode differentiation of Phi itself, so no hand-derived gradient enters the oracle.
#pragma once
#include <cmath>
#include "dual.hpp"

namespace orc {

enum { S_ISOCHRONE = 0, S_MW = 1, S_PRECESSION = 2, S_QUINTESSENCE = 3, S_LOGHALO = 4, S_LINEAR = 5 };

inline void dims(int sys, int* d, int* p) {
  switch (sys) {
    case S_ISOCHRONE: *d = 6; *p = 0; return;
    case S_MW: *d = 6; *p = 4; return;
    case S_PRECESSION: *d = 9; *p = 3; return;
    case S_QUINTESSENCE: *d = 3; *p = 4; return;
    case S_LOGHALO: *d = 6; *p = 3; return;
    case S_LINEAR: *d = 1; *p = 1; return;
    default: *d = 0; *p = 0;
  }
}

// ---------------------------------------------------------------------------------------------
// Gravitational constant in kpc^3 / (1e10 Msun Myr^2), from the IAU nominal solar mass
// parameter GM_sun = 1.3271244e20 m^3 s^-2, 1 kpc = 3.0856775814913673e19 m and
// 1 Myr = 1e6 Julian years = 3.15576e13 s.
inline double g_kpc_myr() {
  const double gm_sun = 1.3271244e20, kpc = 3.0856775814913673e19, myr = 3.15576e13;
  return 1e10 * gm_sun * myr * myr / (kpc * kpc * kpc);
}

// Isochrone potential Phi = -1/(1 + sqrt(1 + r^2)) in units G = M = b = 1 (Binney & Tremaine,
// the textbook the paper cites for its potential, Sec. 3).
template <class T>
T phi_isochrone(const T x[3], const T* /*p*/) {
  T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  return -1.0 / (1.0 + sqrt(1.0 + r2));
}

// Milky-Way-like potential: Miyamoto-Nagai disc (a = 3, b = 0.28 kpc) + Hernquist bulge
// (c = 1 kpc) + NFW halo (r_s = 15.6 kpc) flattened along z by q (r_q^2 = R^2 + z^2/q^2).
// theta = (M_disc, M_bulge, M_halo, q) with masses in 1e10 Msun; M_halo is the NFW scale mass.
template <class T>
T phi_mw(const T x[3], const T* p) {
  const double G = g_kpc_myr();
  const double a = 3.0, b = 0.28, c = 1.0, rs = 15.6;
  T R2 = x[0] * x[0] + x[1] * x[1];
  T z2 = x[2] * x[2];
  T zb = sqrt(z2 + b * b);
  T ad = a + zb;
  T phi_disc = -G * p[0] / sqrt(R2 + ad * ad);
  T r = sqrt(R2 + z2);
  T phi_bulge = -G * p[1] / (r + c);
  T rq = sqrt(R2 + z2 / (p[3] * p[3]));
  T phi_halo = -G * p[2] * log(1.0 + rq / rs) / rq;
  return phi_disc + phi_bulge + phi_halo;
}

// Flattened logarithmic halo, Eq. loghalo: Phi = (v_c^2/2) ln(R_c^2 + R^2 + z^2/q^2);
// theta = (v_c, R_c, q).
template <class T>
T phi_loghalo(const T x[3], const T* p) {
  T R2 = x[0] * x[0] + x[1] * x[1];
  T z2 = x[2] * x[2];
  return 0.5 * p[0] * p[0] * log(p[1] * p[1] + R2 + z2 / (p[2] * p[2]));
}

template <class T>
T potential(int sys, const T x[3], const T* p) {
  if (sys == S_ISOCHRONE) return phi_isochrone(x, p);
  if (sys == S_MW) return phi_mw(x, p);
  return phi_loghalo(x, p);
}

// dx/dt = v, dv/dt = -grad Phi (Eq. loghalo, first line). The gradient comes from one
// forward-mode pass over Phi with the three position components as seeds.
template <class T>
void rhs_orbit(int sys, const T* y, const T* p, int np, T* f) {
  typedef Dual<T, 3> D;
  D x[3];
  for (int i = 0; i < 3; i++) { x[i].v = y[i]; x[i].d[i] = 1.0; }
  D pd[4];
  for (int k = 0; k < np; k++) pd[k].v = p[k];
  D phi = potential(sys, x, pd);
  for (int i = 0; i < 3; i++) { f[i] = y[3 + i]; f[3 + i] = -phi.d[i]; }
}

// ---------------------------------------------------------------------------------------------
// Orbit-averaged spin precession in units G = c = M = 1, integrated in the orbital velocity v
// (Sec. 5, Eqs. prec-spins, prec-L, prec-omega, prec-rr). State y = (Lhat, S1hat, S2hat),
// theta = (q, chi1, chi2). The radiation-reaction coefficients b_k are not printed in the
// paper; here b_2, b_3, b_4 are the 2PN spin-orbit and spin-spin flux terms of Kidder (1995),
// the work the paper cites for these equations, and b_5..b_7 = 0. They are pinned by the 2PN
// energy balance -F / (dE/dv) of the published binding energy and flux (tests).
template <class T>
void cross3(const T a[3], const T b[3], T r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
template <class T>
T dot3(const T a[3], const T b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

template <class T>
void rhs_precession(const T& v, const T* y, const T* p, T* f) {
  const double pi = 3.14159265358979323846;
  T q = p[0], chi1 = p[1], chi2 = p[2];
  T m1 = 1.0 / (1.0 + q), m2 = q / (1.0 + q);
  T eta = m1 * m2;
  T S1 = chi1 * m1 * m1, S2 = chi2 * m2 * m2;
  T L = eta / v;  // Newtonian magnitude of the orbital angular momentum
  const T* Lh = y;
  const T* s1 = y + 3;
  const T* s2 = y + 6;
  T Lv[3], S1v[3], S2v[3];
  for (int i = 0; i < 3; i++) { Lv[i] = L * Lh[i]; S1v[i] = S1 * s1[i]; S2v[i] = S2 * s2[i]; }
  T v2 = v * v, v3 = v2 * v, v6 = v3 * v3;
  // Eq. prec-omega, and its 1 <-> 2, q -> 1/q image for the second spin
  T w1[3], w2[3];
  T a1[3], a2[3];
  for (int i = 0; i < 3; i++) { a1[i] = S2v[i] + q * S1v[i]; a2[i] = S1v[i] + S2v[i] / q; }
  T proj1 = dot3(Lh, a1), proj2 = dot3(Lh, a2);
  for (int i = 0; i < 3; i++) {
    w1[i] = 0.5 * v6 * ((4.0 + 3.0 * q) * Lv[i] + S2v[i] - 3.0 * proj1 * Lh[i]);
    w2[i] = 0.5 * v6 * ((4.0 + 3.0 / q) * Lv[i] + S1v[i] - 3.0 * proj2 * Lh[i]);
  }
  // Eq. prec-spins and Eq. prec-L (derivatives with respect to time)
  T ds1[3], ds2[3], dL[3];
  cross3(w1, s1, ds1);
  cross3(w2, s2, ds2);
  for (int i = 0; i < 3; i++) dL[i] = -(v / eta) * (S1 * ds1[i] + S2 * ds2[i]);
  // Eq. prec-rr with the 2PN coefficients
  T ls1 = dot3(Lh, s1), ls2 = dot3(Lh, s2), s1s2 = dot3(s1, s2);
  T b2 = -(743.0 + 924.0 * eta) / 336.0;
  T beta = (chi1 * ls1 * (113.0 * m1 * m1 + 75.0 * eta) + chi2 * ls2 * (113.0 * m2 * m2 + 75.0 * eta)) / 12.0;
  T b3 = 4.0 * pi - beta;
  T b4 = 34103.0 / 18144.0 + 13661.0 * eta / 2016.0 + 59.0 * eta * eta / 18.0 -
         (eta / 48.0) * chi1 * chi2 * (247.0 * s1s2 - 721.0 * ls1 * ls2);
  T v9 = v6 * v3;
  T dvdt = (32.0 / 5.0) * eta * v9 * (1.0 + b2 * v2 + b3 * v3 + b4 * v2 * v2);
  // integrate in v: dy/dv = (dy/dt) / (dv/dt)
  for (int i = 0; i < 3; i++) {
    f[i] = dL[i] / dvdt;
    f[3 + i] = ds1[i] / dvdt;
    f[6 + i] = ds2[i] / dvdt;
  }
}

// ---------------------------------------------------------------------------------------------
// Thawing quintessence in e-folds N = ln a (Sec. 4.1, Eq. de-model; Appendix C, Eq. de-rhs).
// State y = (phi, u, I), theta = (a0, lambda, Omega_m, Omega_r). E^2 follows from the
// Friedmann equation at every evaluation.
template <class T>
T quint_E2(const T& N, const T* y, const T* p) {
  T vphi = p[0] * exp(-p[1] * y[0]);
  T num = p[2] * exp(-3.0 * N) + p[3] * exp(-4.0 * N) + vphi;
  return num / (1.0 - y[1] * y[1] / 6.0);
}

template <class T>
void rhs_quintessence(const T& N, const T* y, const T* p, T* f) {
  T u = y[1];
  T vphi = p[0] * exp(-p[1] * y[0]);
  T em3 = exp(-3.0 * N), em4 = exp(-4.0 * N);
  T E2 = (p[2] * em3 + p[3] * em4 + vphi) / (1.0 - u * u / 6.0);
  T dlnE = -(3.0 * p[2] * em3 + 4.0 * p[3] * em4) / (2.0 * E2) - u * u / 2.0;
  // v'(phi) = -lambda v(phi)
  f[0] = u;
  f[1] = -(3.0 + dlnE) * u + 3.0 * p[1] * vphi / E2;
  f[2] = exp(-N) / sqrt(E2);
}

// ---------------------------------------------------------------------------------------------
// Dahlquist's linear test equation y' = lambda y (d = 1, theta = lambda), the problem on which a
// Runge-Kutta step reduces to multiplication by its stability polynomial (Hairer & Wanner II,
// Sec. IV.2). Not one of the paper's systems: the tests use it to fix the error norm and the
// step-size controller of Appendix A (Eqs. errnorm, controller) against a closed form.
template <class T>
void rhs_linear(const T* y, const T* p, T* f) {
  f[0] = p[0] * y[0];
}

// ---------------------------------------------------------------------------------------------
template <class T>
void rhs(int sys, const T& t, const T* y, const T* p, T* f) {
  int d, np;
  dims(sys, &d, &np);
  if (sys == S_PRECESSION) rhs_precession(t, y, p, f);
  else if (sys == S_QUINTESSENCE) rhs_quintessence(t, y, p, f);
  else if (sys == S_LINEAR) rhs_linear(y, p, f);
  else rhs_orbit(sys, y, p, np, f);
}

}  // namespace orc
