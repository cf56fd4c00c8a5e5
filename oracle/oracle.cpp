// Oracle (test infrastructure only): a plain, slow FP64 CPU restatement of the paper's adaptive
// explicit Runge-Kutta integration of an ensemble of independent initial-value problems.
// It is used by the test suite, by the smoke check and by the CPU-baseline leg of the benchmark,
// never by the product path. It shares no code with the GPU library.
//
// What it follows, step by step (paper section / equation):
//   ensemble problem ............ Sec. 2.1, Eq. ivp
//   Runge-Kutta step ............ Appendix A, Eq. rk
//   scaled RMS error norm ....... Appendix A, Eq. errnorm (max of |y| and |y+| in the scale)
//   step-size controller ........ Appendix A, Eq. controller, (alpha_min, alpha_max) = (0.2, 5),
//                                 the same rule after accepted and rejected attempts; the PI form
//                                 h*clamp(safety*err^-beta1*err_prev^beta2) reduces to it for
//                                 (beta1, beta2) = (1/nu, 0), the default
//   step attempts N_i ........... Sec. 2.2 (accepted + rejected attempts)
//   dense output ................ Appendix A, Eq. dense (Tsit5 / Dopri5 polynomials; Verner 7
//                                 re-runs a shortened step from the start of the step)
//   forward sensitivities ....... Sec. 2.3, Eq. sens; Appendix A, Eq. stage-sens: the step run on
//                                 dual numbers with h held fixed, so S is the exact derivative of
//                                 the discrete solution on the step sequence taken
//   chain rule .................. Appendix A, Eq. chain (per trajectory, no sum over members)
// Where the paper is silent (initial step, last step, failure handling) the readings are:
//   initial step: the starting-step algorithm of Hairer, Norsett & Wanner I, Sec. II.4, with
//     exponent 1/(nu+1); last step: clipped to land exactly on t1 when h(1+4 eps) >= t1 - t;
//     the time is advanced with compensated (Kahan) summation; h underflow when
//     h < 16 eps max(|t|, |t1|); at most max_steps attempts; a failed trajectory returns NaN.
//
// Parity pins: the tableaux are checked against the Butcher order conditions and measured
// convergence orders; whole solves against isochrone closed forms, conserved quantities of
// every system, and Lambda-CDM distances by quadrature; the forward sensitivities against
// central finite differences of the fixed-step replay; the starting step against SciPy's
// implementation of the same published algorithm; the precession radiation reaction against the
// 2PN energy balance.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "dual.hpp"
#include "systems.hpp"
#include "tableaux.hpp"

namespace orc {

enum { ST_MAX_STEPS = 1, ST_H_UNDERFLOW = 2, ST_NONFINITE = 4, ST_EMPTY_INTERVAL = 8,
       ST_SAVEAT_OUTSIDE = 16 };

struct Opts {
  int method;
  int max_steps;
  double safety, alpha_min, alpha_max, beta1, beta2, h0;
};

static const double kNaN = std::numeric_limits<double>::quiet_NaN();

template <class T> inline void set_nan(T& x) { x = T(kNaN); }

inline double rms_scaled(int d, const double* v, const double* sc) {
  double acc = 0.0;
  for (int i = 0; i < d; i++) { double r = v[i] / sc[i]; acc += r * r; }
  return std::sqrt(acc / d);
}

// Starting step size, Hairer, Norsett & Wanner I, Sec. II.4 (value parts only).
inline double initial_step(int sys, int nu, double t0, double t1, const double* y0, const double* p,
                           const double* f0, double rtol, double atol, int d) {
  double sc[9], tmp[9], y1[9], f1[9];
  for (int i = 0; i < d; i++) sc[i] = atol + rtol * std::fabs(y0[i]);
  double d0 = rms_scaled(d, y0, sc);
  double d1 = rms_scaled(d, f0, sc);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * (d0 / d1);
  if (h0 > t1 - t0) h0 = t1 - t0;
  for (int i = 0; i < d; i++) y1[i] = y0[i] + h0 * f0[i];
  rhs<double>(sys, t0 + h0, y1, p, f1);
  for (int i = 0; i < d; i++) tmp[i] = f1[i] - f0[i];
  double d2 = rms_scaled(d, tmp, sc) / h0;
  double dm = d1 > d2 ? d1 : d2;
  double h1 = (dm <= 1e-15) ? (h0 * 1e-3 > 1e-6 ? h0 * 1e-3 : 1e-6) : std::pow(0.01 / dm, 1.0 / (nu + 1));
  double h = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
  if (h > t1 - t0) h = t1 - t0;
  return h;
}

// Stages of one explicit Runge-Kutta step of length h from (t, y), Eq. rk.
// k[0] must hold f(t, y) on entry. Fills k[1..nst-1] and Y for the last stage computed.
template <class T>
void stages(int sys, const Tableau& tab, int nst, double t, const T* y, const T* p, double h, int d,
            T k[][9]) {
  T Y[9];
  for (int j = 1; j < nst; j++) {
    for (int i = 0; i < d; i++) {
      T acc = T(0.0);
      for (int l = 0; l < j; l++)
        if (tab.A[j][l] != 0.0) acc = acc + tab.A[j][l] * k[l][i];
      Y[i] = y[i] + h * acc;
    }
    rhs<T>(sys, T(t + tab.c[j] * h), Y, p, k[j]);
  }
}

// Solution at a point inside an accepted step: Eq. dense for Tsit5 / Dopri5, the shortened
// step of Appendix A for Verner 7. sig in [0, 1].
template <class T>
void dense_point(int sys, int method, const Tableau& tab, double t, const T* y, const T* p, double h,
                 double sig, int d, T k[][9], T* out) {
  if (method == M_VERN7) {
    T kk[10][9];
    for (int i = 0; i < d; i++) kk[0][i] = k[0][i];
    double hs = sig * h;
    stages(sys, tab, 9, t, y, p, hs, d, kk);  // stage 10 has b_10 = 0
    for (int i = 0; i < d; i++) {
      T acc = T(0.0);
      for (int j = 0; j < 9; j++)
        if (tab.b[j] != 0.0) acc = acc + tab.b[j] * kk[j][i];
      out[i] = y[i] + hs * acc;
    }
    return;
  }
  double w[10];
  dense_weights(method, sig, w);
  for (int i = 0; i < d; i++) {
    T acc = T(0.0);
    for (int j = 0; j < tab.s; j++) acc = acc + w[j] * k[j][i];
    out[i] = y[i] + h * acc;
  }
}

// Integrate one trajectory. Modes: adaptive (tape_in == nullptr), optionally recording the
// accepted step sizes; or replay of a recorded sequence of step sizes (tape_in != nullptr).
template <class T>
void integrate(int sys, const Opts& o, const T* y0, const T* p, double t0, double t1, double rtol,
               double atol, int K, const double* save, T* yout, int* status, int* nacc, int* nrej,
               double* tape_out, int tape_cap, int* ntape, const double* tape_in, int ntape_in) {
  int d, np;
  dims(sys, &d, &np);
  const Tableau tab = get_tableau(o.method);
  const int s = tab.s;
  const int nu = tab.order;
  *status = 0; *nacc = 0; *nrej = 0;
  if (ntape) *ntape = 0;

  bool fin = std::isfinite(t0) && std::isfinite(t1);
  for (int i = 0; i < d; i++) fin = fin && std::isfinite(val(y0[i]));
  for (int k = 0; k < np; k++) fin = fin && std::isfinite(val(p[k]));
  if (!fin) {
    *status = ST_NONFINITE;
    for (int k = 0; k < K * d; k++) set_nan(yout[k]);
    return;
  }
  if (!(t1 > t0)) {  // empty (or reversed) interval: the state stays y0
    *status = ST_EMPTY_INTERVAL;
    for (int k = 0; k < K; k++)
      for (int i = 0; i < d; i++) yout[k * d + i] = y0[i];
    return;
  }
  // saveat validity: inside [t0, t1] and non-decreasing
  std::vector<char> valid(K > 0 ? K : 1, 0);
  for (int k = 0; k < K; k++) {
    bool ok = (save[k] >= t0) && (save[k] <= t1) && (k == 0 || save[k] >= save[k - 1]);
    valid[k] = ok;
    if (!ok) {
      *status |= ST_SAVEAT_OUTSIDE;
      for (int i = 0; i < d; i++) set_nan(yout[k * d + i]);
    }
  }
  int kk = 0;
  while (kk < K && (!valid[kk] || save[kk] == t0)) {
    if (valid[kk])
      for (int i = 0; i < d; i++) yout[kk * d + i] = y0[i];
    kk++;
  }

  T y[9], ynew[9], k[10][9], e[9], dense[9];
  for (int i = 0; i < d; i++) y[i] = y0[i];
  rhs<T>(sys, T(t0), y, p, k[0]);

  double h;
  if (tape_in) {
    h = ntape_in > 0 ? tape_in[0] : (t1 - t0);
  } else if (o.h0 > 0.0) {
    h = o.h0 < t1 - t0 ? o.h0 : t1 - t0;
  } else {
    double yv[9], pv[4], fv[9];
    for (int i = 0; i < d; i++) { yv[i] = val(y[i]); fv[i] = val(k[0][i]); }
    for (int q = 0; q < np; q++) pv[q] = val(p[q]);
    h = initial_step(sys, nu, t0, t1, yv, pv, fv, rtol, atol, d);
  }
  const double beta1 = o.beta1 > 0.0 ? o.beta1 : 1.0 / nu;
  const double beta2 = o.beta2;
  double t = t0, tc = 0.0, err_prev = 1.0;
  bool failed = false, done = false;
  int nstep_replay = 0;

  while (!done) {
    double rem = (t1 - t) + tc;
    if (rem <= 0.0) { done = true; break; }
    bool last = false;
    if (tape_in) {
      if (nstep_replay >= ntape_in) { done = true; break; }
      h = tape_in[nstep_replay];
      if (nstep_replay == ntape_in - 1) { h = rem; last = true; }
    } else {
      if (*nacc + *nrej >= o.max_steps) { *status |= ST_MAX_STEPS; failed = true; break; }
      if (h * (1.0 + 4.0 * DBL_EPSILON) >= rem) {
        h = rem;
        last = true;
      } else {
        double tm = std::fabs(t) > std::fabs(t1) ? std::fabs(t) : std::fabs(t1);
        if (!(h >= 16.0 * DBL_EPSILON * tm)) {  // also catches a non-finite step size
          *status |= std::isnan(h) ? (ST_H_UNDERFLOW | ST_NONFINITE) : ST_H_UNDERFLOW;
          failed = true;
          break;
        }
      }
    }
    stages(sys, tab, s, t, y, p, h, d, k);
    // propagated solution; for FSAL pairs it is the last stage state itself
    for (int i = 0; i < d; i++) {
      T acc = T(0.0);
      for (int j = 0; j < s; j++)
        if (tab.b[j] != 0.0) acc = acc + tab.b[j] * k[j][i];
      ynew[i] = y[i] + h * acc;
    }
    if (tab.fsal) {
      // recompute exactly as the last stage state, so that k[s-1] = f(ynew) bit for bit
      for (int i = 0; i < d; i++) {
        T acc = T(0.0);
        for (int l = 0; l < s - 1; l++)
          if (tab.A[s - 1][l] != 0.0) acc = acc + tab.A[s - 1][l] * k[l][i];
        ynew[i] = y[i] + h * acc;
      }
    }
    bool accept;
    double err = 0.0;
    if (tape_in) {
      accept = true;
    } else {
      for (int i = 0; i < d; i++) {
        T acc = T(0.0);
        for (int j = 0; j < s; j++) {
          double bt = tab.b[j] - tab.bh[j];
          if (bt != 0.0) acc = acc + bt * k[j][i];
        }
        e[i] = h * acc;
      }
      double sq = 0.0;
      for (int i = 0; i < d; i++) {
        double a = std::fabs(val(y[i])), b = std::fabs(val(ynew[i]));
        double sc = atol + rtol * (a > b ? a : b);
        double r = val(e[i]) / sc;
        sq += r * r;
      }
      err = std::sqrt(sq / d);
      accept = (err <= 1.0);
    }
    if (accept) {
      *nacc += 1;
      if (tape_out && *nacc <= tape_cap) tape_out[*nacc - 1] = h;
      if (ntape) *ntape = *nacc;
      // dense output for saveat points in (t_n, t_n + h]
      while (kk < K) {
        if (!valid[kk]) { kk++; continue; }
        double dk = (save[kk] - t) + tc;
        if (last && save[kk] == t1) {
          for (int i = 0; i < d; i++) yout[kk * d + i] = ynew[i];
        } else if (last || dk <= h) {
          double sig = dk / h;
          if (sig > 1.0) sig = 1.0;
          if (sig < 0.0) sig = 0.0;
          dense_point(sys, o.method, tab, t, y, p, h, sig, d, k, dense);
          for (int i = 0; i < d; i++) yout[kk * d + i] = dense[i];
        } else {
          break;
        }
        kk++;
      }
      for (int i = 0; i < d; i++) y[i] = ynew[i];
      if (tab.fsal) {
        for (int i = 0; i < d; i++) k[0][i] = k[s - 1][i];
      }
      if (last) {
        t = t1; tc = 0.0; done = true;
      } else {
        double yk = h - tc;  // Kahan summation of the time
        double tn = t + yk;
        tc = (tn - t) - yk;
        t = tn;
        if (!tab.fsal) rhs<T>(sys, T(t), y, p, k[0]);
      }
      if (tape_in) {
        nstep_replay++;
      } else if (!done) {
        double fac = o.safety * std::pow(err, -beta1) * (beta2 != 0.0 ? std::pow(err_prev, beta2) : 1.0);
        if (fac > o.alpha_max) fac = o.alpha_max;
        if (fac < o.alpha_min) fac = o.alpha_min;
        h = h * fac;
        err_prev = err > 1e-4 ? err : 1e-4;
      }
    } else {
      *nrej += 1;
      double fac;
      if (std::isnan(err)) {
        fac = o.alpha_min;
      } else {
        fac = o.safety * std::pow(err, -beta1) * (beta2 != 0.0 ? std::pow(err_prev, beta2) : 1.0);
        if (fac > o.alpha_max) fac = o.alpha_max;
        if (fac < o.alpha_min) fac = o.alpha_min;
      }
      h = h * fac;
      err_prev = 1.0;
    }
  }
  if (done) {
    // points at t1 not yet emitted when the interval closed without a final step
    while (kk < K) {
      if (valid[kk]) for (int i = 0; i < d; i++) yout[kk * d + i] = y[i];
      kk++;
    }
  }
  if (failed) {
    for (int q = 0; q < K * d; q++) set_nan(yout[q]);
  }
}

// Forward sensitivities with respect to (y0, theta) on dual numbers of width M = d + p,
// contracted with per-output cotangents w (Eq. chain, one member). Outputs the solution,
// dL/dy0 and dL/dtheta.
template <int M>
void grad_one(int sys, const Opts& o, const double* y0, const double* p, double t0, double t1,
              double rtol, double atol, int K, const double* save, const double* w, double* yout,
              double* gy0, double* gp, int* status, int* nacc, int* nrej, const double* tape_in,
              int ntape_in) {
  typedef Dual<double, M> D;
  int d, np;
  dims(sys, &d, &np);
  D yd[9], pd[4];
  for (int i = 0; i < d; i++) { yd[i].v = y0[i]; yd[i].d[i] = 1.0; }
  for (int q = 0; q < np; q++) { pd[q].v = p[q]; pd[q].d[d + q] = 1.0; }
  std::vector<D> out(K * d > 0 ? K * d : 1);
  integrate<D>(sys, o, yd, pd, t0, t1, rtol, atol, K, save, out.data(), status, nacc, nrej, nullptr,
               0, nullptr, tape_in, ntape_in);
  for (int m = 0; m < d + np; m++) {
    double acc = 0.0;
    for (int q = 0; q < K * d; q++) acc += w[q] * out[q].d[m];
    if (m < d) gy0[m] = acc; else gp[m - d] = acc;
  }
  for (int q = 0; q < K * d; q++) yout[q] = out[q].v;
}

// The full forward-sensitivity matrix S[k][i][m] = d y_i(t_k) / d x_m, x = (y0, theta), on
// dual numbers of width M = d + p (Eq. sens, Eq. stage-sens), along the adaptive step sequence.
template <int M>
void sens_one(int sys, const Opts& o, const double* y0, const double* p, double t0, double t1, double rtol,
              double atol, int K, const double* save, double* yout, double* S, int* status, int* nacc,
              int* nrej) {
  typedef Dual<double, M> D;
  int d, np;
  dims(sys, &d, &np);
  D yd[9], pd[4];
  for (int i = 0; i < d; i++) { yd[i].v = y0[i]; yd[i].d[i] = 1.0; }
  for (int q = 0; q < np; q++) { pd[q].v = p[q]; pd[q].d[d + q] = 1.0; }
  std::vector<D> out(K * d > 0 ? K * d : 1);
  integrate<D>(sys, o, yd, pd, t0, t1, rtol, atol, K, save, out.data(), status, nacc, nrej, nullptr, 0,
               nullptr, nullptr, 0);
  for (int q = 0; q < K * d; q++) {
    yout[q] = out[q].v;
    for (int m = 0; m < M; m++) S[q * M + m] = out[q].d[m];
  }
}

}  // namespace orc

using namespace orc;

extern "C" {

typedef struct {
  int method;
  int max_steps;
  double safety, alpha_min, alpha_max, beta1, beta2, h0;
} orc_opts;

static Opts to_opts(const orc_opts* x) {
  Opts o;
  o.method = x->method; o.max_steps = x->max_steps; o.safety = x->safety;
  o.alpha_min = x->alpha_min; o.alpha_max = x->alpha_max; o.beta1 = x->beta1;
  o.beta2 = x->beta2; o.h0 = x->h0;
  return o;
}

int orc_dims(int sys, int* d, int* p) {
  dims(sys, d, p);
  return (*d > 0) ? 0 : 1;
}

int orc_tableau(int method, int* s, int* order, int* fsal, double* A, double* b, double* bh, double* c) {
  Tableau T = get_tableau(method);
  *s = T.s; *order = T.order; *fsal = T.fsal ? 1 : 0;
  for (int i = 0; i < T.s; i++) {
    for (int j = 0; j < T.s; j++) A[i * T.s + j] = T.A[i][j];
    b[i] = T.b[i]; bh[i] = T.bh[i]; c[i] = T.c[i];
  }
  return 0;
}

int orc_dense_weights(int method, double sigma, double* w) { return dense_weights(method, sigma, w) ? 0 : 1; }

int orc_rhs(int sys, double t, const double* y, const double* p, double* f) {
  rhs<double>(sys, t, y, p, f);
  return 0;
}

// The starting step every solve of `method` takes from (t0, y0) towards t1 (Hairer, Norsett &
// Wanner I, Sec. II.4, with p the method's order), exposed so that tests can compare it with an
// independent implementation of that algorithm.
double orc_initial_step(int sys, int method, double t0, double t1, const double* y0, const double* p, double rtol,
                        double atol) {
  int d, np;
  dims(sys, &d, &np);
  double f0[9];
  rhs<double>(sys, t0, y0, p, f0);
  return initial_step(sys, get_tableau(method).order, t0, t1, y0, p, f0, rtol, atol, d);
}

// J_y vy + J_theta vp at (t, y, theta), by one forward-mode pass.
int orc_jvp(int sys, double t, const double* y, const double* p, const double* vy, const double* vp, double* out) {
  int d, np;
  dims(sys, &d, &np);
  typedef Dual<double, 1> D;
  D yd[9], pd[4], fd[9];
  for (int i = 0; i < d; i++) { yd[i].v = y[i]; yd[i].d[0] = vy[i]; }
  for (int q = 0; q < np; q++) { pd[q].v = p[q]; pd[q].d[0] = vp ? vp[q] : 0.0; }
  rhs<D>(sys, D(t), yd, pd, fd);
  for (int i = 0; i < d; i++) out[i] = fd[i].d[0];
  return 0;
}

int orc_potential(int sys, const double* x, const double* p, double* phi) {
  *phi = potential<double>(sys, x, p);
  return 0;
}

// Adaptive ensemble solve. saveat is [K] shared, or [N, K] when per_traj != 0.
// If tape != nullptr the accepted step sizes are recorded into tape[N, tape_cap] and their
// count into ntape[N].
int orc_solve(int sys, const orc_opts* opt, long N, const double* y0, const double* params,
              const double* t0, const double* t1, double rtol, double atol, int K, const double* saveat,
              int per_traj, double* yout, int* status, int* nacc, int* nrej, double* tape, int tape_cap,
              int* ntape, int nthreads) {
  int d, np;
  dims(sys, &d, &np);
  Opts o = to_opts(opt);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
  for (long n = 0; n < N; n++) {
    const double* sv = per_traj ? saveat + n * K : saveat;
    integrate<double>(sys, o, y0 + n * d, np ? params + n * np : nullptr, t0[n], t1[n], rtol, atol, K,
                      sv, yout + n * K * d, status + n, nacc + n, nrej + n,
                      tape ? tape + n * (long)tape_cap : nullptr, tape_cap, ntape ? ntape + n : nullptr,
                      nullptr, 0);
  }
  return 0;
}

// Fixed-step replay of recorded step sizes tape[N, tape_cap] (ntape[n] steps for member n).
int orc_replay(int sys, const orc_opts* opt, long N, const double* y0, const double* params,
               const double* t0, const double* t1, int K, const double* saveat, int per_traj,
               const double* tape, int tape_cap, const int* ntape, double* yout, int nthreads) {
  int d, np;
  dims(sys, &d, &np);
  Opts o = to_opts(opt);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
  for (long n = 0; n < N; n++) {
    int st, na, nr;
    const double* sv = per_traj ? saveat + n * K : saveat;
    integrate<double>(sys, o, y0 + n * d, np ? params + n * np : nullptr, t0[n], t1[n], 0.0, 0.0, K, sv,
                      yout + n * K * d, &st, &na, &nr, nullptr, 0, nullptr, tape + n * (long)tape_cap,
                      ntape[n]);
  }
  return 0;
}

// Gradient of L = sum_k w_k . y(t_k) for each member by forward sensitivities, along the
// adaptive step sequence (tape == nullptr) or along recorded step sizes.
int orc_grad(int sys, const orc_opts* opt, long N, const double* y0, const double* params,
             const double* t0, const double* t1, double rtol, double atol, int K, const double* saveat,
             int per_traj, const double* w, double* yout, double* gy0, double* gp, int* status, int* nacc,
             int* nrej, const double* tape, int tape_cap, const int* ntape, int nthreads) {
  int d, np;
  dims(sys, &d, &np);
  Opts o = to_opts(opt);
  int M = d + np;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long n = 0; n < N; n++) {
    const double* sv = per_traj ? saveat + n * K : saveat;
    const double* yy = y0 + n * d;
    const double* pp = np ? params + n * np : nullptr;
    const double* ww = w + n * K * d;
    double* yo = yout + n * K * d;
    double* g1 = gy0 + n * d;
    double* g2 = np ? gp + n * np : nullptr;
    const double* tp = tape ? tape + n * (long)tape_cap : nullptr;
    int nt = tape ? ntape[n] : 0;
    switch (M) {
      case 6: grad_one<6>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, ww, yo, g1, g2, status + n, nacc + n, nrej + n, tp, nt); break;
      case 7: grad_one<7>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, ww, yo, g1, g2, status + n, nacc + n, nrej + n, tp, nt); break;
      case 9: grad_one<9>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, ww, yo, g1, g2, status + n, nacc + n, nrej + n, tp, nt); break;
      case 10: grad_one<10>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, ww, yo, g1, g2, status + n, nacc + n, nrej + n, tp, nt); break;
      case 12: grad_one<12>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, ww, yo, g1, g2, status + n, nacc + n, nrej + n, tp, nt); break;
      default: status[n] = -1;
    }
  }
  return 0;
}

// Solution and full sensitivity matrix S[N, K, d, d + p] (derivatives with respect to y0, then theta).
int orc_sens(int sys, const orc_opts* opt, long N, const double* y0, const double* params, const double* t0,
             const double* t1, double rtol, double atol, int K, const double* saveat, int per_traj, double* yout,
             double* S, int* status, int* nacc, int* nrej, int nthreads) {
  int d, np;
  dims(sys, &d, &np);
  Opts o = to_opts(opt);
  int M = d + np;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long n = 0; n < N; n++) {
    const double* sv = per_traj ? saveat + n * K : saveat;
    const double* yy = y0 + n * d;
    const double* pp = np ? params + n * np : nullptr;
    double* yo = yout + n * K * d;
    double* Sn = S + n * (long)K * d * M;
    switch (M) {
      case 6: sens_one<6>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, yo, Sn, status + n, nacc + n, nrej + n); break;
      case 7: sens_one<7>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, yo, Sn, status + n, nacc + n, nrej + n); break;
      case 9: sens_one<9>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, yo, Sn, status + n, nacc + n, nrej + n); break;
      case 10: sens_one<10>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, yo, Sn, status + n, nacc + n, nrej + n); break;
      case 12: sens_one<12>(sys, o, yy, pp, t0[n], t1[n], rtol, atol, K, sv, yo, Sn, status + n, nacc + n, nrej + n); break;
      default: status[n] = -1;
    }
  }
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
