// Profile-likelihood Gauss-Newton fits of the quintessence model to BAO and supernova data
// (Sec. 4.3, Appendix C, Eq. de-gn), many minimisations at once.
//
// Model. For (lambda, Om) the flat cosmology (a0 from Eq. de-flat, gs_solve_flat) is saved at n
// nodes uniform in x = ln(1+z), z = 0 first, with its derivative along the flat models (Eq.
// de-ift). At the nodes f_M = ln(D_M / z) (limit -ln E(0) at z = 0) and f_H = ln D_H, D in c/H0;
// the data redshifts are reached by a not-a-knot cubic spline in x of f_M and f_H.
//
// Data. BAO points D_V/r_d, D_M/r_d, D_H/r_d (r_d of Aubourg et al. 2015) with covariance
// C_b = L_b L_b^T; supernova magnitudes m = 5 log10((1+z) D_M c/H0 / 10 pc) + M with C_s = L_s L_s^T.
// Residuals are whitened, r = L^{-1}(model - data), the supernova part projected orthogonally to
// u = L_s^{-1} 1 (marginalising M), chi^2 = r^T r.
//
// Node space. The spline is linear in the node values, so with X = L_s^{-1} A_s (A_s the spline
// matrix at the supernova redshifts), P = I - u u^T / u^T u, e = L_s^{-1}(d - k) for each mock
// (k = 5 log10((1+z) z), the H0 and M offsets being constant and projected out):
//   chi^2_sn = mu^T Q mu - 2 b^T mu + c,   Q = X^T P X,  b = X^T P e,  c = e^T P e,
// with mu = (5 / ln 10) f_M at the nodes. Q (n x n) is shared by all fits, (b, c) belong to a mock;
// gs_profile_prepare computes them once, and each Gauss-Newton iteration costs O(n^2) per fit
// instead of a triangular solve over every supernova. The 13-or-so BAO points are whitened directly.
//
// Iteration (Eq. de-gn): psi = (Om, H0), J = dr/dpsi (Om column from dy/dOm along flat models,
// H0 column analytic), psi <- psi - (J^T J + mu diag J^T J)^{-1} J^T r, the step scaled into the
// trust region; the next flatness solve starts from a0 + (da0/dOm) dOm. After n_iter updates chi^2
// is recomputed at the returned parameters and the fit passes if |Delta chi^2| and the Gauss-Newton
// decrement g^T (J^T J)^{-1} g (g = J^T r) are below their limits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "gs.h"
#include "gs_internal.h"

namespace {

constexpr int kMaxNodes = 64;
constexpr double kC = 299792.458;  // km/s
constexpr double kRdA = 55.154, kRdNu = 72.3, kRdCb = 0.25351, kRdB = 0.12807;

size_t r256(size_t x) { return (x + 255) / 256 * 256; }
int pfail(int code, const char* msg) { return gs::set_error(code, msg); }

// ---- prepared data: offsets in the caller's buffer (scratch for the supernova solve last)
struct PrepLayout {
  size_t x, Ab, Wb, zb, kind, db, Q, b, c, scratch, total, fit_total;
};
PrepLayout prep_layout(long long n, long long nb, long long ns, long long nm) {
  PrepLayout L;
  L.x = 0;
  L.Ab = L.x + r256(n * 8);
  L.Wb = L.Ab + r256(nb * n * 8);
  L.zb = L.Wb + r256(nb * nb * 8);
  L.kind = L.zb + r256(nb * 8);
  L.db = L.kind + r256(nb * 4);
  L.Q = L.db + r256(nm * nb * 8);
  L.b = L.Q + r256(n * n * 8);
  L.c = L.b + r256(nm * n * 8);
  L.fit_total = L.c + r256(nm * 8);
  L.scratch = L.fit_total;
  L.total = L.scratch + r256(ns * (n + 1 + nm) * 8);
  return L;
}

// ---- not-a-knot cubic spline as a linear map from node values to second derivatives G [n x n]:
// rows 1..n-2 continuity of the first derivative, rows 0 and n-1 continuity of the third derivative
// at x_1 and x_{n-2}. One block: Gauss-Jordan elimination with partial pivoting on [K | R].
__global__ void k_spline_G(int n, const double* x, double* G, double* work) {
  // work: K [n x n] then R [n x n]
  double* K = work;
  double* R = work + n * n;
  const int t = threadIdx.x;
  for (int e = t; e < n * n; e += blockDim.x) { K[e] = 0.0; R[e] = 0.0; }
  __syncthreads();
  if (t == 0) {
    for (int i = 1; i < n - 1; i++) {
      const double h0 = x[i] - x[i - 1], h1 = x[i + 1] - x[i];
      K[i * n + i - 1] = h0;
      K[i * n + i] = 2.0 * (h0 + h1);
      K[i * n + i + 1] = h1;
      R[i * n + i - 1] = 6.0 / h0;
      R[i * n + i] = -6.0 / h0 - 6.0 / h1;
      R[i * n + i + 1] = 6.0 / h1;
    }
    const double a0 = x[1] - x[0], a1 = x[2] - x[1];
    K[0] = a1; K[1] = -(a0 + a1); K[2] = a0;
    const double c0 = x[n - 2] - x[n - 3], c1 = x[n - 1] - x[n - 2];
    K[(n - 1) * n + n - 3] = c1; K[(n - 1) * n + n - 2] = -(c0 + c1); K[(n - 1) * n + n - 1] = c0;
  }
  __syncthreads();
  __shared__ int piv;
  for (int col = 0; col < n; col++) {
    if (t == 0) {
      int p = col;
      double best = fabs(K[col * n + col]);
      for (int r = col + 1; r < n; r++)
        if (fabs(K[r * n + col]) > best) { best = fabs(K[r * n + col]); p = r; }
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != col)
      for (int j = t; j < n; j += blockDim.x) {
        double a = K[col * n + j]; K[col * n + j] = K[p * n + j]; K[p * n + j] = a;
        a = R[col * n + j]; R[col * n + j] = R[p * n + j]; R[p * n + j] = a;
      }
    __syncthreads();
    const double inv = 1.0 / K[col * n + col];
    __syncthreads();
    for (int j = t; j < n; j += blockDim.x) { K[col * n + j] *= inv; R[col * n + j] *= inv; }
    __syncthreads();
    for (int r = 0; r < n; r++) {
      if (r == col) continue;
      const double f = K[r * n + col];
      __syncthreads();
      for (int j = t; j < n; j += blockDim.x) {
        K[r * n + j] -= f * K[col * n + j];
        R[r * n + j] -= f * R[col * n + j];
      }
      __syncthreads();
    }
  }
  for (int e = t; e < n * n; e += blockDim.x) G[e] = R[e];
}

// spline weights of point z for every node value: out[k], k < n (x = ln(1+z); ends extrapolate)
__device__ void spline_row(int n, const double* x, const double* G, double z, double* out) {
  const double xx = log1p(z);
  int i = 0;
  while (i < n - 2 && xx > x[i + 1]) i++;
  const double h = x[i + 1] - x[i];
  const double A = (x[i + 1] - xx) / h, B = (xx - x[i]) / h;
  const double cA = (A * A * A - A) * h * h / 6.0, cB = (B * B * B - B) * h * h / 6.0;
  for (int k = 0; k < n; k++) out[k] = cA * G[i * n + k] + cB * G[(i + 1) * n + k];
  out[i] += A;
  out[i + 1] += B;
}

__global__ void k_bao_rows(int n, int nb, const double* x, const double* G, const double* zb, double* Ab) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  spline_row(n, x, G, zb[p], Ab + (long long)p * n);
}

// supernova right-hand sides, column-major over ns rows: [A_s (n columns) | 1 | d_m - k (nm columns)]
__global__ void k_sn_rhs(int n, int ns, int nm, const double* x, const double* G, const double* zs, const double* ds,
                         double* B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  double row[kMaxNodes];
  const double z = zs[i];
  spline_row(n, x, G, z, row);
  for (int k = 0; k < n; k++) B[(long long)k * ns + i] = row[k];
  B[(long long)n * ns + i] = 1.0;
  const double kz = 5.0 * log10((1.0 + z) * z);
  for (int m = 0; m < nm; m++) B[(long long)(n + 1 + m) * ns + i] = ds[(long long)m * ns + i] - kz;
}

// L y = b for one column per block (L lower triangular, row-major [ns x ns]); in place on b
__global__ void k_forward_subst(int ns, const double* L, double* B) {
  double* b = B + (long long)blockIdx.x * ns;
  __shared__ double yi;
  for (int i = 0; i < ns; i++) {
    if (threadIdx.x == 0) {
      yi = b[i] / L[(long long)i * ns + i];
      b[i] = yi;
    }
    __syncthreads();
    const double y = yi;
    for (int j = i + 1 + threadIdx.x; j < ns; j += blockDim.x) b[j] -= L[(long long)j * ns + i] * y;
    __syncthreads();
  }
}

__device__ double block_dot(const double* a, const double* b, int ns) {
  __shared__ double part[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s += a[i] * b[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  const double r = part[0];
  __syncthreads();
  return r;
}

// column inner products of the whitened supernova block Y = [X | u | e]: G[i][j] = Y_i . Y_j for the
// pairs needed (X-X, X-u, X-e, u-u, u-e, e-e), one block per pair; then Q, b, c (projection by u)
__global__ void k_sn_gram(int n, int ns, int nm, const double* Y, double* gram) {
  const int ncol = n + 1 + nm;
  const int pair = blockIdx.x;  // i <= j over columns, but only pairs with i < n + 1 or i == j
  int i = 0, j = 0, q = pair;
  // enumerate: all (i, j) with i <= j and (i <= n or i == j)
  for (i = 0; i < ncol; i++) {
    const int cnt = (i <= n) ? ncol - i : 1;
    if (q < cnt) { j = (i <= n) ? i + q : i; break; }
    q -= cnt;
  }
  const double v = block_dot(Y + (long long)i * ns, Y + (long long)j * ns, ns);
  if (threadIdx.x == 0) {
    gram[(long long)i * ncol + j] = v;
    gram[(long long)j * ncol + i] = v;
  }
}
long long gram_pairs(int n, int nm) {
  const long long ncol = n + 1 + nm;
  long long p = 0;
  for (long long i = 0; i < ncol; i++) p += (i <= n) ? ncol - i : 1;
  return p;
}

__global__ void k_sn_project(int n, int nm, const double* gram, double* Q, double* b, double* c) {
  const int ncol = n + 1 + nm;
  const double uu = gram[(long long)n * ncol + n];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * n) {
    const int i = t / n, j = t % n;
    Q[t] = gram[(long long)i * ncol + j] - gram[(long long)i * ncol + n] * gram[(long long)j * ncol + n] / uu;
  }
  if (t < nm * n) {
    const int m = t / n, i = t % n;
    const int e = n + 1 + m;
    b[t] = gram[(long long)i * ncol + e] - gram[(long long)i * ncol + n] * gram[(long long)n * ncol + e] / uu;
  }
  if (t < nm) {
    const int e = n + 1 + t;
    c[t] = gram[(long long)e * ncol + e] - gram[(long long)n * ncol + e] * gram[(long long)n * ncol + e] / uu;
  }
}

// BAO whitening matrix W = L_b^{-1} (one thread, nb is small)
__global__ void k_bao_invert(int nb, const double* Lb, double* Wb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int col = 0; col < nb; col++)
    for (int i = 0; i < nb; i++) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; k++) s -= Lb[i * nb + k] * Wb[k * nb + col];
      Wb[i * nb + col] = s / Lb[i * nb + i];
    }
}

__global__ void k_copy(long long n, const double* src, double* dst) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}
__global__ void k_copy_i(long long n, const int32_t* src, int32_t* dst) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}
__global__ void k_log1p(int n, const double* z, double* x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = log1p(z[i]);
}

// ---- per-iteration kernels
struct FitArrays {
  long long nfit;
  int n, nb, nm;
  const double* lam;
  const int32_t* mock;
  const double* x;   // nodes, z = 0 first
  const double* Ab;  // [nb x n]
  const double* Wb;  // [nb x nb]
  const double* zb;
  const int32_t* kind;
  const double* db;  // [nm x nb]
  const double* Q;   // [n x n]
  const double* b;   // [nm x n]
  const double* c;   // [nm]
  const double* y;      // [nfit x n x 3] solver outputs, e-folds ascending (z descending)
  const double* dy;     // [nfit x n x 3] dy/dOm along flat models
  const double* da0;    // [nfit]
  const int32_t* st;    // solver status
  double *om, *H0, *a0, *chi2, *dec, *chi2_prev;
  int32_t* conv;
  int32_t* status;
  double* params;    // [nfit x 4] next solve's parameters
  double orad, omega_b, omega_nu, mu, trust_om, trust_h0, conv_dchi2, conv_dec;
};

__global__ void k_fit_init(FitArrays F, double om0, double h0) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= F.nfit) return;
  F.om[n] = om0;
  F.H0[n] = h0;
  F.a0[n] = 1.0 - om0 - F.orad;
  F.chi2_prev[n] = __longlong_as_double(0x7ff8000000000000LL);
  F.conv[n] = 0;
  F.status[n] = 0;
  double* p = F.params + n * 4;
  p[0] = F.a0[n]; p[1] = F.lam[n]; p[2] = om0; p[3] = F.orad;
}

__global__ void k_fit_step(FitArrays F, int final_iter) {
  __shared__ double Qs[kMaxNodes * kMaxNodes];
  const int n = F.n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Qs[e] = F.Q[e];
  __syncthreads();
  const long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (f >= F.nfit) return;
  const double nanv = __longlong_as_double(0x7ff8000000000000LL);
  const int32_t sst = F.st[f];
  const int m = F.mock[f];
  if (m < 0 || m >= F.nm) F.status[f] |= GS_ST_NONFINITE;  // no such mock data set
  if (sst != 0 || F.status[f] != 0) {  // a flatness solve failed: the fit stops with NaN results
    F.status[f] |= sst;
    F.chi2[f] = nanv; F.dec[f] = nanv; F.conv[f] = 0;
    return;
  }
  const double lam = F.lam[f], om = F.om[f], H0 = F.H0[f];
  const double a0 = F.params[f * 4], da0 = F.da0[f], orad = F.orad;  // flat a0 from the solve
  const double* Y = F.y + f * (long long)n * 3;
  const double* DY = F.dy + f * (long long)n * 3;
  double fM[kMaxNodes], fH[kMaxNodes], dM[kMaxNodes], dH[kMaxNodes];
  const double I0 = Y[(n - 1) * 3 + 2], dI0 = DY[(n - 1) * 3 + 2];
  for (int j = 0; j < n; j++) {
    const int k = n - 1 - j;  // solver output of node j
    const double N = -F.x[j];
    const double phi = Y[k * 3], u = Y[k * 3 + 1], I = Y[k * 3 + 2];
    const double den = 1.0 - u * u / 6.0;
    const double ev = exp(-lam * phi), e3 = exp(-3.0 * N), e4 = exp(-4.0 * N);
    const double num = om * e3 + orad * e4 + a0 * ev;
    const double E2 = num / den;
    const double dE2 = e3 / den + ev / den * da0 - lam * a0 * ev / den * DY[k * 3] + num * (u / 3.0) / (den * den) * DY[k * 3 + 1];
    fH[j] = -0.5 * log(E2);
    dH[j] = -0.5 * dE2 / E2;
    if (j == 0) {
      fM[0] = fH[0];
      dM[0] = dH[0];
    } else {
      const double DM = I0 - I;
      fM[j] = log(DM / expm1(F.x[j]));
      dM[j] = (dI0 - DY[k * 3 + 2]) / DM;
    }
  }
  // supernovae in node space (the H0 and M offsets are projected out)
  const double c5 = 5.0 / log(10.0);
  const double* bm = F.b + (long long)m * n;
  double muQmu = 0.0, dQmu = 0.0, dQd = 0.0, bmu = 0.0, bd = 0.0;
  for (int i = 0; i < n; i++) {
    double t = 0.0, s = 0.0;
    for (int j = 0; j < n; j++) {
      const double q = Qs[i * n + j];
      t += q * fM[j];
      s += q * dM[j];
    }
    muQmu += fM[i] * t;
    dQmu += dM[i] * t;
    dQd += dM[i] * s;
    bmu += bm[i] * fM[i];
    bd += bm[i] * dM[i];
  }
  double chi2 = c5 * c5 * muQmu - 2.0 * c5 * bmu + F.c[m];
  double g0 = c5 * c5 * dQmu - c5 * bd, g1 = 0.0;
  double j00 = c5 * c5 * dQd, j01 = 0.0, j11 = 0.0;
  // BAO points, whitened directly
  const double h = H0 / 100.0;
  const double wcb = om * h * h - F.omega_nu;
  const double rd = kRdA * exp(-kRdNu * (F.omega_nu + 0.0006) * (F.omega_nu + 0.0006)) /
                    (pow(wcb, kRdCb) * pow(F.omega_b, kRdB));
  const double drd_om = -kRdCb * h * h / wcb, drd_h = -kRdCb * 2.0 * om * h * h / (wcb * H0);
  double v[32], J0[32], J1[32];
  const int nb = F.nb;
  for (int p = 0; p < nb; p++) {
    const double* A = F.Ab + (long long)p * n;
    double lnDM = log(F.zb[p]), lnDH = 0.0, dlnDM = 0.0, dlnDH = 0.0;
    for (int j = 0; j < n; j++) {
      lnDM += A[j] * fM[j];
      lnDH += A[j] * fH[j];
      dlnDM += A[j] * dM[j];
      dlnDH += A[j] * dH[j];
    }
    const int kd = F.kind[p];
    const double lnX = kd == 0 ? (log(F.zb[p]) + 2.0 * lnDM + lnDH) / 3.0 : (kd == 1 ? lnDM : lnDH);
    const double dlnX = kd == 0 ? (2.0 * dlnDM + dlnDH) / 3.0 : (kd == 1 ? dlnDM : dlnDH);
    const double o = kC / H0 * exp(lnX) / rd;
    v[p] = o - F.db[(long long)m * nb + p];
    J0[p] = o * (dlnX - drd_om);
    J1[p] = o * (-1.0 / H0 - drd_h);
  }
  for (int i = 0; i < nb; i++) {
    double r = 0.0, a = 0.0, bb = 0.0;
    for (int k = 0; k <= i; k++) {
      const double w = F.Wb[i * nb + k];
      r += w * v[k];
      a += w * J0[k];
      bb += w * J1[k];
    }
    chi2 += r * r;
    g0 += a * r;
    g1 += bb * r;
    j00 += a * a;
    j01 += a * bb;
    j11 += bb * bb;
  }
  const double det = j00 * j11 - j01 * j01;
  const double decr = (j11 * g0 * g0 - 2.0 * j01 * g0 * g1 + j00 * g1 * g1) / det;
  F.chi2[f] = chi2;
  F.dec[f] = decr;
  if (final_iter) {
    F.conv[f] = (fabs(chi2 - F.chi2_prev[f]) < F.conv_dchi2 && decr < F.conv_dec) ? 1 : 0;
    F.a0[f] = a0;
    return;
  }
  // damped Gauss-Newton step (Eq. de-gn) in the trust region
  const double m00 = j00 * (1.0 + F.mu), m11 = j11 * (1.0 + F.mu);
  const double dm = m00 * m11 - j01 * j01;
  double s0 = -(m11 * g0 - j01 * g1) / dm, s1 = -(m00 * g1 - j01 * g0) / dm;
  double sc = 1.0;
  if (fabs(s0) * sc > F.trust_om) sc = F.trust_om / fabs(s0);
  if (fabs(s1) * sc > F.trust_h0) sc = F.trust_h0 / fabs(s1);
  s0 *= sc;
  s1 *= sc;
  F.chi2_prev[f] = chi2;
  F.om[f] = om + s0;
  F.H0[f] = H0 + s1;
  F.a0[f] = a0 + da0 * s0;
  double* pp = F.params + f * 4;
  pp[0] = F.a0[f]; pp[1] = lam; pp[2] = F.om[f]; pp[3] = orad;
}

__global__ void k_fit_setup(long long nfit, int n, const double* x, double* saveat, double* t0, double* t1, double* y0) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) saveat[i] = -x[n - 1 - i];  // e-folds ascending: today last
  if (i < nfit) {
    t0[i] = -log(51.0);
    t1[i] = 0.0;
    y0[i * 3] = 0.0; y0[i * 3 + 1] = 0.0; y0[i * 3 + 2] = 0.0;
  }
}

struct FitLayout {
  size_t saveat, t0, t1, y0, params, y, dy, da0, g, st, nacc, nrej, nnew, om_prev, flat, total;
};
FitLayout fit_layout(long long nfit, int n) {
  FitLayout L;
  L.saveat = 0;
  L.t0 = r256(n * 8);
  L.t1 = L.t0 + r256(nfit * 8);
  L.y0 = L.t1 + r256(nfit * 8);
  L.params = L.y0 + r256(nfit * 3 * 8);
  L.y = L.params + r256(nfit * 4 * 8);
  L.dy = L.y + r256(nfit * n * 3 * 8);
  L.da0 = L.dy + r256(nfit * n * 3 * 8);
  L.g = L.da0 + r256(nfit * 8);
  L.st = L.g + r256(nfit * 8);
  L.nacc = L.st + r256(nfit * 4);
  L.nrej = L.nacc + r256(nfit * 4);
  L.nnew = L.nrej + r256(nfit * 4);
  L.om_prev = L.nnew + r256(nfit * 4);
  L.flat = L.om_prev + r256(nfit * 8);
  L.total = L.flat + gs_flat_workspace_bytes(nfit, n);
  return L;
}

}  // namespace

extern "C" {

void gs_profile_default_options(gs_profile_options* o) {
  if (!o) return;
  o->method = GS_TSIT5;
  o->precision = GS_FP64;
  o->rtol = 1e-8;
  o->atol = 1e-11;
  o->gtol = 1e-10;
  o->max_newton = 8;
  o->n_iter = 20;
  o->mu = 1e-3;
  o->trust_om = 0.02;
  o->trust_h0 = 2.0;
  o->start_om = 0.30;
  o->start_h0 = 70.0;
  o->orad = 9e-5;
  o->omega_b = 0.02218;
  o->omega_nu = 0.00064;
  o->conv_dchi2 = 1e-4;
  o->conv_decrement = 1e-6;
  o->graph_safe = 0;
  o->sm_limit = 0;
}

size_t gs_profile_prep_bytes(int32_t n_nodes, int32_t n_bao, int32_t n_sn, int32_t n_mocks) {
  if (n_nodes < 4 || n_nodes > kMaxNodes || n_bao < 0 || n_bao > 32 || n_sn < 2 || n_mocks < 1) return 0;
  return prep_layout(n_nodes, n_bao, n_sn, n_mocks).total + r256(2 * size_t(n_nodes) * n_nodes * 8) +
         r256(size_t(n_nodes) * n_nodes * 8) + r256(size_t(n_nodes + 1 + n_mocks) * (n_nodes + 1 + n_mocks) * 8);
}

int gs_profile_prepare(int32_t n_nodes, const double* z_nodes, int32_t n_bao, const double* bao_z,
                       const int32_t* bao_kind, const double* L_bao, int32_t n_sn, const double* z_sn,
                       const double* L_sn, int32_t n_mocks, const double* d_bao, const double* d_sn, void* prep,
                       size_t prep_bytes, void* cuda_stream) {
  const size_t need = gs_profile_prep_bytes(n_nodes, n_bao, n_sn, n_mocks);
  if (!need) return pfail(GS_ERR_INVALID, "gs_profile_prepare: need 4 <= n_nodes <= 64, 0 <= n_bao <= 32, n_sn >= 2, n_mocks >= 1");
  if (!z_nodes || !z_sn || !L_sn || !d_sn || (n_bao > 0 && (!bao_z || !bao_kind || !L_bao || !d_bao)))
    return pfail(GS_ERR_INVALID, "gs_profile_prepare: NULL data pointer");
  if (!prep || reinterpret_cast<uintptr_t>(prep) % 256 != 0 || prep_bytes < need)
    return pfail(GS_ERR_WORKSPACE, "gs_profile_prepare: prep buffer must be 256-byte aligned and gs_profile_prep_bytes long");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = static_cast<unsigned char*>(prep);
  const PrepLayout L = prep_layout(n_nodes, n_bao, n_sn, n_mocks);
  const int n = n_nodes;
  double* x = reinterpret_cast<double*>(base + L.x);
  // after the prepared arrays: G [n x n], the elimination's K and R (2 n^2), the Gram matrix
  double* G = reinterpret_cast<double*>(base + L.total);
  const size_t gw_off = L.total + r256(size_t(n) * n * 8);
  double* gwork = reinterpret_cast<double*>(base + gw_off);
  double* gram = reinterpret_cast<double*>(base + gw_off + r256(2 * size_t(n) * n * 8));
  double* Y = reinterpret_cast<double*>(base + L.scratch);
  k_log1p<<<1, 64, 0, s>>>(n, z_nodes, x);
  k_spline_G<<<1, 128, 0, s>>>(n, x, G, gwork);
  if (n_bao > 0) {
    k_copy<<<1, 64, 0, s>>>(n_bao, bao_z, reinterpret_cast<double*>(base + L.zb));
    k_copy_i<<<1, 64, 0, s>>>(n_bao, bao_kind, reinterpret_cast<int32_t*>(base + L.kind));
    k_copy<<<unsigned((size_t(n_mocks) * n_bao + 255) / 256), 256, 0, s>>>((long long)n_mocks * n_bao, d_bao,
                                                                           reinterpret_cast<double*>(base + L.db));
    k_bao_rows<<<1, 64, 0, s>>>(n, n_bao, x, G, bao_z, reinterpret_cast<double*>(base + L.Ab));
    k_bao_invert<<<1, 32, 0, s>>>(n_bao, L_bao, reinterpret_cast<double*>(base + L.Wb));
  }
  k_sn_rhs<<<unsigned((n_sn + 127) / 128), 128, 0, s>>>(n, n_sn, n_mocks, x, G, z_sn, d_sn, Y);
  k_forward_subst<<<unsigned(n + 1 + n_mocks), 256, 0, s>>>(n_sn, L_sn, Y);
  k_sn_gram<<<unsigned(gram_pairs(n, n_mocks)), 256, 0, s>>>(n, n_sn, n_mocks, Y, gram);
  const long long work = (long long)n * n > (long long)n_mocks * n ? (long long)n * n : (long long)n_mocks * n;
  k_sn_project<<<unsigned((work + 255) / 256), 256, 0, s>>>(n, n_mocks, gram, reinterpret_cast<double*>(base + L.Q),
                                                             reinterpret_cast<double*>(base + L.b),
                                                             reinterpret_cast<double*>(base + L.c));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfail(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}

size_t gs_profile_workspace_bytes(int64_t n_fits, int32_t n_nodes) {
  if (n_fits < 0 || n_nodes < 4 || n_nodes > kMaxNodes) return 0;
  return fit_layout(n_fits, n_nodes).total;
}

int gs_profile_fit(int64_t n_fits, const double* lam, const int32_t* mock, const void* prep, int32_t n_nodes,
                   int32_t n_bao, int32_t n_sn, int32_t n_mocks, const gs_profile_options* opt, double* om, double* H0,
                   double* a0, double* chi2, double* decrement, int32_t* converged, int32_t* status, void* workspace,
                   size_t workspace_bytes, void* cuda_stream) {
  if (!opt) return pfail(GS_ERR_INVALID, "gs_profile_fit: opt is NULL");
  if (!gs_profile_prep_bytes(n_nodes, n_bao, n_sn, n_mocks))
    return pfail(GS_ERR_INVALID, "gs_profile_fit: bad data dimensions");
  if (n_fits < 0) return pfail(GS_ERR_INVALID, "gs_profile_fit: n_fits < 0");
  if (opt->n_iter < 0) return pfail(GS_ERR_INVALID, "gs_profile_fit: n_iter < 0");
  if (n_fits == 0) return GS_OK;
  if (!lam || !mock || !prep || !om || !H0 || !a0 || !chi2 || !decrement || !converged || !status)
    return pfail(GS_ERR_INVALID, "gs_profile_fit: NULL pointer");
  const FitLayout W = fit_layout(n_fits, n_nodes);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 != 0 || workspace_bytes < W.total)
    return pfail(GS_ERR_WORKSPACE, "gs_profile_fit: workspace must be 256-byte aligned and gs_profile_workspace_bytes long");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const unsigned char* pb = static_cast<const unsigned char*>(prep);
  const PrepLayout P = prep_layout(n_nodes, n_bao, n_sn, n_mocks);
  FitArrays F;
  F.nfit = n_fits; F.n = n_nodes; F.nb = n_bao; F.nm = n_mocks;
  F.lam = lam; F.mock = mock;
  F.x = reinterpret_cast<const double*>(pb + P.x);
  F.Ab = reinterpret_cast<const double*>(pb + P.Ab);
  F.Wb = reinterpret_cast<const double*>(pb + P.Wb);
  F.zb = reinterpret_cast<const double*>(pb + P.zb);
  F.kind = reinterpret_cast<const int32_t*>(pb + P.kind);
  F.db = reinterpret_cast<const double*>(pb + P.db);
  F.Q = reinterpret_cast<const double*>(pb + P.Q);
  F.b = reinterpret_cast<const double*>(pb + P.b);
  F.c = reinterpret_cast<const double*>(pb + P.c);
  double* saveat = reinterpret_cast<double*>(ws + W.saveat);
  double* t0 = reinterpret_cast<double*>(ws + W.t0);
  double* t1 = reinterpret_cast<double*>(ws + W.t1);
  double* y0 = reinterpret_cast<double*>(ws + W.y0);
  F.params = reinterpret_cast<double*>(ws + W.params);
  double* y = reinterpret_cast<double*>(ws + W.y);
  double* dy = reinterpret_cast<double*>(ws + W.dy);
  double* da0 = reinterpret_cast<double*>(ws + W.da0);
  int32_t* st = reinterpret_cast<int32_t*>(ws + W.st);
  F.y = y; F.dy = dy; F.da0 = da0; F.st = st;
  F.om = om; F.H0 = H0; F.a0 = a0; F.chi2 = chi2; F.dec = decrement;
  F.chi2_prev = reinterpret_cast<double*>(ws + W.om_prev);
  F.conv = converged; F.status = status;
  F.orad = opt->orad; F.omega_b = opt->omega_b; F.omega_nu = opt->omega_nu; F.mu = opt->mu;
  F.trust_om = opt->trust_om; F.trust_h0 = opt->trust_h0;
  F.conv_dchi2 = opt->conv_dchi2; F.conv_dec = opt->conv_decrement;
  const int block = 128;
  const unsigned grid = unsigned((n_fits + block - 1) / block);
  const long long nset = n_fits > n_nodes ? n_fits : n_nodes;
  k_fit_setup<<<unsigned((nset + 255) / 256), 256, 0, s>>>((long long)n_fits, n_nodes, F.x, saveat, t0, t1, y0);
  k_fit_init<<<grid, block, 0, s>>>(F, opt->start_om, opt->start_h0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pfail(GS_ERR_CUDA, cudaGetErrorString(e));
  gs_options fo;
  gs_default_options(&fo);
  fo.method = opt->method;
  fo.precision = opt->precision;
  fo.kernel = GS_KERNEL_PERSISTENT;
  fo.graph_safe = opt->graph_safe;
  fo.sm_limit = opt->sm_limit;
  for (int it = 0; it <= opt->n_iter; it++) {
    // the flat model at the current (lambda, Om), Newton on a0 from the moved amplitude; the
    // solver's params hold the flat a0 afterwards
    int rc = gs_solve_flat(n_fits, y0, F.params, t0, t1, opt->rtol, opt->atol, n_nodes, saveat, &fo, opt->max_newton,
                           opt->gtol, y, dy, da0, reinterpret_cast<double*>(ws + W.g), st,
                           reinterpret_cast<int32_t*>(ws + W.nacc), reinterpret_cast<int32_t*>(ws + W.nrej),
                           reinterpret_cast<int32_t*>(ws + W.nnew), ws + W.flat, workspace_bytes - W.flat, cuda_stream);
    if (rc) return rc;
    k_fit_step<<<grid, block, 0, s>>>(F, it == opt->n_iter ? 1 : 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(GS_ERR_CUDA, cudaGetErrorString(e));
  }
  return GS_OK;
}

}  // extern "C"
