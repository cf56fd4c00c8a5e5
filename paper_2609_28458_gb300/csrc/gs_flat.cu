// Spatial flatness of the quintessence cosmologies (Sec. 4.1, Eqs. de-flat and de-ift).
//
// A flat model has E(0) = 1:
//   g(a0) = (Om + Or + a0 exp(-lambda phi0)) / (1 - u0^2/6) - 1 = 0,
// where (phi0, u0) is the state today (N = 0, the end of the integration). Newton's method on a0:
// every iteration is one gs_jvp launch carrying two tangent directions, S_a0 = dy/da0 and
// S_Om = dy/dOm, followed by k_flat_newton, which forms
//   dg/da0 = (dg/dy) S_a0(0) + dg/da0|explicit,   dg/dOm = (dg/dy) S_Om(0) + dg/dOm|explicit,
// writes the derivative along the flat models (Eq. de-ift):
//   da0/dOm = -(dg/dOm) / (dg/da0),   dy/dOm = S_Om + (da0/dOm) S_a0   at every output,
// and takes the Newton step a0 <- a0 - g / (dg/da0) where |g| > gtol. A cosmology stops at the first
// iteration with |g| <= gtol and keeps that iteration's outputs: k_flat_newton appends the ones that
// moved to the next iteration's work list, and the next launches integrate only that list. The host
// reads the list's length once per iteration and stops when it is empty; in the graph-safe mode the
// length stays on the device and every one of the max_newton iterations is launched.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "gs.h"
#include "gs_internal.h"

namespace {

constexpr int kD = 3, kP = 4, kM = 2;  // state (phi, u, I), theta (a0, lambda, Om, Or), directions
constexpr int32_t kFailed = GS_ST_MAX_STEPS | GS_ST_H_UNDERFLOW | GS_ST_NONFINITE | GS_ST_TAPE_OVERFLOW;

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// workspace: [0, 256) gs_jvp's work counter, [256, 512) the lengths of the two work lists, then
// S [N,K,3,2], the directions [N,4,2] and two work lists [N] (this iteration's and the next)
struct FlatLayout {
  size_t S, dirs, list0, list1, total;
};
FlatLayout flat_layout(int64_t N, int32_t K) {
  FlatLayout L;
  L.S = 512;
  L.dirs = L.S + round256(size_t(N) * size_t(K) * kD * kM * sizeof(double));
  L.list0 = L.dirs + round256(size_t(N) * kP * kM * sizeof(double));
  L.list1 = L.list0 + round256(size_t(N) * sizeof(int32_t));
  L.total = L.list1 + round256(size_t(N) * sizeof(int32_t));
  return L;
}

int flat_fail(int code, const char* msg) { return gs::set_error(code, msg); }

__global__ void k_flat_dirs(long long N, double* dirs) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  // direction 0: theta = e_a0, direction 1: theta = e_Om; dirs[(n * 4 + q) * 2 + m]
#pragma unroll
  for (int q = 0; q < kP; q++)
#pragma unroll
    for (int m = 0; m < kM; m++) dirs[(n * kP + q) * kM + m] = ((q == 0 && m == 0) || (q == 2 && m == 1)) ? 1.0 : 0.0;
}

// One Newton iteration over the cosmologies work[0 .. n_work - 1] (all when work is null; the
// length is *n_work_dev when that is set), just integrated; the ones that take a step are appended
// to next[] (*n_next entries).
__global__ void k_flat_newton(long long n_work, const unsigned int* n_work_dev, const int32_t* work, int K,
                              const double* saveat, int per_traj, const double* t1, double* params,
                              const double* y_out, const double* S, int32_t* status, int32_t* n_newton, double* dydOm,
                              double* da0dOm, double* g_out, int it, int max_newton, double gtol, int32_t* next,
                              unsigned int* n_next) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nw = n_work_dev ? (long long)*n_work_dev : n_work;
  if (i >= nw) return;
  const long long n = work ? (long long)work[i] : i;
  const double nanv = __longlong_as_double(0x7ff8000000000000LL);
  double* th = params + n * kP;
  const int32_t st = status[n];
  n_newton[n] = it + 1;
  const double last_out = per_traj ? saveat[n * K + K - 1] : saveat[K - 1];
  const bool at_today = last_out == t1[n];
  if ((st & kFailed) || !at_today) {  // the state today is not available: no Newton step
    if (!at_today) status[n] = st | GS_ST_NO_CONVERGENCE;
    if (dydOm)
      for (int q = 0; q < K * kD; q++) dydOm[n * K * kD + q] = nanv;
    if (da0dOm) da0dOm[n] = nanv;
    if (g_out) g_out[n] = nanv;
    return;
  }
  const double* yT = y_out + (n * K + K - 1) * kD;
  const double* ST = S + (n * K + K - 1) * kD * kM;  // S[n][K-1][i][m]
  const double phi = yT[0], u = yT[1];
  const double a0 = th[0], lam = th[1], om = th[2], orad = th[3];
  const double den = 1.0 - u * u / 6.0;
  const double ev = exp(-lam * phi);
  const double num = om + orad + a0 * ev;
  const double g = num / den - 1.0;
  // dg/dy (the distance integral I does not enter g)
  const double g_phi = -lam * a0 * ev / den;
  const double g_u = num * (u / 3.0) / (den * den);
  const double dg_da0 = g_phi * ST[0 * kM + 0] + g_u * ST[1 * kM + 0] + ev / den;
  const double dg_dom = g_phi * ST[0 * kM + 1] + g_u * ST[1 * kM + 1] + 1.0 / den;
  const double da0 = -dg_dom / dg_da0;
  if (dydOm) {
    const double* Sn = S + n * (long long)K * kD * kM;
    for (int q = 0; q < K * kD; q++) dydOm[n * K * kD + q] = Sn[q * kM + 1] + da0 * Sn[q * kM + 0];
  }
  if (da0dOm) da0dOm[n] = da0;
  if (g_out) g_out[n] = g;
  if (fabs(g) <= gtol) return;
  if (it + 1 >= max_newton) {
    status[n] = st | GS_ST_NO_CONVERGENCE;
    return;
  }
  th[0] = a0 - g / dg_da0;
  next[atomicAdd(n_next, 1u)] = int32_t(n);
}

}  // namespace

extern "C" {

size_t gs_flat_workspace_bytes(int64_t N, int32_t K) {
  if (N < 0 || K < 1) return 0;
  return flat_layout(N, K).total;
}

int gs_solve_flat(int64_t N, const double* y0, double* params, const double* t0, const double* t1, double rtol,
                  double atol, int32_t K, const double* saveat, const gs_options* opt, int32_t max_newton,
                  double gtol, double* y_out, double* dydOm, double* da0dOm, double* g_out, int32_t* status,
                  int32_t* n_accept, int32_t* n_reject, int32_t* n_newton, void* workspace, size_t workspace_bytes,
                  void* cuda_stream) {
  if (!opt) return flat_fail(GS_ERR_INVALID, "opt must not be NULL");
  if (N < 0) return flat_fail(GS_ERR_INVALID, "N < 0");
  if (K < 1) return flat_fail(GS_ERR_INVALID, "gs_solve_flat needs K >= 1 outputs, the last at t1 (today)");
  if (max_newton < 1) return flat_fail(GS_ERR_INVALID, "max_newton must be >= 1");
  if (!(gtol > 0.0) || !std::isfinite(gtol)) return flat_fail(GS_ERR_INVALID, "gtol must be positive and finite");
  if (N == 0) return GS_OK;
  if (!params || !y_out || !status || !n_accept || !n_reject || !n_newton)
    return flat_fail(GS_ERR_INVALID, "params, y_out, status, step counts and n_newton must not be NULL");
  const FlatLayout L = flat_layout(N, K);
  if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return flat_fail(GS_ERR_WORKSPACE, "gs_solve_flat needs a 256-byte aligned workspace");
  if (workspace_bytes < L.total) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "workspace of %zu bytes is smaller than the %zu of gs_flat_workspace_bytes",
                  workspace_bytes, L.total);
    return flat_fail(GS_ERR_WORKSPACE, msg);
  }
  if (N > 0x7fffffffLL) return flat_fail(GS_ERR_INVALID, "gs_solve_flat takes at most 2^31 - 1 cosmologies");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  unsigned int* counts = reinterpret_cast<unsigned int*>(ws + 256);  // lengths of lists[0], lists[1]
  double* S = reinterpret_cast<double*>(ws + L.S);
  double* dirs = reinterpret_cast<double*>(ws + L.dirs);
  int32_t* lists[2] = {reinterpret_cast<int32_t*>(ws + L.list0), reinterpret_cast<int32_t*>(ws + L.list1)};
  const int per_traj = opt->per_traj_saveat ? 1 : 0;
  const bool sync_free = opt->graph_safe != 0;
  const int block = 256;
  k_flat_dirs<<<unsigned((N + block - 1) / block), block, 0, s>>>((long long)N, dirs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return flat_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  // the first iteration integrates every cosmology; later ones the list the previous one built, whose
  // length the host reads back (or, graph-safe, the kernels read on the device)
  const int32_t* work = nullptr;
  long long n_work = N;
  const unsigned int* n_work_dev = nullptr;
  for (int it = 0; it < max_newton && n_work > 0; it++) {
    const int rc = gs::jvp_on(GS_SYS_QUINTESSENCE, N, y0, params, t0, t1, rtol, atol, K, saveat, opt, kM, nullptr, dirs,
                              y_out, S, status, n_accept, n_reject, workspace, 256, cuda_stream, work, n_work,
                              n_work_dev);
    if (rc) return rc;
    int32_t* next = lists[it & 1];
    unsigned int* n_next = counts + (it & 1);
    e = cudaMemsetAsync(n_next, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return flat_fail(GS_ERR_CUDA, cudaGetErrorString(e));
    k_flat_newton<<<unsigned((n_work + block - 1) / block), block, 0, s>>>(
        n_work, n_work_dev, work, K, saveat, per_traj, t1, params, y_out, S, status, n_newton, dydOm, da0dOm, g_out, it,
        max_newton, gtol, next, n_next);
    e = cudaGetLastError();
    if (e != cudaSuccess) return flat_fail(GS_ERR_CUDA, cudaGetErrorString(e));
    work = next;
    if (sync_free) {
      n_work_dev = n_next;  // n_work stays N: the grid is sized for the longest possible list
    } else {
      unsigned int left = 0;
      e = cudaMemcpyAsync(&left, n_next, sizeof left, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return flat_fail(GS_ERR_CUDA, cudaGetErrorString(e));
      n_work = (long long)left;
    }
  }
  return GS_OK;
}

}  // extern "C"
