// Kernels of the ensemble solver and their launchers, instantiated once per system in the
// gs_inst_*.cu translation units.
//
//  k_plain    one thread per trajectory for its whole solve; a warp lasts as long as its slowest
//             lane (the per-thread kernel of Sec. 2.4 / Appendix A, Eq. cost).
//  k_persist  persistent CTAs (SM count x resident CTAs per SM). Each warp takes trajectory
//             indices from a device counter with one atomicAdd per refill (warp ballot of the
//             lanes that need work), so a lane whose trajectory has finished starts the next one
//             at its next step attempt instead of idling until the warp's slowest lane is done.
//             There is no spin-wait: the counter only grows, and a lane that draws an index past
//             N retires.
//  k_reverse  discrete adjoint, one thread per trajectory over its recorded tape.
//  k_rhs      f and its VJPs at given states (library utility; used by the tests).
#pragma once
#include <cuda_runtime.h>

#include "gs_adjoint.cuh"
#include "gs_stepper.cuh"

namespace gs {

struct LaunchCfg {
  int method, precision, kernel, block;
  cudaStream_t stream;
};

template <template <class> class SysT, class Tab, bool F32>
__global__ void __launch_bounds__(128) k_plain(const Problem pb) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= pb.N) return;
  Traj<SysT, Tab, F32> tr;
  tr.init(pb, n);
  while (!tr.done) tr.attempt(pb);
  tr.finish(pb);
}

template <template <class> class SysT, class Tab, bool F32>
__global__ void __launch_bounds__(128) k_persist(const Problem pb) {
  Traj<SysT, Tab, F32> tr;
  bool running = false, exhausted = false;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  while (true) {
    const bool need = !running && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned base = 0;
      if (int(lane) == leader) base = atomicAdd(pb.queue, unsigned(__popc(m)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const unsigned long long idx = (unsigned long long)base + unsigned(__popc(m & lt_mask));
        if (idx < (unsigned long long)pb.N) {
          tr.init(pb, (long long)idx);
          running = true;
          if (tr.done) { tr.finish(pb); running = false; }
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted)) break;
    if (running) {
      tr.attempt(pb);
      if (tr.done) { tr.finish(pb); running = false; }
    }
  }
}

template <template <class> class SysT, class Tab, bool F32>
__global__ void __launch_bounds__(128) k_reverse(const Problem pb) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= pb.N) return;
  Adjoint<SysT, Tab, F32> adj;
  adj.init(pb, n);
  while (!adj.done) adj.step(pb);
}

// Reverse sweeps from a work queue (counter pb.queue), lanes refilled as in k_persist.
template <template <class> class SysT, class Tab, bool F32>
__global__ void __launch_bounds__(128) k_reverse_persist(const Problem pb) {
  Adjoint<SysT, Tab, F32> adj;
  bool running = false, exhausted = false;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  while (true) {
    const bool need = !running && !exhausted;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned base = 0;
      if (int(lane) == leader) base = atomicAdd(pb.queue, unsigned(__popc(m)));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const unsigned long long idx = (unsigned long long)base + unsigned(__popc(m & lt_mask));
        if (idx < (unsigned long long)pb.N) {
          adj.init(pb, (long long)idx);
          running = !adj.done;
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted)) break;
    if (running) {
      adj.step(pb);
      if (adj.done) running = false;
    }
  }
}

template <template <class> class SysT, bool F32>
__global__ void k_rhs(long long M, const double* t, const double* y, const double* p, const double* w,
                      double* f, double* gy, double* gp) {
  using R = typename std::conditional<F32, float, double>::type;
  using Sys = SysT<R>;
  constexpr int D = Sys::D, NP = Sys::P, NPA = NP > 0 ? NP : 1;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= M) return;
  R yy[D], pp[NPA], ff[D];
  for (int i = 0; i < D; i++) yy[i] = R(y[n * D + i]);
  for (int q = 0; q < NP; q++) pp[q] = R(p[n * NP + q]);
  if (NP == 0) pp[0] = R(0);
  const R tt = R(t[n]);
  if (f) {
    Sys::f(tt, yy, pp, ff);
    for (int i = 0; i < D; i++) f[n * D + i] = double(ff[i]);
  }
  if (w && (gy || gp)) {
    R ww[D], gyy[D], gpp[NPA];
    for (int i = 0; i < D; i++) ww[i] = R(w[n * D + i]);
    Sys::vjp(tt, yy, pp, ww, gyy, gpp);
    if (gy)
      for (int i = 0; i < D; i++) gy[n * D + i] = double(gyy[i]);
    if (gp)
      for (int q = 0; q < NP; q++) gp[n * NP + q] = double(gpp[q]);
  }
}

// ------------------------------------------------------------------------------------------------
inline int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
  }
  return cached;
}

template <class K>
inline int persistent_grid(K kernel, int block) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sm_count();
}

template <template <class> class SysT, class Tab, bool F32>
cudaError_t launch_forward_t(const Problem& pb, const LaunchCfg& c) {
  const int block = c.block > 0 ? c.block : 128;
  if (c.kernel == 2) {
    auto kern = k_persist<SysT, Tab, F32>;
    long long grid = persistent_grid(kern, block);
    const long long need = (pb.N + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<unsigned(grid), block, 0, c.stream>>>(pb);
  } else {
    const long long grid = (pb.N + block - 1) / block;
    k_plain<SysT, Tab, F32><<<unsigned(grid), block, 0, c.stream>>>(pb);
  }
  return cudaGetLastError();
}

template <template <class> class SysT, class Tab, bool F32>
cudaError_t launch_reverse_t(const Problem& pb, const LaunchCfg& c) {
  const int block = c.block > 0 ? c.block : 128;
  if (c.kernel == 2) {
    auto kern = k_reverse_persist<SysT, Tab, F32>;
    long long grid = persistent_grid(kern, block);
    const long long need = (pb.N + block - 1) / block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<unsigned(grid), block, 0, c.stream>>>(pb);
  } else {
    const long long grid = (pb.N + block - 1) / block;
    k_reverse<SysT, Tab, F32><<<unsigned(grid), block, 0, c.stream>>>(pb);
  }
  return cudaGetLastError();
}

template <template <class> class SysT>
cudaError_t launch_forward(const Problem& pb, const LaunchCfg& c) {
  const bool f32 = c.precision == 1;
  switch (c.method) {
    case 0: return f32 ? launch_forward_t<SysT, Tsit5, true>(pb, c) : launch_forward_t<SysT, Tsit5, false>(pb, c);
    case 1: return f32 ? launch_forward_t<SysT, Dopri5, true>(pb, c) : launch_forward_t<SysT, Dopri5, false>(pb, c);
    default: return f32 ? launch_forward_t<SysT, Vern7, true>(pb, c) : launch_forward_t<SysT, Vern7, false>(pb, c);
  }
}

template <template <class> class SysT>
cudaError_t launch_reverse(const Problem& pb, const LaunchCfg& c) {
  const bool f32 = c.precision == 1;
  switch (c.method) {
    case 0: return f32 ? launch_reverse_t<SysT, Tsit5, true>(pb, c) : launch_reverse_t<SysT, Tsit5, false>(pb, c);
    case 1: return f32 ? launch_reverse_t<SysT, Dopri5, true>(pb, c) : launch_reverse_t<SysT, Dopri5, false>(pb, c);
    default: return f32 ? launch_reverse_t<SysT, Vern7, true>(pb, c) : launch_reverse_t<SysT, Vern7, false>(pb, c);
  }
}

template <template <class> class SysT>
cudaError_t launch_rhs(int precision, long long M, const double* t, const double* y, const double* p,
                       const double* w, double* f, double* gy, double* gp, cudaStream_t s) {
  const int block = 128;
  const long long grid = (M + block - 1) / block;
  if (grid == 0) return cudaSuccess;
  if (precision == 1) k_rhs<SysT, true><<<unsigned(grid), block, 0, s>>>(M, t, y, p, w, f, gy, gp);
  else k_rhs<SysT, false><<<unsigned(grid), block, 0, s>>>(M, t, y, p, w, f, gy, gp);
  return cudaGetLastError();
}

// per-system entry points defined in gs_inst_*.cu
#define GS_DECLARE_SYSTEM(name)                                                                        \
  cudaError_t forward_##name(const Problem& pb, const LaunchCfg& c);                                   \
  cudaError_t reverse_##name(const Problem& pb, const LaunchCfg& c);                                   \
  cudaError_t rhs_##name(int precision, long long M, const double* t, const double* y, const double* p, \
                         const double* w, double* f, double* gy, double* gp, cudaStream_t s);

#define GS_DEFINE_SYSTEM(name, SysT)                                                                   \
  cudaError_t forward_##name(const Problem& pb, const LaunchCfg& c) { return launch_forward<SysT>(pb, c); } \
  cudaError_t reverse_##name(const Problem& pb, const LaunchCfg& c) { return launch_reverse<SysT>(pb, c); } \
  cudaError_t rhs_##name(int precision, long long M, const double* t, const double* y, const double* p, \
                         const double* w, double* f, double* gy, double* gp, cudaStream_t s) {         \
    return launch_rhs<SysT>(precision, M, t, y, p, w, f, gy, gp, s);                                  \
  }

}  // namespace gs
