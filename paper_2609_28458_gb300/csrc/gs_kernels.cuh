// Kernels of the ensemble solver and their launchers, instantiated once per system and method in
// the gs_inst_*.cu translation units.
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
  int sm_limit;  // persistent kernels: at most this many SMs' worth of resident blocks (0: all SMs)
};

// Resident 128-thread blocks per SM requested from the register allocator (__launch_bounds__), for
// 7-stage pairs on states of at most 6 components: the FP32-pipe forward 5 (96 registers; measured on
// the 3 Gyr Milky-Way ensemble: with the stages in Nystrom form, forward with tape 29.1 ms against
// 33.4 ms at 4 blocks; in the general form 4 blocks had been faster, 28.1 against 30.7 ms forward
// alone, and 6 blocks 42% slower), the FP64-control forward 4 (115 registers; 5 blocks: 35.5 against
// 35.3 ms), the FP32 reverse 4 (128 registers: with its stage sweep in Nystrom form, 31.1 against
// 31.6 ms at 3 blocks; the general form had spilled there and was 5% slower, 2 blocks 15%), the
// checkpointed FP32 reverse 3 (<= 168: its segment replay keeps the register budget it was verified
// with). The FP64 forward of the 9-component
// precession state 4 blocks (16 warps per SM at 128 registers, against 8 at the compiler's 255: the
// FP64 pipe gets more warps to overlap; 10^6 Verner 7 solves 243.9 -> 222.5 ms despite spilling, 3
// blocks 229.9 ms). Other FP64 and Verner 7 kernels keep the compiler's choice.
#ifndef GS_FWD_BLOCKS_FP32DF
#define GS_FWD_BLOCKS_FP32DF 5
#endif
#ifndef GS_FWD_BLOCKS_FP32
#define GS_FWD_BLOCKS_FP32 4
#endif
#ifndef GS_REV_BLOCKS_FP32
#define GS_REV_BLOCKS_FP32 4
#endif
#ifndef GS_REV_CKPT_BLOCKS_FP32
#define GS_REV_CKPT_BLOCKS_FP32 3
#endif
#ifndef GS_FWD_BLOCKS_FP64_D9
#define GS_FWD_BLOCKS_FP64_D9 4
#endif
template <template <class> class SysT, class Tab, int PM, int MT = 0>
struct Occupancy {
  static constexpr bool small = Tab::S <= 7 && SysT<float>::D <= 6 && MT == 0;
  static constexpr int fwd = (PM == 2 && small) ? GS_FWD_BLOCKS_FP32DF
                             : (PM == 1 && small) ? GS_FWD_BLOCKS_FP32
                             : (PM == 0 && SysT<float>::D == 9 && MT == 0) ? GS_FWD_BLOCKS_FP64_D9 : 1;
  static constexpr int rev = ((PM == 1 || PM == 2) && small) ? GS_REV_BLOCKS_FP32 : 1;
  static constexpr int revck = ((PM == 1 || PM == 2) && small) ? GS_REV_CKPT_BLOCKS_FP32 : 1;
};

template <template <class> class SysT, class Tab, int PM>
__global__ void __launch_bounds__(128) k_plain(const Problem pb) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= pb.n_work) return;
  const long long n = pb.work ? (long long)pb.work[i] : i;
  Traj<SysT, Tab, PM> tr;
  tr.init(pb, n);
  while (!tr.done) tr.attempt(pb);
  tr.finish(pb);
}

// Prepared starts (Problem::start): init() for every trajectory of the launch, one thread each, rows
// written for the persistent kernel; trajectories that init() already finishes (empty or non-finite
// input) are finished here. Run as a plain kernel, a trajectory start no longer holds up the other
// lanes of a persistent warp, and the persistent kernel's code loses init() and the starting-step
// evaluation.
template <template <class> class SysT, class Tab, int PM>
__global__ void __launch_bounds__(128) k_start(const Problem pb) {
  const unsigned long long n_work = pb.n_work_dev ? (unsigned long long)*pb.n_work_dev : (unsigned long long)pb.n_work;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n_work;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const long long n = pb.work ? (long long)pb.work[i] : (long long)i;
    Traj<SysT, Tab, PM> tr;
    tr.init(pb, n);
    if (tr.done) tr.finish(pb);
    tr.save_start(pb);
  }
}

// PRE: trajectories start from the rows k_start prepared (MT == 0, PM 0-2), else in place
template <template <class> class SysT, class Tab, int PM, int MT = 0, bool PRE = false>
__global__ void __launch_bounds__(128, (Occupancy<SysT, Tab, PM, MT>::fwd)) k_persist(const Problem pb) {
  static_assert(!PRE || (MT == 0 && PM != 3), "prepared starts: modes 0-2 without sensitivities");
  Traj<SysT, Tab, PM, MT> tr;
  const unsigned long long n_work = pb.n_work_dev ? (unsigned long long)*pb.n_work_dev : (unsigned long long)pb.n_work;
  const unsigned lane = threadIdx.x & 31u;
  // lanes at or above pb.warp_lanes take no work: a small ensemble spreads over more warps
  bool running = false, exhausted = lane >= unsigned(pb.warp_lanes);
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
        if (idx < n_work) {
          const long long traj = pb.work ? (long long)pb.work[idx] : (long long)idx;
          if constexpr (PRE) {
            running = tr.load_start(pb, traj);
          } else {
            tr.init(pb, traj);
            running = true;
            if (tr.done) { tr.finish(pb); running = false; }
          }
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

template <template <class> class SysT, class Tab, int PM>
__global__ void __launch_bounds__(128) k_reverse(const Problem pb) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= pb.n_work) return;
  const long long n = pb.work ? (long long)pb.work[i] : i;
  Adjoint<SysT, Tab, PM> adj;
  adj.init(pb, n);
  while (!adj.done) adj.step(pb);
}

// Shared memory of the persistent reverse pass per thread: the stage Jacobian factors (FP32 modes
// of systems with f_save, 7-stage pairs), S x SaveQ float4 = 224 bytes for the Milky-Way system,
// 28.7 KB per 128-thread block.
template <template <class> class SysT, class Tab, int PM>
struct RevSlab {
  static constexpr int Q = SaveQ<SysT<float>>::value;
  static constexpr bool on = (PM == 1 || PM == 2) && Q > 0 && Tab::S <= 7;
  static constexpr int bytes_per_thread = on ? Tab::S * Q * 16 : 0;
};

// Reverse sweeps from a work queue (counter pb.queue), lanes refilled as in k_persist.
template <template <class> class SysT, class Tab, int PM>
__global__ void __launch_bounds__(128, (Occupancy<SysT, Tab, PM>::rev)) k_reverse_persist(const Problem pb) {
  constexpr bool SLAB = RevSlab<SysT, Tab, PM>::on;
  Adjoint<SysT, Tab, PM, SLAB> adj;
  if constexpr (SLAB) {
    extern __shared__ float4 gs_rev_slab[];
    adj.sl = unsigned(__cvta_generic_to_shared(gs_rev_slab + threadIdx.x));
    adj.st = 16u * blockDim.x;
  }
  const unsigned long long n_work = pb.n_work_dev ? (unsigned long long)*pb.n_work_dev : (unsigned long long)pb.n_work;
  const unsigned lane = threadIdx.x & 31u;
  // lanes at or above pb.warp_lanes take no work: a small ensemble spreads over more warps
  bool running = false, exhausted = lane >= unsigned(pb.warp_lanes);
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
        if (idx < n_work) {
          adj.init(pb, pb.work ? (long long)pb.work[idx] : (long long)idx);
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

// Reverse sweeps over a checkpointed tape (stride S > 1) from a work queue. Each round of the loop
// gives every lane one segment: the lane replays it from its checkpoint (up to S - 1 forward steps)
// and then reverses its steps. Whole segments per round keep the lanes of a warp in the same phase,
// replaying together and reversing together; only a trajectory's first (newest, partial) segment
// leaves a lane idle for part of a round. Lanes are refilled between rounds.
template <template <class> class SysT, class Tab, int PM>
__global__ void __launch_bounds__(128, (Occupancy<SysT, Tab, PM>::revck)) k_reverse_ckpt(const Problem pb) {
  constexpr bool SLAB = RevSlab<SysT, Tab, PM>::on;
  Adjoint<SysT, Tab, PM, SLAB, true> adj;
  if constexpr (SLAB) {
    extern __shared__ float4 gs_rev_slab[];
    adj.sl = unsigned(__cvta_generic_to_shared(gs_rev_slab + threadIdx.x));
    adj.st = 16u * blockDim.x;
  }
  const unsigned long long n_work = pb.n_work_dev ? (unsigned long long)*pb.n_work_dev : (unsigned long long)pb.n_work;
  const unsigned lane = threadIdx.x & 31u;
  // lanes at or above pb.warp_lanes take no work: a small ensemble spreads over more warps
  bool running = false, exhausted = lane >= unsigned(pb.warp_lanes);
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
        if (idx < n_work) {
          adj.init(pb, pb.work ? (long long)pb.work[idx] : (long long)idx);
          running = !adj.done;
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted)) break;
    if (running) {
      adj.load_segment(pb);
      do {
        adj.step_ck(pb);
      } while (!adj.done && adj.a >= adj.seg_lo);
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
  constexpr int NPP = PrepCount<Sys>::value > 0 ? PrepCount<Sys>::value : 1;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= M) return;
  R yy[D], pp[NPP], ff[D];
  for (int i = 0; i < D; i++) yy[i] = R(y[n * D + i]);
  for (int q = 0; q < NP; q++) pp[q] = R(p[n * NP + q]);
  if (NP == 0) pp[0] = R(0);
  prep_params<Sys>(pp);
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
      for (int q = 0; q < NP; q++) gp[n * NP + q] = double(gpp[q]) * VjpParamScale<Sys>::of(q);
  }
}

// ------------------------------------------------------------------------------------------------
// Longest-first work lists. A persistent launch ends when its slowest lane does, so the trajectories
// taken last should be the short ones; a plain launch's warps run as long as their longest member,
// so members of similar length should share a warp. Costs are bucketed on a log scale (16 buckets per
// octave, 4096 in all), buckets in descending cost; three small kernels and no host synchronisation.
constexpr int kOrderBuckets = 4096;
__device__ __forceinline__ int cost_bucket(float c) {
  int b = 0;
  if (c > 0.0f) {
    b = int(floorf(log2f(c) * 16.0f)) + 2048;
    b = b < 1 ? 1 : (b > kOrderBuckets - 1 ? kOrderBuckets - 1 : b);
  }
  return kOrderBuckets - 1 - b;  // zero or invalid cost: the last bucket
}
__device__ __forceinline__ float cost_of(const float* fc, const int32_t* ic, long long n) {
  if (fc) return fc[n];
  const int32_t v = ic[n];
  return v > 0 ? float(v) : 0.0f;
}
// Both passes aggregate per warp: the lanes that share a bucket are counted (and placed) by one
// atomic of their lowest lane. Ensembles of near-equal cost fall into a few buckets, where one atomic
// per member would serialise on a single address. Blocks are whole warps (256 threads).
static __global__ void k_order_hist(long long N, const float* fc, const int32_t* ic, unsigned int* cnt) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool ok = n < N;
  const int b = ok ? cost_bucket(cost_of(fc, ic, n)) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  const int lane = threadIdx.x & 31;
  if (ok && lane == __ffs(peers) - 1) atomicAdd(&cnt[b], unsigned(__popc(peers)));
}
// exclusive scan of the kOrderBuckets counters in place (one block of 1024 threads, 4 each)
static __global__ void k_order_scan(unsigned int* cnt) {
  __shared__ unsigned int part[1024];
  const int t = threadIdx.x;
  unsigned int v[4], sum = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) { v[i] = cnt[4 * t + i]; sum += v[i]; }
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned int x = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  unsigned int run = part[t] - sum;
#pragma unroll
  for (int i = 0; i < 4; i++) { cnt[4 * t + i] = run; run += v[i]; }
}
static __global__ void k_order_scatter(long long N, const float* fc, const int32_t* ic, unsigned int* pos,
                                       int32_t* order) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool ok = n < N;
  const int b = ok ? cost_bucket(cost_of(fc, ic, n)) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  unsigned base = 0;
  if (ok && lane == leader) base = atomicAdd(&pos[b], unsigned(__popc(peers)));
  base = __shfl_sync(0xffffffffu, base, leader);
  // lanes of one bucket keep their relative order, so runs of equal cost stay contiguous
  if (ok) order[base + unsigned(__popc(peers & ((1u << lane) - 1u)))] = int32_t(n);
}
// order[0 .. N-1]: trajectory indices by descending cost (fc, or ic when fc is null)
inline cudaError_t build_order(long long N, const float* fc, const int32_t* ic, unsigned int* cnt, int32_t* order,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, size_t(kOrderBuckets) * 4, s);
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned((N + 255) / 256);
  k_order_hist<<<grid, 256, 0, s>>>(N, fc, ic, cnt);
  k_order_scan<<<1, 1024, 0, s>>>(cnt);
  k_order_scatter<<<grid, 256, 0, s>>>(N, fc, ic, cnt, order);
  return cudaGetLastError();
}

// Estimated cost of a trajectory: (t1 - t0) ||f(t0, y0)/s|| / ||y0/s||, s = atol + rtol |y0| (RMS
// norms): the interval over the local time scale of the starting-step heuristic, from one FP32
// evaluation of f. Empty or non-finite trajectories cost 0.
template <template <class> class SysT>
__global__ void k_cost_estimate(const Problem pb) {
  using Sys = SysT<float>;
  constexpr int D = Sys::D, NP = Sys::P;
  constexpr int NPP = PrepCount<Sys>::value > 0 ? PrepCount<Sys>::value : 1;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= pb.N) return;
  const double t0 = pb.t0[n], t1 = pb.t1[n];
  float y[D], f[D], p[NPP];
#pragma unroll
  for (int i = 0; i < D; i++) y[i] = float(pb.y0[n * D + i]);
#pragma unroll
  for (int q = 0; q < NP; q++) p[q] = float(pb.params[n * NP + q]);
  if (NP == 0) p[0] = 0.0f;
  prep_params<Sys>(p);
  Sys::f(float(t0), y, p, f);
  const float at = float(pb.atol), rt = float(pb.rtol);
  float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
  for (int i = 0; i < D; i++) {
    const float sc = at + rt * fabsf(y[i]);
    d0 += (y[i] / sc) * (y[i] / sc);
    d1 += (f[i] / sc) * (f[i] / sc);
  }
  float c = float(t1 - t0) * sqrtf(d1 / fmaxf(d0, 1e-30f));
  if (!(c > 0.0f) || !isfinite(c)) c = 0.0f;
  pb.ord_cost[n] = c;
}

// The ordered copy of pb for a forward launch (pb itself when no ordering is asked for).
template <template <class> class SysT>
inline cudaError_t ordered(const Problem& pb, cudaStream_t s, Problem& q) {
  q = pb;
  if (!pb.ord_order || pb.work) return cudaSuccess;
  const float* fc = nullptr;
  if (!pb.cost_hint) {
    k_cost_estimate<SysT><<<unsigned((pb.N + 255) / 256), 256, 0, s>>>(pb);
    fc = pb.ord_cost;
  }
  const cudaError_t e = build_order(pb.N, fc, pb.cost_hint, pb.ord_cnt, pb.ord_order, s);
  if (e != cudaSuccess) return e;
  q.work = pb.ord_order;
  q.n_work = pb.N;
  return cudaSuccess;
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
inline int persistent_grid(K kernel, int block, int sm_limit, size_t smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  if (per_sm < 1) per_sm = 1;
  const int sms = (sm_limit > 0 && sm_limit < sm_count()) ? sm_limit : sm_count();
  return per_sm * sms;
}

template <template <class> class SysT, class Tab, int PM>
cudaError_t launch_forward_t(const Problem& pb0, const LaunchCfg& c) {
  const int block = c.block > 0 ? c.block : 128;
  if (pb0.n_work <= 0) return cudaSuccess;
  Problem pb;
  const cudaError_t eo = ordered<SysT>(pb0, c.stream, pb);
  if (eo != cudaSuccess) return eo;
  if (c.kernel == 2) {
    auto kern = k_persist<SysT, Tab, PM>;
    if constexpr (PM != 3) {
      if (pb.start) {  // the starts, in the launch's own (unordered) work list: coalesced input reads
        const long long sgrid = (pb0.n_work + 127) / 128;
        k_start<SysT, Tab, PM><<<unsigned(sgrid < 1 ? 1 : sgrid), 128, 0, c.stream>>>(pb0);
        kern = k_persist<SysT, Tab, PM, 0, true>;
      }
    }
    long long grid = persistent_grid(kern, block, c.sm_limit);
    const long long per_block = (long long)block * pb.warp_lanes / 32;
    const long long need = (pb.n_work + per_block - 1) / per_block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<unsigned(grid), block, 0, c.stream>>>(pb);
  } else {
    const long long grid = (pb.n_work + block - 1) / block;
    k_plain<SysT, Tab, PM><<<unsigned(grid), block, 0, c.stream>>>(pb);
  }
  return cudaGetLastError();
}

template <template <class> class SysT, class Tab, int PM>
cudaError_t launch_reverse_t(const Problem& pb, const LaunchCfg& c) {
  const int block = c.block > 0 ? c.block : 128;
  if (pb.n_work <= 0) return cudaSuccess;
  if (pb.tape.stride > 1) {  // checkpointed tape: persistent kernel only (checked by the caller)
    if constexpr (PM == 3) {
      return cudaErrorInvalidValue;
    } else {
      auto kern = k_reverse_ckpt<SysT, Tab, PM>;
      const size_t smem = size_t(RevSlab<SysT, Tab, PM>::bytes_per_thread) * size_t(block);
      long long grid = persistent_grid(kern, block, c.sm_limit, smem);
      const long long per_block = (long long)block * pb.warp_lanes / 32;
      const long long need = (pb.n_work + per_block - 1) / per_block;
      if (grid > need) grid = need;
      if (grid < 1) grid = 1;
      kern<<<unsigned(grid), block, smem, c.stream>>>(pb);
      return cudaGetLastError();
    }
  }
  if (c.kernel == 2) {
    auto kern = k_reverse_persist<SysT, Tab, PM>;
    const size_t smem = size_t(RevSlab<SysT, Tab, PM>::bytes_per_thread) * size_t(block);
    long long grid = persistent_grid(kern, block, c.sm_limit, smem);
    const long long per_block = (long long)block * pb.warp_lanes / 32;
    const long long need = (pb.n_work + per_block - 1) / per_block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<unsigned(grid), block, smem, c.stream>>>(pb);
  } else {
    const long long grid = (pb.n_work + block - 1) / block;
    k_reverse<SysT, Tab, PM><<<unsigned(grid), block, 0, c.stream>>>(pb);
  }
  return cudaGetLastError();
}

// forward solve carrying MT sensitivity directions (persistent kernel)
template <template <class> class SysT, class Tab, int PM, int MT>
cudaError_t launch_jvp_t(const Problem& pb0, const LaunchCfg& c) {
  const int block = c.block > 0 ? c.block : 128;
  if (pb0.n_work <= 0) return cudaSuccess;
  Problem pb;
  const cudaError_t eo = ordered<SysT>(pb0, c.stream, pb);
  if (eo != cudaSuccess) return eo;
  auto kern = k_persist<SysT, Tab, PM, MT>;
  long long grid = persistent_grid(kern, block, c.sm_limit);
  const long long per_block = (long long)block * pb.warp_lanes / 32;
  const long long need = (pb.n_work + per_block - 1) / per_block;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<unsigned(grid), block, 0, c.stream>>>(pb);
  return cudaGetLastError();
}
// directions per launch: up to 4 for the 7-stage pairs, 1 for Verner 7 (its 10 stages of duals would
// not fit the register file)
template <class Tab>
constexpr int max_jvp_group() { return Tab::S <= 7 ? 4 : 1; }

template <template <class> class SysT, class Tab, int PM>
cudaError_t launch_jvp_p(const Problem& pb, const LaunchCfg& c, int mt) {
  if constexpr (Tab::S <= 7) {
    switch (mt) {
      case 1: return launch_jvp_t<SysT, Tab, PM, 1>(pb, c);
      case 2: return launch_jvp_t<SysT, Tab, PM, 2>(pb, c);
      default: return launch_jvp_t<SysT, Tab, PM, 4>(pb, c);
    }
  } else {
    return launch_jvp_t<SysT, Tab, PM, 1>(pb, c);
  }
}
template <template <class> class SysT, class Tab>
cudaError_t launch_jvp_m(const Problem& pb, const LaunchCfg& c, int mt) {
  return c.precision == 0 ? launch_jvp_p<SysT, Tab, 0>(pb, c, mt) : launch_jvp_p<SysT, Tab, 2>(pb, c, mt);
}

template <template <class> class SysT, class Tab>
cudaError_t launch_forward_m(const Problem& pb, const LaunchCfg& c) {
  switch (c.precision) {
    case 0: return launch_forward_t<SysT, Tab, 0>(pb, c);
    case 1: return launch_forward_t<SysT, Tab, 1>(pb, c);
    case 3:
      if constexpr (HasDF64<SysT>::value) return launch_forward_t<SysT, Tab, 3>(pb, c);
      else return cudaErrorInvalidValue;
    default: return launch_forward_t<SysT, Tab, 2>(pb, c);
  }
}
template <template <class> class SysT, class Tab>
cudaError_t launch_reverse_m(const Problem& pb, const LaunchCfg& c) {
  switch (c.precision) {
    case 0: return launch_reverse_t<SysT, Tab, 0>(pb, c);
    case 1: return launch_reverse_t<SysT, Tab, 1>(pb, c);
    case 3:
      if constexpr (HasDF64<SysT>::value) return launch_reverse_t<SysT, Tab, 3>(pb, c);
      else return cudaErrorInvalidValue;
    default: return launch_reverse_t<SysT, Tab, 2>(pb, c);
  }
}

template <template <class> class SysT>
cudaError_t launch_rhs(int precision, long long M, const double* t, const double* y, const double* p,
                       const double* w, double* f, double* gy, double* gp, cudaStream_t s) {
  const int block = 128;
  const long long grid = (M + block - 1) / block;
  if (grid == 0) return cudaSuccess;
  if (precision != 0) k_rhs<SysT, true><<<unsigned(grid), block, 0, s>>>(M, t, y, p, w, f, gy, gp);
  else k_rhs<SysT, false><<<unsigned(grid), block, 0, s>>>(M, t, y, p, w, f, gy, gp);
  return cudaGetLastError();
}

// bytes of a prepared-start row (Problem::start) of a system in a precision mode (0: none, for
// the df64 mode); the row does not depend on the method
template <template <class> class SysT>
long long start_row_t(int precision) {
  switch (precision) {
    case 0: return Traj<SysT, Tsit5, 0>::kStartBytes;
    case 1: return Traj<SysT, Tsit5, 1>::kStartBytes;
    case 2: return Traj<SysT, Tsit5, 2>::kStartBytes;
    default: return 0;
  }
}

// per-system, per-method entry points defined in gs_inst_<system>_<method>.cu, and the right-hand-side
// evaluator and prepared-start row size of each system (in its Tsit5 unit)
#define GS_DECLARE_METHOD(name, Tab)                                      \
  cudaError_t forward_##name##_##Tab(const Problem& pb, const LaunchCfg& c); \
  cudaError_t reverse_##name##_##Tab(const Problem& pb, const LaunchCfg& c); \
  cudaError_t jvp_##name##_##Tab(const Problem& pb, const LaunchCfg& c, int mt);
#define GS_DECLARE_SYSTEM(name)                                                                         \
  GS_DECLARE_METHOD(name, Tsit5)                                                                        \
  GS_DECLARE_METHOD(name, Dopri5)                                                                       \
  GS_DECLARE_METHOD(name, Vern7)                                                                        \
  cudaError_t rhs_##name(int precision, long long M, const double* t, const double* y, const double* p, \
                         const double* w, double* f, double* gy, double* gp, cudaStream_t s);         \
  long long start_row_##name(int precision);

// The heaviest instantiations (precession) put the reverse kernels in a translation unit of their own
// (GS_DEFINE_FORWARD_JVP + GS_DEFINE_REVERSE) so that the two halves compile in parallel.
#define GS_DEFINE_FORWARD_JVP(name, SysT, Tab)                                                            \
  cudaError_t forward_##name##_##Tab(const Problem& pb, const LaunchCfg& c) {                             \
    return launch_forward_m<SysT, Tab>(pb, c);                                                           \
  }                                                                                                      \
  cudaError_t jvp_##name##_##Tab(const Problem& pb, const LaunchCfg& c, int mt) {                         \
    return launch_jvp_m<SysT, Tab>(pb, c, mt);                                                           \
  }
#define GS_DEFINE_REVERSE(name, SysT, Tab)                                                                \
  cudaError_t reverse_##name##_##Tab(const Problem& pb, const LaunchCfg& c) {                             \
    return launch_reverse_m<SysT, Tab>(pb, c);                                                           \
  }
#define GS_DEFINE_METHOD(name, SysT, Tab) \
  GS_DEFINE_FORWARD_JVP(name, SysT, Tab)  \
  GS_DEFINE_REVERSE(name, SysT, Tab)
#define GS_DEFINE_RHS(name, SysT)                                                                         \
  cudaError_t rhs_##name(int precision, long long M, const double* t, const double* y, const double* p,  \
                         const double* w, double* f, double* gy, double* gp, cudaStream_t s) {           \
    return launch_rhs<SysT>(precision, M, t, y, p, w, f, gy, gp, s);                                    \
  }                                                                                                      \
  long long start_row_##name(int precision) { return start_row_t<SysT>(precision); }

}  // namespace gs
