// Per-trajectory adaptive explicit Runge-Kutta integration as a step state machine.
//
// One object of Traj holds a trajectory's private state (Sec. 2.4: state, stages and FSAL stage in
// the thread's registers). init() loads a trajectory, attempt() makes one step attempt
// (Appendix A: Eq. rk stages, Eq. errnorm norm, Eq. controller new step, Eq. dense outputs) and
// finish() writes the status and step counts. The plain kernel runs init/attempt.../finish per
// thread; the persistent kernel interleaves them so a lane that finishes takes new work at once.
//
// Precision mode PM:
//  0  FP64: every operation in FP64.
//  1  FP32 stages: stage vectors, right-hand sides and dense outputs in FP32; the state is a
//     compensated FP32 pair (hi + lo, updated with an error-free TwoSum; stage states are formed
//     from the high part, whose rounding they share anyway); the squares of the scaled
//     errors are accumulated in FP64; t is FP64 with Kahan compensation; h, the accept test and the
//     step-size update are FP64, with the controller's power taken in FP32 (it only scales a
//     proposal that is then clamped to [alpha_min, alpha_max]).
//  2  FP32 stages, FP32-pipe control: as 1, but the time is an unevaluated FP32 pair (th + tl,
//     >= 48 significant bits, advanced by TwoSum), the step size the stages use is the FP32 step
//     itself (so state and time advance by the same number), and the norm accumulation and the
//     controller are FP32. No FP64 instruction is left in the attempt loop; FP64 on GB300 issues
//     at a small fraction of the FP32 rate.
//  3  df64 stages: the state, the stages, the stage times, the error estimate and the dense outputs
//     in double-FP32 arithmetic (gs_df64.cuh, ~48 bits), the time and the controller as in mode 2.
//     For the tolerances FP32 cannot reach (rtol ~1e-10) without the FP64 pipe.
//
// Readings where the paper is silent (the same as the CPU oracle's): Hairer-Norsett-Wanner starting
// step with exponent 1/(nu+1); the last step is clipped to land on t1 when h(1+4eps) >= t1 - t;
// h underflow when h < 16 eps max(|t|,|t1|) (eps of the time representation); max_steps attempts;
// failures give NaN outputs.
#pragma once
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "gs_bits.cuh"
#include "gs_dual.cuh"
#include "gs_systems.cuh"
#include "gs_tableaux.cuh"

namespace gs {

enum : int32_t {
  ST_MAX_STEPS = 1, ST_H_UNDERFLOW = 2, ST_NONFINITE = 4, ST_EMPTY = 8, ST_SAVEAT_OUTSIDE = 16,
  ST_TAPE_OVERFLOW = 32
};
constexpr int32_t ST_FAILED = ST_MAX_STEPS | ST_H_UNDERFLOW | ST_NONFINITE | ST_TAPE_OVERFLOW;
constexpr int kChunk = 32;  // accepted steps per tape chunk

// Step tape: per accepted step the state at its start, its time, its length and a last-step flag, in
// chunks of kChunk slots taken from a pool with an atomic bump counter (no waits anywhere). Each
// chunk starts with a 16-byte header holding the index of the trajectory's previous chunk, so the
// chunks of one trajectory form a list walked backwards by the reverse pass from head[n].
constexpr int kChunkHeader = 16;
//
// Checkpoint stride S > 1 (S divides kChunk): a chunk holds, after its header, the lengths of its
// kChunk steps (the last, clipped step of a trajectory recorded with a negative sign) and one
// checkpoint per S steps: the full integrator state at the start of every S-th accepted step (the
// state, its FP32 low part, the first stage k1 and the time). The reverse pass replays each segment
// of S steps from its checkpoint with those lengths (Traj::replay_step, the arithmetic of attempt())
// and so recovers every step's start state bit for bit. Outputs are attributed to the step that
// emitted them through emit[N, K], since the replay does not know the times of the previous segment.
struct Tape {
  unsigned char* pool;
  long long pool_chunks;
  long long chunk_bytes;
  unsigned long long* pool_next;
  int32_t* head;   // [N] last chunk of each trajectory (-1: none)
  int32_t* n_rec;  // [N] accepted steps recorded (-1: the tape overflowed)
  int32_t cap;     // most steps recorded per trajectory (more: the tape overflows)
  int32_t stride;  // checkpoint stride S (1: a full slot per accepted step)
  int32_t* emit;   // S > 1: [N, K] the accepted step that emitted each output; -1: the output is
                   // y0 (at t0), -2: unused (outside [t0, t1]), n_acc: emitted after the last step
  unsigned int* verify;  // S > 1, optional: [2] replayed segment ends compared with the next
                         // checkpoint, and those that differed (the reverse pass's self-check)
};
constexpr int kEmitT0 = -1, kEmitUnused = -2;

struct Problem {
  long long N;
  // optional work list: a launch processes trajectories work[0 .. n_work - 1] (indices into the
  // [N, ...] arrays) and leaves the others untouched; without one, n_work = N and work = null. The
  // persistent kernels take the length from *n_work_dev instead when it is set (n_work is then
  // the largest possible length, used to size the grid).
  const int32_t* work;
  long long n_work;
  const unsigned int* n_work_dev;
  // longest-first ordering of a forward launch (all null: as stored): either by cost_hint or by the
  // estimate written to ord_cost; the order goes to ord_order, ord_cnt holds the bucket counters
  const int32_t* cost_hint;
  float* ord_cost;
  int32_t* ord_order;
  unsigned int* ord_cnt;
  int32_t K, per_traj;
  const double* y0;
  const double* params;
  const double* t0;
  const double* t1;
  const double* saveat;
  double rtol, atol;
  int32_t max_steps;
  double safety, alpha_min, alpha_max, beta1, beta2, h0;
  float fsafety, falpha_min, falpha_max, fbeta1, fbeta2;  // FP32 copies for the FP32 controllers
  double* y_out;
  int32_t* status;
  int32_t* n_acc;
  int32_t* n_rej;
  int32_t record;
  Tape tape;
  unsigned int* queue;  // persistent kernel work counter
  int32_t warp_lanes;   // persistent kernels: lanes per warp that take work (1..32)
  // forward sensitivities: seeds dy0 [N, d, m_total] and dp [N, p, m_total] (either may be null),
  // output S [N, K, d, m_total]; a launch handles the directions m_off .. m_off + MT - 1
  const double* dy0;
  const double* dp;
  double* S_out;
  int32_t m_total, m_off;
  // adjoint
  const double* dLdy;
  double* dLdy0;
  double* dLdp;
  // prepared starts (persistent forward solves without sensitivities, precision modes 0-2): k_start
  // runs init() for every trajectory of the launch and leaves its state in row n of `start`
  // (start_row bytes apart, 16-byte aligned); the persistent kernel then loads a row where it would
  // otherwise start the trajectory itself. Null: the persistent kernel runs init() in place.
  unsigned char* start;
  long long start_row;
};

__device__ __forceinline__ double save_at(const Problem& pb, long long n, int k) {
  return pb.per_traj ? pb.saveat[n * pb.K + k] : pb.saveat[k];
}

// An output time is used iff it lies in [t0, t1] and does not decrease (t0, t1 finite).
// save_valid_bits: the same answer from the bit patterns (gs_bits.cuh), for trajectory start-up in the
// FP32-stage mode.
__device__ __forceinline__ bool save_valid(const Problem& pb, long long n, int k, double t0, double t1) {
  const double s = save_at(pb, n, k);
  return s >= t0 && s <= t1 && (k == 0 || s >= save_at(pb, n, k - 1));
}
__device__ __forceinline__ bool save_valid_bits(const Problem& pb, long long n, int k, double t0, double t1) {
  const double s = save_at(pb, n, k);
  return le_f64_bits(t0, s) && le_f64_bits(s, t1) && (k == 0 || le_f64_bits(save_at(pb, n, k - 1), s));
}

template <class R>
__device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
  s = a + b;
  const R bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// x = hi + lo with hi = fl32(x): an exact split of an FP64 number into an FP32 pair (48 bits).
__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = float(x);
  lo = float(x - double(hi));
}

constexpr float kEps48 = 3.5527136788005009e-15f;  // 2^-48: unit roundoff of an FP32 pair

// a * b + c with one rounding, as an explicit fused multiply-add. The stage sums and state updates of
// a step are written with it, so that every kernel that inlines them (the forward attempt, and the
// reverse pass's replay of a checkpoint segment) rounds them alike, whichever multiply-add fusions the
// compiler would otherwise pick in each: a product that two sums share (for FSAL pairs the last
// stage's weights are the new state's) may be rounded once and reused in one kernel and fused into
// both sums in another. (Measured: with plain expressions the FP32-pair replay missed the next
// checkpoint at 17% of segment ends; with these, at none.)
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ F2 fmadd(const F2& a, const F2& b, const F2& c) { return a * b + c; }
template <class R, int M>
__device__ __forceinline__ Dual<R, M> fmadd(R a, const Dual<R, M>& b, const Dual<R, M>& c) {
  Dual<R, M> r;
  r.v = fmadd(a, b.v, c.v);
#pragma unroll
  for (int m = 0; m < M; m++) r.d[m] = fmadd(a, b.d[m], c.d[m]);
  return r;
}

// value part and derivative part m of a plain real (derivative 0) or a dual number
__device__ __forceinline__ float dpart(float, int) { return 0.0f; }
__device__ __forceinline__ double dpart(double, int) { return 0.0; }
template <class R, int M> __device__ __forceinline__ R dpart(const Dual<R, M>& x, int m) { return x.d[m]; }

// new state y + incr of an FP32 mode: the value is split error-free into (hi, lo); derivative parts
// (forward sensitivities) are carried by hi and need no compensation
__device__ __forceinline__ void state_update(float y, float incr, float& hi, float& lo) {
  two_sum(y, incr, hi, lo);
}
template <int M>
__device__ __forceinline__ void state_update(const Dual<float, M>& y, const Dual<float, M>& incr, Dual<float, M>& hi,
                                             float& lo) {
  two_sum(y.v, incr.v, hi.v, lo);
#pragma unroll
  for (int m = 0; m < M; m++) hi.d[m] = y.d[m] + incr.d[m];
}

template <int PM>
struct PrecTraits {
  static constexpr bool F32 = PM == 1 || PM == 2;  // FP32 stages with an FP32-pair state
  static constexpr bool DF = PM == 2 || PM == 3;   // FP32-pair time, FP32 step size and controller
  static constexpr bool DD = PM == 3;              // df64 stages and state
  using R = typename std::conditional<F32, float, typename std::conditional<DD, F2, double>::type>::type;
};

// MT: number of forward-sensitivity directions carried with the state (0: none). With MT > 0 every
// stage quantity is a Dual<R, MT>, so f evaluated on it returns k_j and J_y S_j + J_theta dtheta at once
// (Sec. 2.3, Eq. sens; Appendix A, Eq. stage-sens); step control uses the value parts only.
template <template <class> class SysT, class Tab, int PM, int MT = 0>
struct Traj {
  static constexpr bool F32 = PrecTraits<PM>::F32;
  static constexpr bool DF = PrecTraits<PM>::DF;
  static constexpr bool DD = PrecTraits<PM>::DD;
  // PM 1 keeps FP64 numbers beside FP32 stages; its conversions between the two and its tests of
  // FP64 inputs go through the integer helpers of gs_bits.cuh, so that the FP64 pipe carries only the
  // FP64 arithmetic of the precision split (the other modes use the instructions)
  static constexpr bool BITS = PM == 1;
  using R = typename PrecTraits<PM>::R;
  using T = typename std::conditional<(MT > 0), Dual<R, (MT > 0 ? MT : 1)>, R>::type;
  using Sys = SysT<T>;
  static constexpr int D = Sys::D, NP = Sys::P, S = Tab::S;
  static constexpr int NPA = NP > 0 ? NP : 1;
  static constexpr int NPP = PrepCount<Sys>::value > 0 ? PrepCount<Sys>::value : 1;  // theta + prepared constants
  static constexpr int DL = F32 ? D : 1;
  // FP32 modes on second-order systems with a 7-stage FSAL pair: the stages in Nystrom form
  // (gs_tableaux.cuh, Nystrom): stage sums over the DH position components only
  static constexpr bool RKN = F32 && MT == 0 && Tab::FSAL && Tab::S == 7 && SecondOrder<Sys>::value;
  static constexpr int DH = D / 2;
  using NY = Nystrom<Tab>;
  // slot layout: y[D] as FP64 (PM 0), its FP32 high part (PM 1, 2; the reverse pass recomputes
  // the stages from the high part alone, as the forward attempt does) or its df64 pairs (PM 3), then
  // the tail: PM 0, 1: t, tc and the step length h (FP64, 24 bytes from the next 8-byte boundary;
  // the last, clipped step of a trajectory with a negative sign); PM 2, 3: th, tl, h, flag (FP32,
  // 16 bytes from the next 16-byte boundary). Slots are padded to 16 bytes and chunk headers are 16
  // bytes, so every slot starts 16-byte aligned for the 16-byte stores and loads below.
  static constexpr int kStateBytes = (F32 ? 4 : 8) * D;
  static constexpr int kTailOff = DF ? (kStateBytes + 15) / 16 * 16 : (kStateBytes + 7) / 8 * 8;
  static constexpr int kSlotBytes = DF ? kTailOff + 16 : (kTailOff + 24 + 15) / 16 * 16;
  static_assert(kTailOff % (DF ? 16 : 8) == 0 && kSlotBytes % 16 == 0 && kChunkHeader % 16 == 0,
                "tape slots must stay aligned");
  static constexpr int kSlotWords = kSlotBytes / 4;
  static_assert(kStateBytes <= kTailOff, "state part of a slot overlaps its tail");
  // checkpoint stride S > 1: chunk = header, kChunk step lengths (FP64, or FP32 in PM 2), then
  // kChunk / S checkpoints. A checkpoint is the state (FP64, or the FP32 high and low parts), the
  // first stage k1 of the step (FSAL: the previous step's last stage, which a recomputation from the
  // state would not reproduce bit for bit), padded to 16 bytes, then the time: t, tc (FP64) or
  // th, tl (FP32 pair, padded to 16 bytes). Not used in PM 3.
  static constexpr int kHBytes = DF ? 4 : 8;
  static constexpr int kCkStateWords = F32 ? 3 * D : 4 * D;
  static constexpr int kCkTimeOff = (4 * kCkStateWords + 15) / 16 * 16;
  static constexpr int kCkBytes = kCkTimeOff + 16;
  static constexpr int kCkWords = kCkBytes / 4;
  static constexpr int kCkOff = kChunkHeader + kChunk * kHBytes;
  static_assert(kCkOff % 16 == 0 && kCkBytes % 16 == 0, "checkpoints must stay 16-byte aligned");

  T y[D];     // state (FP64) / high part (FP32), with its sensitivities when MT > 0
  R ylo[DL];  // low part (FP32)
  T k1[D];    // f(t, y): the first stage of the next attempt
  T p[NPP];
  double t, tc, h, t0, t1, err_prev, sv;  // PM 0, 1 (t0, t1 in all modes)
  double rem_c, hmin_c;  // PM 0: (t1 - t) + tc and 16 eps max(|t|, |t1|), updated when t is
  float remf;            // PM 1: an FP32 lower bound of the exact remainder t1 - t0 - (sum of the steps)
  float marg;            // PM 1: an FP32 upper bound of 2^-47 max(|t0|, |t1|), at least 2^-100
  int32_t kend;          // PM 1: outputs kend.. are all at t1 (or unused): none is due before the last step
  float th, tl, hf, t1h, t1l, svh, svl;   // PM 2, 3
  float atolf, rtolf, lerr_prev;          // PM 1, 2, 3
  long long n;
  int32_t kk, nacc, nrej, status, chunk;
  bool done, failed, rec_ok, sv_ok;

  __device__ __forceinline__ static R cvt(double x) {
    if constexpr (BITS) return narrow_f64(x);
    else return R(x);
  }
  __device__ __forceinline__ R stage_time(double ts) const { return cvt(ts); }

  __device__ __forceinline__ double yval(int i) const {
    if constexpr (F32) return double(val(y[i])) + double(ylo[i]);
    else if constexpr (DD) return to_f64(y[i]);
    else return double(val(y[i]));
  }

  // y(t_k) = hi + lo (FP32 modes) or hi (FP64), and its sensitivities when MT > 0
  template <class L>
  __device__ void write_out(const Problem& pb, int k, const T* hi, const L* lo) {
    double* o = pb.y_out + (n * pb.K + k) * D;
#pragma unroll
    for (int i = 0; i < D; i++) {
      if constexpr (F32) o[i] = double(val(hi[i])) + double(val(lo[i]));
      else if constexpr (DD) o[i] = to_f64(hi[i]);
      else o[i] = double(val(hi[i]));
    }
    if constexpr (MT > 0) {
      double* so = pb.S_out + (n * pb.K + k) * (long long)D * pb.m_total + pb.m_off;
#pragma unroll
      for (int i = 0; i < D; i++)
#pragma unroll
        for (int m = 0; m < MT; m++) {
          if constexpr (F32) so[i * pb.m_total + m] = double(dpart(hi[i], m)) + double(dpart(lo[i], m));
          else so[i * pb.m_total + m] = double(dpart(hi[i], m));
        }
    }
  }
  __device__ void write_nan(const Problem& pb, int k) {
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);
    double* o = pb.y_out + (n * pb.K + k) * D;
#pragma unroll
    for (int i = 0; i < D; i++) o[i] = nanv;
    if constexpr (MT > 0) {
      double* so = pb.S_out + (n * pb.K + k) * (long long)D * pb.m_total + pb.m_off;
#pragma unroll
      for (int i = 0; i < D; i++)
#pragma unroll
        for (int m = 0; m < MT; m++) so[i * pb.m_total + m] = nanv;
    }
  }

  // output k is y0 exactly (and its sensitivity the seed dy0)
  __device__ void write_y0(const Problem& pb, int k, const double* y0d) {
    double* o = pb.y_out + (n * pb.K + k) * D;
#pragma unroll
    for (int i = 0; i < D; i++) o[i] = y0d[i];
    if constexpr (MT > 0) {
      double* so = pb.S_out + (n * pb.K + k) * (long long)D * pb.m_total + pb.m_off;
#pragma unroll
      for (int i = 0; i < D; i++)
#pragma unroll
        for (int m = 0; m < MT; m++)
          so[i * pb.m_total + m] = pb.dy0 ? pb.dy0[(n * D + i) * (long long)pb.m_total + pb.m_off + m] : 0.0;
    }
  }

  // cache the output time of index kk (and whether it is used)
  __device__ __forceinline__ void load_sv(const Problem& pb) {
    if (kk < pb.K) {
      sv_ok = save_valid(pb, n, kk, t0, t1);
      sv = save_at(pb, n, kk);
      if constexpr (DF) split_df(sv, svh, svl);
    }
  }

  // Hairer, Norsett & Wanner I, Sec. II.4 starting step (FP64 norms).
  __device__ double initial_step(const Problem& pb) {
    double sc[D];
    double d0 = 0.0, d1 = 0.0;
#pragma unroll
    for (int i = 0; i < D; i++) {
      const double yi = yval(i);
      sc[i] = pb.atol + pb.rtol * fabs(yi);
      const double r0 = yi / sc[i];
      d0 += r0 * r0;
      const double r1 = double(val(k1[i])) / sc[i];
      d1 += r1 * r1;
    }
    d0 = sqrt(d0 / D);
    d1 = sqrt(d1 / D);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * (d0 / d1);
    if (h0 > t1 - t0) h0 = t1 - t0;
    T y1[D], f1[D];
#pragma unroll
    for (int i = 0; i < D; i++) {
      if constexpr (F32) y1[i] = y[i] + (ylo[i] + R(h0) * k1[i]);
      else y1[i] = y[i] + h0 * k1[i];
    }
    Sys::f(stage_time(t0 + h0), y1, p, f1);
    double d2 = 0.0;
#pragma unroll
    for (int i = 0; i < D; i++) {
      const double r = (double(val(f1[i])) - double(val(k1[i]))) / sc[i];
      d2 += r * r;
    }
    d2 = sqrt(d2 / D) / h0;
    const double dm = d1 > d2 ? d1 : d2;
    const double h1 = (dm <= 1e-15) ? (h0 * 1e-3 > 1e-6 ? h0 * 1e-3 : 1e-6) : pow(0.01 / dm, 1.0 / (Tab::ORDER + 1));
    double hh = 100.0 * h0 < h1 ? 100.0 * h0 : h1;
    if (hh > t1 - t0) hh = t1 - t0;
    return hh;
  }

  // FP32-stage modes: the same starting-step heuristic with FP32 norms, ratio and power, so that
  // starting a trajectory issues no FP64 arithmetic beyond splitting its inputs (on GB300 an FP64
  // instruction costs 64 FP32 ones, and the lanes of a warp wait while one of them starts its
  // trajectory: in a persistent warp some lane starts one every few attempts). tstart: t0 in the
  // stage precision; span: t1 - t0 in FP32.
  __device__ float initial_step_f(R tstart, float span) {
    float sc[D];
    float d0 = 0.0f, d1 = 0.0f;
#pragma unroll
    for (int i = 0; i < D; i++) {
      const float yi = val(y[i]);
      sc[i] = atolf + rtolf * fabsf(yi);
      const float r0 = yi / sc[i];
      d0 += r0 * r0;
      const float r1 = val(k1[i]) / sc[i];
      d1 += r1 * r1;
    }
    d0 = sqrtf(d0 / D);
    d1 = sqrtf(d1 / D);
    float h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * (d0 / d1);
    h0 = fminf(h0, span);
    T y1[D], f1[D];
#pragma unroll
    for (int i = 0; i < D; i++) {
      if constexpr (DD) y1[i] = y[i] + R(h0) * k1[i];
      else y1[i] = y[i] + (ylo[i] + h0 * k1[i]);
    }
    Sys::f(tstart + R(h0), y1, p, f1);
    float d2 = 0.0f;
#pragma unroll
    for (int i = 0; i < D; i++) {
      const float r = (val(f1[i]) - val(k1[i])) / sc[i];
      d2 += r * r;
    }
    d2 = sqrtf(d2 / D) / h0;
    const float dm = fmaxf(d1, d2);
    const float h1 = (dm <= 1e-15f) ? fmaxf(h0 * 1e-3f, 1e-6f) : exp2f(log2f(0.01f / dm) / float(Tab::ORDER + 1));
    return fminf(fminf(100.0f * h0, h1), span);
  }

  __device__ void init(const Problem& pb, long long traj) {
    n = traj;
    status = 0; nacc = 0; nrej = 0; kk = 0;
    done = false; failed = false; rec_ok = true; chunk = -1; sv_ok = false;
    t0 = pb.t0[n];
    t1 = pb.t1[n];
    // (PM 1: tests and conversions on the bit patterns; a lane of a persistent warp starts a
    // trajectory alone, and each FP64-pipe instruction would cost the warp's whole share of the pipe)
    const auto finite = [](double x) {
      if constexpr (BITS) return isfinite_f64_bits(x);
      else return bool(isfinite(x));
    };
    const auto valid = [&](int k) {
      if constexpr (BITS) return save_valid_bits(pb, n, k, t0, t1);
      else return save_valid(pb, n, k, t0, t1);
    };
    bool fin = finite(t0) && finite(t1);
    double y0d[D];
#pragma unroll
    for (int i = 0; i < D; i++) {
      y0d[i] = pb.y0[n * D + i];
      fin = fin && finite(y0d[i]);
      if constexpr (BITS) {
        const float hi = narrow_f64(y0d[i]);
        y[i] = T(hi);
        ylo[i] = narrow_f64(y0d[i] - widen_f32(hi));
      } else if constexpr (F32) {
        const float hi = float(y0d[i]);
        y[i] = T(hi);
        ylo[i] = float(y0d[i] - double(hi));
      } else {
        y[i] = T(y0d[i]);
      }
    }
#pragma unroll
    for (int q = 0; q < NP; q++) {
      const double pv = pb.params[n * NP + q];
      fin = fin && finite(pv);
      p[q] = T(cvt(pv));
    }
    if (NP == 0) p[0] = T(R(0));
    if constexpr (MT > 0) {  // sensitivity seeds: S(t0) = dy0, parameter directions dtheta
#pragma unroll
      for (int i = 0; i < D; i++)
#pragma unroll
        for (int m = 0; m < MT; m++)
          y[i].d[m] = pb.dy0 ? R(pb.dy0[(n * D + i) * (long long)pb.m_total + pb.m_off + m]) : R(0);
#pragma unroll
      for (int q = 0; q < NP; q++)
#pragma unroll
        for (int m = 0; m < MT; m++)
          p[q].d[m] = pb.dp ? R(pb.dp[(n * NP + q) * (long long)pb.m_total + pb.m_off + m]) : R(0);
    }
    prep_params<Sys>(p);  // derived constants carry the parameter directions too
    if (!fin) {
      status = ST_NONFINITE;
      failed = true;
      done = true;
      return;
    }
    bool empty;
    if constexpr (BITS) empty = le_f64_bits(t1, t0);
    else empty = !(t1 > t0);
    if (empty) {  // empty or reversed interval: every output is y0 (and S = dy0)
      status = ST_EMPTY;
      for (int k = 0; k < pb.K; k++) write_y0(pb, k, y0d);
      done = true;
      return;
    }
    if constexpr (BITS) kend = 0;
    for (int k = 0; k < pb.K; k++) {
      if (!valid(k)) {
        status |= ST_SAVEAT_OUTSIDE;
        write_nan(pb, k);
      } else if constexpr (BITS) {
        if (!eq_f64_bits(save_at(pb, n, k), t1)) kend = k + 1;
      }
    }
    const auto at_t0 = [&](int k) {
      if constexpr (BITS) return eq_f64_bits(save_at(pb, n, k), t0);
      else return save_at(pb, n, k) == t0;
    };
    while (kk < pb.K && (!valid(kk) || at_t0(kk))) {
      if (valid(kk)) write_y0(pb, kk, y0d);
      kk++;
    }
    if (pb.tape.emit) {  // checkpointed tape: outputs at t0 and unused ones are known now
      for (int k = 0; k < pb.K; k++) {
        if (!valid(k)) pb.tape.emit[n * pb.K + k] = kEmitUnused;
        else if (k < kk) pb.tape.emit[n * pb.K + k] = kEmitT0;
      }
    }
    t = t0;
    tc = 0.0;
    rem_c = t1 - t0;
    load_sv(pb);
    Sys::f(stage_time(t0), y, p, k1);
    time_cache();
    err_prev = 1.0;
    lerr_prev = 0.0f;
    if constexpr (BITS) {
      atolf = narrow_f64(pb.atol);
      rtolf = narrow_f64(pb.rtol);
      // the bounds of the step-length test's fast path (attempt()); 2^-48 max(|t0|, |t1|) is 0
      // below the normal range, and rounding to FP32 costs at most 2^-24 of it
      marg = fmaxf(__fmul_ru(narrow_f64(max_abs_2m48_bits(t0, t1)), 2.0f + 0x1p-19f), 0x1p-100f);
      remf = remainder_bound(rem_c);
      // the caller's first step (h0 > 0) at most the interval, else the starting-step heuristic;
      // rem_c = t1 - t0 > 0 here
      const long long hb = __double_as_longlong(pb.h0);
      const bool given = hb > 0LL && hb <= 0x7ff0000000000000LL;
      h = given ? (le_nonneg_f64(pb.h0, rem_c) ? pb.h0 : rem_c)
                : widen_f32(initial_step_f(narrow_f64(t0), narrow_f64(rem_c)));
    } else if constexpr (DF) {
      atolf = float(pb.atol);
      rtolf = float(pb.rtol);
      split_df(t0, th, tl);
      split_df(t1, t1h, t1l);
      hf = pb.h0 > 0.0 ? float(pb.h0 < t1 - t0 ? pb.h0 : t1 - t0) : initial_step_f(R(th) + R(tl), float(t1 - t0));
      h = double(hf);
    } else {
      atolf = float(pb.atol);
      rtolf = float(pb.rtol);
      h = pb.h0 > 0.0 ? (pb.h0 < t1 - t0 ? pb.h0 : t1 - t0) : initial_step(pb);
    }
  }

  // Stages of one step of length hh from (tt, y): Eq. rk. k[0] = k1 on entry.
  // Y[j] receives the state at which stage j was evaluated (Y[0] = y). SAVE (FP32 reverse pass):
  // f_save leaves stage j's Jacobian factors at shared address sl + j * SaveQ * st for its VJP.
  template <bool SAVE = false>
  __device__ __forceinline__ void stages(double tt, double hh, T (*k)[D], T (*Y)[D], int nst, unsigned sl = 0,
                                         unsigned st = 0) const {
    const R hr = cvt(hh);
    [[maybe_unused]] R hr2;
    [[maybe_unused]] T hv[DH];
    if constexpr (RKN) {
      hr2 = hr * hr;
#pragma unroll
      for (int i = 0; i < DH; i++) hv[i] = hr * y[DH + i];
    }
#pragma unroll
    for (int i = 0; i < D; i++) { k[0][i] = k1[i]; if (Y) Y[0][i] = y[i]; }
#pragma unroll
    for (int j = 1; j < S; j++) {
      if (j < nst) {
        T Yj[D];
        if constexpr (RKN) {
          nystrom_stage(j, hr2, hv, k, Yj);
        } else {
#pragma unroll
          for (int i = 0; i < D; i++) {
            T acc = T(R(0));
#pragma unroll
            for (int l = 0; l < j; l++)
              if (Tab::a(j, l) != 0.0) acc = fmadd(R(Tab::a(j, l)), k[l][i], acc);
            if constexpr (F32 || DD) Yj[i] = fmadd(hr, acc, y[i]);
            else Yj[i] = fmadd(hh, acc, y[i]);
          }
        }
        if (Y)
#pragma unroll
          for (int i = 0; i < D; i++) Y[j][i] = Yj[i];
        if constexpr (SAVE) {
          constexpr int Q = SaveQ<Sys>::value;
          if constexpr (DF) Sys::f_save(R(tt) + R(Tab::c(j)) * hr, Yj, p, k[j], sl + unsigned(j * Q) * st, st);
          else Sys::f_save(stage_time(tt + Tab::c(j) * hh), Yj, p, k[j], sl + unsigned(j * Q) * st, st);
        } else if constexpr (DF) {
          Sys::f(R(tt) + R(Tab::c(j)) * hr, Yj, p, k[j]);
        } else {
          Sys::f(stage_time(tt + Tab::c(j) * hh), Yj, p, k[j]);
        }
      }
    }
  }

  // Solution at tt + sig*hh inside the accepted step just taken (Eq. dense; Verner 7: shortened
  // step from the start of the step). k holds the step's stages.
  __device__ void dense_point(double tt, double hh, R sig, T (*k)[D], T* hi, T* lo) const {
    if constexpr (RKN) {
      // Nystrom form: sum_j w_j V_j = (sum_j w_j) v + h sum_m (w A)_m a_m, from the accelerations
      R w[S], wa[S];
      Tab::dense(sig, w);
      const R hr = R(hh);
      R ws = R(0);
#pragma unroll
      for (int j = 0; j < S; j++) ws = ws + w[j];
#pragma unroll
      for (int m = 0; m < S; m++) {
        wa[m] = R(0);
#pragma unroll
        for (int j = m + 1; j < S; j++)
          if (Tab::a(j, m) != 0.0) wa[m] = wa[m] + w[j] * R(Tab::a(j, m));
      }
#pragma unroll
      for (int i = 0; i < DH; i++) {
        T ax = T(R(0)), av = T(R(0));
#pragma unroll
        for (int m = 0; m < S; m++) {
          ax = ax + wa[m] * k[m][DH + i];
          av = av + w[m] * k[m][DH + i];
        }
        hi[i] = y[i];
        lo[i] = ylo[i] + hr * (ws * y[DH + i] + hr * ax);
        hi[DH + i] = y[DH + i];
        lo[DH + i] = ylo[DH + i] + hr * av;
      }
    } else if constexpr (Tab::DENSE_POLY) {
      R w[S];
      Tab::dense(sig, w);
      const R hr = R(hh);
#pragma unroll
      for (int i = 0; i < D; i++) {
        T acc = T(R(0));
#pragma unroll
        for (int j = 0; j < S; j++) acc = acc + w[j] * k[j][i];
        if constexpr (F32) { hi[i] = y[i]; lo[i] = ylo[i] + hr * acc; }
        else if constexpr (DD) { hi[i] = y[i] + hr * acc; lo[i] = T(R(0)); }
        else { hi[i] = y[i] + hh * acc; lo[i] = T(R(0)); }
      }
    } else {
      T ks[S][D];
      const double hs = to_f64(sig) * hh;
      stages(tt, hs, ks, nullptr, Tab::NREV);
      const R hr = R(hs);
#pragma unroll
      for (int i = 0; i < D; i++) {
        T acc = T(R(0));
#pragma unroll
        for (int j = 0; j < Tab::NREV; j++)
          if (Tab::b(j) != 0.0) acc = acc + R(Tab::b(j)) * ks[j][i];
        if constexpr (F32) { hi[i] = y[i]; lo[i] = ylo[i] + hr * acc; }
        else if constexpr (DD) { hi[i] = y[i] + hr * acc; lo[i] = T(R(0)); }
        else { hi[i] = y[i] + hs * acc; lo[i] = T(R(0)); }
      }
    }
  }

  // the words of the slot of the step just accepted (state at its start, padding, tail)
  __device__ void slot_words(bool last, R hstep, uint32_t* w) const {
    if constexpr (F32) {
#pragma unroll
      for (int i = 0; i < D; i++) w[i] = __float_as_uint(val(y[i]));
    } else if constexpr (DD) {
#pragma unroll
      for (int i = 0; i < D; i++) { w[2 * i] = __float_as_uint(y[i].hi); w[2 * i + 1] = __float_as_uint(y[i].lo); }
    } else {
#pragma unroll
      for (int i = 0; i < D; i++) {
        const double v = val(y[i]);
        w[2 * i] = uint32_t(__double2loint(v));
        w[2 * i + 1] = uint32_t(__double2hiint(v));
      }
    }
#pragma unroll
    for (int i = kStateBytes / 4; i < kTailOff / 4; i++) w[i] = 0u;
    constexpr int T0 = kTailOff / 4;
    if constexpr (DF) {
      w[T0] = __float_as_uint(th);
      w[T0 + 1] = __float_as_uint(tl);
      w[T0 + 2] = __float_as_uint(val(hstep));
      w[T0 + 3] = __float_as_uint(last ? 1.0f : 0.0f);
    } else {
      const double tv[3] = {t, tc, h};
#pragma unroll
      for (int q = 0; q < 3; q++) {
        w[T0 + 2 * q] = uint32_t(__double2loint(tv[q]));
        w[T0 + 2 * q + 1] = uint32_t(__double2hiint(tv[q]));
      }
      if (last) w[T0 + 5] |= 0x80000000u;  // the sign of h marks the last step
#pragma unroll
      for (int i = T0 + 6; i < kSlotWords; i++) w[i] = 0u;
    }
  }
  // A slot is written as kSlotBytes / 16 stores of 16 bytes, assembled in registers (state, zero
  // padding, tail). Measured on the 2^20-orbit Milky-Way forward: 35.6 ms, against 38.3 ms for the
  // same data written per field (three 8-byte stores for the six FP32 components, one for the tail),
  // and against 38.3 ms for whole 32-byte sectors written in slot pairs through a shared-memory
  // stash, although that removes the 34 GB of DRAM reads that completing partly written sectors
  // costs: the stores are bound by issue, not by DRAM.
  __device__ void record_slot(const Problem& pb, bool last, R hstep) {
    if constexpr (MT == 0) {  // the tape is recorded by the solve without sensitivities
    const int a = nacc - 1;  // index of the step just accepted
    if (!rec_ok) return;
    if (a >= pb.tape.cap) { rec_ok = false; return; }
    const int o = a % kChunk;
    if (o == 0) {
      const unsigned long long idx = atomicAdd(pb.tape.pool_next, 1ULL);
      if (idx >= (unsigned long long)pb.tape.pool_chunks) { rec_ok = false; return; }
      long long* hdr = reinterpret_cast<long long*>(pb.tape.pool + (long long)idx * pb.tape.chunk_bytes);
      hdr[0] = chunk;
      chunk = int32_t(idx);
    }
    if constexpr (!DD) {
      if (pb.tape.stride > 1) {
        record_ck(pb, o, a, last);
        return;
      }
    }
    // slots start 16-byte aligned (16-byte header, slots of multiples of 16 bytes)
    uint4* s4 = reinterpret_cast<uint4*>(pb.tape.pool + (long long)chunk * pb.tape.chunk_bytes + kChunkHeader +
                                         (long long)o * kSlotBytes);
    uint32_t w[kSlotWords];
    slot_words(last, hstep, w);
#pragma unroll
    for (int q = 0; q < kSlotWords / 4; q++) s4[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
  }

  // Checkpoint stride S > 1: the length of the step just accepted (chunk position o, trajectory
  // step a; negative for the last, clipped step) and, every S steps, the checkpoint of its start:
  // state, first stage and time, assembled in registers and written as 16-byte stores.
  __device__ void record_ck(const Problem& pb, int o, int a, bool last) {
    unsigned char* base = pb.tape.pool + (long long)chunk * pb.tape.chunk_bytes;
    if constexpr (DF) reinterpret_cast<float*>(base + kChunkHeader)[o] = last ? -hf : hf;
    else reinterpret_cast<double*>(base + kChunkHeader)[o] = last ? neg_f64_bits(h) : h;
    if (a % pb.tape.stride != 0) return;
    uint32_t w[kCkWords];
    if constexpr (F32) {
#pragma unroll
      for (int i = 0; i < D; i++) {
        w[i] = __float_as_uint(val(y[i]));
        w[D + i] = __float_as_uint(ylo[i]);
        w[2 * D + i] = __float_as_uint(val(k1[i]));
      }
    } else {
#pragma unroll
      for (int i = 0; i < D; i++) {
        const double v = val(y[i]), kv = val(k1[i]);
        w[2 * i] = uint32_t(__double2loint(v));
        w[2 * i + 1] = uint32_t(__double2hiint(v));
        w[2 * D + 2 * i] = uint32_t(__double2loint(kv));
        w[2 * D + 2 * i + 1] = uint32_t(__double2hiint(kv));
      }
    }
#pragma unroll
    for (int i = kCkStateWords; i < kCkTimeOff / 4; i++) w[i] = 0u;
    constexpr int T0 = kCkTimeOff / 4;
    if constexpr (DF) {
      w[T0] = __float_as_uint(th);
      w[T0 + 1] = __float_as_uint(tl);
      w[T0 + 2] = 0u;
      w[T0 + 3] = 0u;
    } else {
      w[T0] = uint32_t(__double2loint(t));
      w[T0 + 1] = uint32_t(__double2hiint(t));
      w[T0 + 2] = uint32_t(__double2loint(tc));
      w[T0 + 3] = uint32_t(__double2hiint(tc));
    }
    uint4* s4 = reinterpret_cast<uint4*>(base + kCkOff + (long long)(o / pb.tape.stride) * kCkBytes);
#pragma unroll
    for (int q = 0; q < kCkWords / 4; q++) s4[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
  }

  __device__ void fail(int32_t bit) {
    status |= bit;
    failed = true;
    done = true;
  }

  // the interval closed without a clipped last step: the remaining outputs are the state
  __device__ void close_interval(const Problem& pb) {
    while (kk < pb.K) {
      if (save_valid(pb, n, kk, t0, t1)) {
        write_out(pb, kk, y, ylo);
        if (pb.tape.emit) pb.tape.emit[n * pb.K + kk] = nacc;
      }
      kk++;
    }
    done = true;
  }

  // safety * ||e||^-beta1 * err_prev^beta2 clamped to [alpha_min, alpha_max] (Eq. controller).
  // The FP32 modes take the power in FP32 from log2 ||e|| (||e|| = 0 gives alpha_max, inf alpha_min).
  __device__ __forceinline__ float factor_f(const Problem& pb, float lerr) const {
    float lf = -pb.fbeta1 * lerr;
    if (pb.fbeta2 != 0.0f) lf += pb.fbeta2 * lerr_prev;
    const float fac = pb.fsafety * exp2f(lf);
    return fminf(fmaxf(fac, pb.falpha_min), pb.falpha_max);
  }
  __device__ __forceinline__ double factor_d(const Problem& pb, double err) const {
    double fac = pb.safety * pow(err, -pb.beta1) * (pb.beta2 != 0.0 ? pow(err_prev, pb.beta2) : 1.0);
    if (fac > pb.alpha_max) fac = pb.alpha_max;
    if (fac < pb.alpha_min) fac = pb.alpha_min;
    return fac;
  }

  // Stages 2..S of a step of length h (hr in the stage precision) from the current state, Eq. rk
  // (k[0] = k1), and the new state y + h sum_j b_j k_j: for FSAL pairs in FP64 and df64 the last
  // stage state itself; in the FP32 modes the compensated update of the (hi, lo) pair. Shared by
  // attempt() and replay_step(), so that the reverse pass's replay of a checkpoint segment
  // reproduces the forward's states bit for bit.
  __device__ __forceinline__ void step_core(R hr, T (*k)[D], T* ynew, R* ynlo) const {
    if constexpr (RKN) {
      step_core_nystrom(hr, k, ynew, ynlo);
      return;
    }
    T Ylast[D];
#pragma unroll
    for (int i = 0; i < D; i++) k[0][i] = k1[i];
#pragma unroll
    for (int j = 1; j < S; j++) {
      T Yj[D];
#pragma unroll
      for (int i = 0; i < D; i++) {
        T acc = T(R(0));
#pragma unroll
        for (int l = 0; l < j; l++)
          if (Tab::a(j, l) != 0.0) acc = fmadd(R(Tab::a(j, l)), k[l][i], acc);
        // FP32 modes: the stage state is y_hi + h sum a k; the low part of the state only enters the
        // update of the state itself (below), its effect on a stage is below the stage's FP32 rounding
        if constexpr (F32 || DD) Yj[i] = fmadd(hr, acc, y[i]);
        else Yj[i] = fmadd(h, acc, y[i]);
        if (j == S - 1) Ylast[i] = Yj[i];
      }
      if constexpr (DF) Sys::f((R(th) + R(tl)) + R(Tab::c(j)) * hr, Yj, p, k[j]);
      else Sys::f(stage_time(t + Tab::c(j) * h), Yj, p, k[j]);
    }
#pragma unroll
    for (int i = 0; i < D; i++) {
      if constexpr (Tab::FSAL && !F32) {
        ynew[i] = Ylast[i];
      } else {
        T acc = T(R(0));
#pragma unroll
        for (int j = 0; j < S; j++)
          if (Tab::b(j) != 0.0) acc = fmadd(R(Tab::b(j)), k[j][i], acc);
        if constexpr (F32) {
          state_update(y[i], fmadd(hr, acc, T(ylo[i])), ynew[i], ynlo[i]);
        } else if constexpr (DD) {
          ynew[i] = fmadd(hr, acc, y[i]);
        } else {
          ynew[i] = fmadd(h, acc, y[i]);
        }
      }
    }
  }
  // The stage position X_j = x + c'_j h v + h^2 sum_m (A^2)_jm a_m of the Nystrom form (c'_j the
  // row sum of A; hv = h v); the stage's velocity slot keeps v, which the acceleration does not read.
  __device__ __forceinline__ void nystrom_stage(int j, R hr2, const T* hv, T (*k)[D], T* Yj) const {
#pragma unroll
    for (int i = 0; i < DH; i++) {
      T xs = y[i];
      if (j >= 2) {
        T acc = T(R(0));
#pragma unroll
        for (int m = 0; m < j - 1; m++)
          if (NY::aa(j, m) != 0.0) acc = fmadd(R(NY::aa(j, m)), k[m][DH + i], acc);
        xs = fmadd(hr2, acc, xs);
      }
      Yj[i] = fmadd(R(NY::row(j)), hv[i], xs);
      Yj[DH + i] = y[DH + i];
    }
  }
  // step_core in Nystrom form: the stages of the general form with k[j] = f(X_j), of which only the
  // accelerations a_j are used; the new state x + h (v + h sum_m (bA)_m a_m), v + h sum_j b_j a_j,
  // each an increment of the compensated pair as in the general form
  __device__ __forceinline__ void step_core_nystrom(R hr, T (*k)[D], T* ynew, R* ynlo) const {
    const R hr2 = hr * hr;
    T hv[DH];
#pragma unroll
    for (int i = 0; i < DH; i++) hv[i] = hr * y[DH + i];
#pragma unroll
    for (int i = 0; i < D; i++) k[0][i] = k1[i];
#pragma unroll
    for (int j = 1; j < S; j++) {
      T Yj[D];
      nystrom_stage(j, hr2, hv, k, Yj);
      if constexpr (DF) Sys::f((R(th) + R(tl)) + R(Tab::c(j)) * hr, Yj, p, k[j]);
      else Sys::f(stage_time(t + Tab::c(j) * h), Yj, p, k[j]);
    }
#pragma unroll
    for (int i = 0; i < DH; i++) {
      T ax = T(R(0)), av = T(R(0));
#pragma unroll
      for (int m = 0; m < S; m++) {
        if (NY::ba(m) != 0.0) ax = fmadd(R(NY::ba(m)), k[m][DH + i], ax);
        if (Tab::b(m) != 0.0) av = fmadd(R(Tab::b(m)), k[m][DH + i], av);
      }
      state_update(y[i], fmadd(hr, fmadd(hr, ax, y[DH + i]), T(ylo[i])), ynew[i], ynlo[i]);
      state_update(y[DH + i], fmadd(hr, av, T(ylo[DH + i])), ynew[DH + i], ynlo[DH + i]);
    }
  }
  // the state after an accepted step (FSAL pairs: its first stage is the step's last one)
  __device__ __forceinline__ void take_state(T (*k)[D], const T* ynew, const R* ynlo) {
#pragma unroll
    for (int i = 0; i < D; i++) {
      y[i] = ynew[i];
      if constexpr (F32) ylo[i] = ynlo[i];
      if constexpr (Tab::FSAL) k1[i] = k[S - 1][i];
    }
  }
  // PM 1: an FP32 number below the FP64 remainder rem by more than that remainder's error against
  // the exact t1 - t0 - (sum of the steps): rem rounded to FP32 (at most FLT_MAX, which a remainder
  // that rounds to infinity exceeds), less 2^-20 of itself and marg, rounded down
  __device__ __forceinline__ float remainder_bound(double rem) const {
    return __fmaf_rd(fminf(narrow_f64(rem), FLT_MAX), 1.0f - 0x1p-20f, -marg);
  }
  // the quantities of the step-length tests that change only with the time (PM 0): the remaining
  // interval and the step-size floor of the underflow test. PM 1 forms them in attempt(), only when
  // its FP32 bound does not settle the tests.
  __device__ __forceinline__ void time_cache() {
    if constexpr (!F32 && !DF) {
      rem_c = (t1 - t) + tc;
      const double tm = fabs(t) > fabs(t1) ? fabs(t) : fabs(t1);
      hmin_c = 16.0 * DBL_EPSILON * tm;
    }
  }
  // the time after an accepted step that is not the last (Kahan summation, or the error-free
  // advance of the FP32 time pair), then the next first stage of pairs without FSAL
  __device__ __forceinline__ void next_time() {
    if constexpr (DF) {
      float s, e2;  // (th, tl) += hf without rounding error
      two_sum(th, hf, s, e2);
      const float l = tl + e2;
      th = s + l;
      tl = l - (th - s);
      if constexpr (!Tab::FSAL) Sys::f(R(th) + R(tl), y, p, k1);
    } else {
      const double yk = h - tc;  // Kahan summation of the time
      const double tn = t + yk;
      tc = (tn - t) - yk;
      t = tn;
      if constexpr (!Tab::FSAL) Sys::f(stage_time(t), y, p, k1);
    }
  }
  // One accepted step of recorded length hrec (FP64, or the FP32 step of PM 2) from the current
  // state, time and first stage, with the arithmetic of attempt() and no error estimate: the reverse
  // pass's replay of a checkpoint segment. Never the last, clipped step of a trajectory.
  __device__ __forceinline__ void replay_step(double hrec) {
    R hr;
    if constexpr (DF) {
      hf = float(hrec);
      hr = hf;
    } else {
      h = hrec;
      hr = cvt(h);
    }
    T k[S][D];
    T ynew[D];
    R ynlo[DL];
    step_core(hr, k, ynew, ynlo);
    take_state(k, ynew, ynlo);
    next_time();
  }

  // One step attempt.
  __device__ void attempt(const Problem& pb) {
    // ---- step length: land exactly on t1, or stop on underflow / too many attempts
    bool last = false;
    R hr;
    if constexpr (DF) {
      const float rem = (t1h - th) + (t1l - tl);
      if (!(rem > 0.0f)) { close_interval(pb); return; }
      if (nacc + nrej >= pb.max_steps) { fail(ST_MAX_STEPS); return; }
      if (hf * (1.0f + 4.0f * FLT_EPSILON) >= rem) {
        hf = rem;
        last = true;
      } else {
        const float tm = fmaxf(fabsf(th), fabsf(t1h));
        if (!(hf >= 16.0f * kEps48 * tm)) { fail(isnan(hf) ? (ST_H_UNDERFLOW | ST_NONFINITE) : ST_H_UNDERFLOW); return; }
      }
      hr = hf;
      // df64: the last step spans the exact remainder t1 - t (an FP32 length would leave the final
      // state one FP32 rounding of the step short of t1, far above df64's resolution)
      if constexpr (DD)
        if (last) hr = (R(t1h) + R(t1l)) - (R(th) + R(tl));
    } else if constexpr (F32) {
      // PM 1: the same tests with the FP64 values compared as bit patterns (non-negative, NaN
      // apart), the last-step threshold eight units in the last place below the remainder (where
      // rem (1 - 2^-50) lies, 4 to 8 units below it) and 16 eps max(|t|, |t1|) formed by the exponent
      // field. The remainder itself, two FP64 additions, is formed only where the FP32 bound remf
      // does not settle the tests: with remf <= t1 - t0 - (sum of the steps) and h <= hr (1 + 2^-24),
      // hr >= marg and hr (1 + 2^-10) + marg < remf give rem > 0, h < rem - 8 ulp and h above the
      // floor, since the Kahan sum and the remainder's two roundings err by less than 2^-51 max(|t0|,
      // |t1|) + 2^-52 rem. The decisions, and h, are those of the FP64 tests in every case.
      hr = cvt(h);
      if (hr >= marg && __fmaf_ru(hr, 1.0f + 0x1p-10f, marg) < remf) {
        if (nacc + nrej >= pb.max_steps) { fail(ST_MAX_STEPS); return; }
      } else {
        const double rem = (t1 - t) + tc;
        const long long rb = __double_as_longlong(rem);
        if (rb <= 0LL) { close_interval(pb); return; }
        if (nacc + nrej >= pb.max_steps) { fail(ST_MAX_STEPS); return; }
        if (isnan_f64_bits(h)) { fail(ST_H_UNDERFLOW | ST_NONFINITE); return; }
        if (le_nonneg_f64(__longlong_as_double(rb > 8LL ? rb - 8LL : 0LL), h)) {
          h = rem;
          hr = cvt(h);
          last = true;
        } else if (!le_nonneg_f64(max_abs_2m48_bits(t, t1), h)) {
          fail(ST_H_UNDERFLOW);
          return;
        }
        remf = remainder_bound(rem);
      }
    } else {
      if (rem_c <= 0.0) { close_interval(pb); return; }
      if (nacc + nrej >= pb.max_steps) { fail(ST_MAX_STEPS); return; }
      if (h * (1.0 + 4.0 * DBL_EPSILON) >= rem_c) {
        h = rem_c;
        last = true;
      } else if (!(h >= hmin_c)) {
        fail(isnan(h) ? (ST_H_UNDERFLOW | ST_NONFINITE) : ST_H_UNDERFLOW);
        return;
      }
      hr = R(h);
    }
    // ---- stages 2..S and the new state, Eq. rk
    T k[S][D];
    T ynew[D];
    R ynlo[DL];
    step_core(hr, k, ynew, ynlo);
    // ---- error estimate e = h sum (b_j - bhat_j) k_j and its scaled RMS norm, Eq. errnorm:
    // ||e|| = sqrt(sq / d), sq = sum_i (e_i / s_i)^2, s_i = atol + rtol max(|y_i|, |y+_i|)
    bool accept, bad;
    double err = 0.0;
    float lerr = 0.0f;
    if constexpr (PM == 0) {
      double sq = 0.0;
#pragma unroll
      for (int i = 0; i < D; i++) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < S; j++)
          if (Tab::bt(j) != 0.0) acc = acc + Tab::bt(j) * val(k[j][i]);
        const double e = h * acc;
        const double a = fabs(val(y[i])), b = fabs(val(ynew[i]));
        const double sc = pb.atol + pb.rtol * (a > b ? a : b);
        const double r = e / sc;
        sq += r * r;
      }
      err = sqrt(sq / D);
      accept = err <= 1.0;
      bad = isnan(err);
    } else if constexpr (DD) {
      // the weighted stage sum nearly cancels (it is the local error): it is formed in df64 and
      // rounded to FP32 only afterwards; scale, ratio and sum of squares are FP32 as in mode 2
      float sq = 0.0f;
#pragma unroll
      for (int i = 0; i < D; i++) {
        R acc = R(0);
#pragma unroll
        for (int j = 0; j < S; j++)
          if (Tab::bt(j) != 0.0) acc = acc + R(Tab::bt(j)) * k[j][i];
        const float e = val(hr * acc);
        const float a = fabsf(val(y[i])), b = fabsf(val(ynew[i]));
        const float sc = atolf + rtolf * (a > b ? a : b);
        const float r = __fdividef(e, sc);
        sq += r * r;
      }
      accept = sq <= float(D);
      lerr = 0.5f * (__log2f(sq) - log2f(float(D)));
      bad = isnan(sq);
    } else {
      // PM 1 accumulates the squares in FP64 (each FP32 ratio widened exactly, by integer
      // instructions, then one FP64 multiply-add), PM 2 in FP32. PM 1 then takes the accept test,
      // the NaN test and log2 ||e|| for the controller's power from the FP64 sum's bits, so that the
      // FP64 pipe carries only the accumulation itself.
      using Acc = typename std::conditional<PM == 1, double, float>::type;
      Acc sq = Acc(0);
#pragma unroll
      for (int i = 0; i < D; i++) {
        R acc = R(0);
        if (RKN && i < DH) {
          // Nystrom form: the position error h sum_j bt_j V_j = h^2 sum_m (bt A)_m a_m (sum_j bt_j = 0)
#pragma unroll
          for (int m = 0; m < S; m++)
            if (NY::bta(m) != 0.0) acc = acc + R(NY::bta(m)) * val(k[m][DH + i]);
          acc = hr * acc;
        } else {
#pragma unroll
          for (int j = 0; j < S; j++)
            if (Tab::bt(j) != 0.0) acc = acc + R(Tab::bt(j)) * val(k[j][i]);
        }
        const R e = hr * acc;
        const R a = fabsf(val(y[i])), b = fabsf(val(ynew[i]));
        const R sc = atolf + rtolf * (a > b ? a : b);
        if constexpr (PM == 1) {
          const double r = widen_f32(__fdividef(e, sc));
          sq = fma(r, r, sq);
        } else {
          const Acc r = Acc(__fdividef(e, sc));
          sq += r * r;
        }
      }
      if constexpr (PM == 1) {
        accept = le_nonneg_f64(sq, double(D));
        lerr = 0.5f * (log2_f64_f32(sq) - log2f(float(D)));  // log2 ||e||
        bad = isnan_f64_bits(sq);
      } else {
        accept = sq <= Acc(D);
        lerr = 0.5f * (__log2f(float(sq)) - log2f(float(D)));  // log2 ||e||
        bad = isnan(sq);
      }
    }
    if (accept) {
      nacc += 1;
      if (pb.record) record_slot(pb, last, hr);
      // ---- outputs inside (t, t + h] (Eq. dense), or the new state itself at t1. PM 1 skips the
      // scan while every pending output is at t1 and the step is not the last (an integer test; the
      // FP64 distance to the pending output is formed only where an output may be due)
      bool scan = true;
      if constexpr (BITS) scan = last || kk < kend;
      while (scan && kk < pb.K) {
        if (!sv_ok) { kk++; load_sv(pb); continue; }
        bool at_end, inside;
        double dk = 0.0;
        if constexpr (DF) {
          at_end = last && svh == t1h && svl == t1l;
          inside = last || ((svh - th) + (svl - tl)) <= hf;
        } else if constexpr (F32) {  // PM 1: h > 0, so the bit patterns order as the values
          const bool at_t1 = __double_as_longlong(sv) == __double_as_longlong(t1);
          at_end = last && at_t1;
          if (at_t1) {
            inside = last;  // an output at t1 falls in the last step only
          } else {
            dk = (sv - t) + tc;
            inside = last || __double_as_longlong(dk) <= __double_as_longlong(h);
          }
        } else {
          at_end = last && sv == t1;
          inside = last || ((sv - t) + tc) <= h;
        }
        if (at_end) {
          if constexpr (F32) write_out(pb, kk, ynew, ynlo);
          else write_out(pb, kk, ynew, ynew);
        } else if (inside) {
          // the fraction of the step at the output time, only for an output inside the step (in
          // FP64 modes a division)
          R sig;
          if constexpr (DF) {
            if constexpr (DD) {  // the fraction of the step in df64, from the exact time pairs
              sig = ((R(svh) + R(svl)) - (R(th) + R(tl))) / hr;
              if (val(sig) > 1.0f) sig = R(1.0f);
              if (val(sig) < 0.0f) sig = R(0.0f);
            } else {
              sig = fminf(fmaxf(__fdividef((svh - th) + (svl - tl), hf), 0.0f), 1.0f);
            }
          } else {
            double sg;
            if constexpr (F32) sg = dk / h;
            else sg = ((sv - t) + tc) / h;
            if (sg > 1.0) sg = 1.0;
            if (sg < 0.0) sg = 0.0;
            sig = R(sg);
          }
          T hi[D], lo[D];
          if constexpr (DD) dense_point(double(th) + double(tl), to_f64(hr), sig, k, hi, lo);
          else if constexpr (DF) dense_point(double(th) + double(tl), double(hf), sig, k, hi, lo);
          else dense_point(t, h, sig, k, hi, lo);
          write_out(pb, kk, hi, lo);
        } else {
          break;
        }
        if (pb.tape.emit) pb.tape.emit[n * pb.K + kk] = nacc - 1;
        kk++;
        load_sv(pb);
      }
      take_state(k, ynew, ynlo);
      if (last) {
        done = true;
        if constexpr (DF) { th = t1h; tl = t1l; }
        else { t = t1; tc = 0.0; }
      } else if constexpr (DF) {
        next_time();
        hf = hf * factor_f(pb, lerr);
        lerr_prev = lerr > -13.287712f ? lerr : -13.287712f;  // log2(1e-4)
      } else {
        next_time();
        time_cache();
        // PM 1: the bound moves down by at least the step (hr (1 + 2^-22) >= h; marg covers an h
        // below the FP32 normal range), rounded down
        if constexpr (BITS) remf = __fmaf_rd(-fmaxf(hr, marg), 1.0f + 0x1p-22f, remf);
        if constexpr (!F32) {  // (PM 1: the new h after both branches, below)
          h = h * factor_d(pb, err);
          err_prev = err > 1e-4 ? err : 1e-4;
        }
      }
    } else {
      nrej += 1;
      if constexpr (DF) hf = hf * (bad ? pb.falpha_min : factor_f(pb, lerr));
      else if constexpr (!F32) h = h * (bad ? pb.alpha_min : factor_d(pb, err));
      err_prev = 1.0;
      if constexpr (DF) lerr_prev = 0.0f;
    }
    if constexpr (F32 && !DF) {
      // PM 1: the step-size update of both branches (an accepted step other than the last, and a
      // rejected one) as one FP64 multiply after them, so that a warp whose lanes went both ways
      // issues it once (the factor picked by an integer select of the two FP64 bit patterns). The
      // factor takes the previous step's log2 ||e||, replaced only after it.
      if (!done) {
        const long long fb = bad ? __double_as_longlong(pb.alpha_min)
                                 : __double_as_longlong(widen_f32(factor_f(pb, lerr)));
        h = h * __longlong_as_double(fb);
      }
      lerr_prev = accept ? (lerr > -13.287712f ? lerr : -13.287712f) : 0.0f;
    }
  }

  // ---- prepared start: the state init() leaves, as one row of 32-bit words. Layout: y (the FP32
  // high parts, or FP64), the FP32 low parts (FP32 modes), k1, theta with its prepared constants,
  // then PM 0: h, rem_c, hmin_c (FP64), 0; PM 1: h (FP64), remf, marg, 0 (4 words); PM 2: h (FP64),
  // th, tl, hf, t1h, t1l, svh, svl; then
  // atolf, rtolf, status, kk, kend, flags (bit 0: sv_ok, bit 1: done at start). Not for PM 3 or
  // with sensitivities (MT > 0): those start in place.
  static constexpr int kRW = sizeof(R) / 4;
  static constexpr int kSY = 0, kSLO = kSY + D * kRW, kSK1 = kSLO + (F32 ? D : 0), kSP = kSK1 + D * kRW;
  static constexpr int kST = kSP + NPP * kRW;
  static constexpr int kSTail = kST + (DF ? 9 : 8);
  static constexpr int kStartWords = (kSTail + 6 + 3) / 4 * 4;
  static constexpr int kStartBytes = 4 * kStartWords;

  __device__ static void put_r(uint32_t* w, int o, float v) { w[o] = __float_as_uint(v); }
  __device__ static void put_r(uint32_t* w, int o, double v) {
    w[o] = uint32_t(__double2loint(v));
    w[o + 1] = uint32_t(__double2hiint(v));
  }
  __device__ static void get_r(const uint32_t* w, int o, float& v) { v = __uint_as_float(w[o]); }
  __device__ static void get_r(const uint32_t* w, int o, double& v) { v = __hiloint2double(int(w[o + 1]), int(w[o])); }

  // the row of trajectory n after init() (done: init() finished it; the persistent kernel skips it)
  __device__ void save_start(const Problem& pb) const {
    static_assert(MT == 0 && !DD, "prepared starts are built for modes 0-2 without sensitivities");
    uint32_t w[kStartWords];
#pragma unroll
    for (int i = 0; i < D; i++) {
      put_r(w, kSY + i * kRW, y[i]);
      put_r(w, kSK1 + i * kRW, k1[i]);
      if constexpr (F32) w[kSLO + i] = __float_as_uint(ylo[i]);
    }
#pragma unroll
    for (int q = 0; q < NPP; q++) put_r(w, kSP + q * kRW, p[q]);
    put_r(w, kST, h);
    if constexpr (DF) {
      w[kST + 2] = __float_as_uint(th); w[kST + 3] = __float_as_uint(tl); w[kST + 4] = __float_as_uint(hf);
      w[kST + 5] = __float_as_uint(t1h); w[kST + 6] = __float_as_uint(t1l);
      w[kST + 7] = __float_as_uint(svh); w[kST + 8] = __float_as_uint(svl);
    } else {
      if constexpr (BITS) {
        w[kST + 2] = __float_as_uint(remf); w[kST + 3] = __float_as_uint(marg);
#pragma unroll
        for (int q = 4; q < 8; q++) w[kST + q] = 0u;
      } else {
        put_r(w, kST + 2, rem_c); put_r(w, kST + 4, hmin_c); put_r(w, kST + 6, 0.0);
      }
    }
    w[kSTail] = __float_as_uint(atolf);
    w[kSTail + 1] = __float_as_uint(rtolf);
    w[kSTail + 2] = uint32_t(status);
    w[kSTail + 3] = uint32_t(kk);
    w[kSTail + 4] = BITS ? uint32_t(kend) : 0u;
    w[kSTail + 5] = (sv_ok ? 1u : 0u) | (done ? 2u : 0u);
#pragma unroll
    for (int q = kSTail + 6; q < kStartWords; q++) w[q] = 0u;
    uint4* r4 = reinterpret_cast<uint4*>(pb.start + n * pb.start_row);
#pragma unroll
    for (int q = 0; q < kStartWords / 4; q++) r4[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
  }
  // trajectory traj from its row: the state init() would leave. Returns false (nothing to do) for a
  // trajectory that init() already finished.
  __device__ bool load_start(const Problem& pb, long long traj) {
    n = traj;
    uint32_t w[kStartWords];
    const uint4* r4 = reinterpret_cast<const uint4*>(pb.start + n * pb.start_row);
#pragma unroll
    for (int q = 0; q < kStartWords / 4; q++) {
      const uint4 v = r4[q];
      w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
    }
    if (w[kSTail + 5] & 2u) return false;
#pragma unroll
    for (int i = 0; i < D; i++) {
      get_r(w, kSY + i * kRW, y[i]);
      get_r(w, kSK1 + i * kRW, k1[i]);
      if constexpr (F32) ylo[i] = __uint_as_float(w[kSLO + i]);
    }
#pragma unroll
    for (int q = 0; q < NPP; q++) get_r(w, kSP + q * kRW, p[q]);
    get_r(w, kST, h);
    if constexpr (DF) {
      th = __uint_as_float(w[kST + 2]); tl = __uint_as_float(w[kST + 3]); hf = __uint_as_float(w[kST + 4]);
      t1h = __uint_as_float(w[kST + 5]); t1l = __uint_as_float(w[kST + 6]);
      svh = __uint_as_float(w[kST + 7]); svl = __uint_as_float(w[kST + 8]);
    } else {
      if constexpr (BITS) {
        remf = __uint_as_float(w[kST + 2]); marg = __uint_as_float(w[kST + 3]);
      } else {
        get_r(w, kST + 2, rem_c); get_r(w, kST + 4, hmin_c);
      }
    }
    atolf = __uint_as_float(w[kSTail]);
    rtolf = __uint_as_float(w[kSTail + 1]);
    status = int32_t(w[kSTail + 2]);
    kk = int32_t(w[kSTail + 3]);
    if constexpr (BITS) kend = int32_t(w[kSTail + 4]);
    sv_ok = (w[kSTail + 5] & 1u) != 0u;
    t0 = pb.t0[n];
    t1 = pb.t1[n];
    t = t0;
    tc = 0.0;
    if (kk < pb.K) sv = save_at(pb, n, kk);
    nacc = 0; nrej = 0; chunk = -1;
    done = false; failed = false; rec_ok = true;
    err_prev = 1.0;
    lerr_prev = 0.0f;
    return true;
  }

  __device__ void finish(const Problem& pb) {
    if (failed) {
      for (int k = 0; k < pb.K; k++) write_nan(pb, k);
    }
    if (pb.record) {
      if (!rec_ok) status |= ST_TAPE_OVERFLOW;
      pb.tape.n_rec[n] = rec_ok ? nacc : -1;
      pb.tape.head[n] = chunk;
    }
    pb.status[n] = status;
    pb.n_acc[n] = nacc;
    pb.n_rej[n] = nrej;
  }
};

}  // namespace gs
