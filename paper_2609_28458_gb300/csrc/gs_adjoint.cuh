// Discrete adjoint of the accepted step sequence (the reverse-mode counterpart of Appendix A,
// Eqs. adjoint and stage-sens). The forward pass records, per accepted step, the state at its
// start, t, tc, h and whether it was the last (clipped) step. The reverse pass walks that tape
// backwards; for each step it recomputes the stages from the recorded state with h held fixed
// (the same device code as the forward attempt) and propagates the cotangent through Eq. rk:
//   y+ = y + h sum_j b_j k_j,   k_j = f(t + c_j h, Y_j),   Y_j = y + h sum_{l<j} a_jl k_l
//   kbar_j = h (b_j ybar+ + sum_{l>j} a_lj Ybar_l) + dense-output injections,
//   Ybar_j = J_y(Y_j)^T kbar_j,   thetabar += J_theta(Y_j)^T kbar_j,   ybar = ybar+ + sum_j Ybar_j.
// Output cotangents dL/dy(t_k) enter at the step that produced y(t_k): through the dense-output
// weights b_j(sigma) (Eq. dense) for Tsit5/Dopri5, through a shortened step for Verner 7, or
// directly on y+ / y0 for outputs at t1 / t0. Since h is held fixed, the result is the exact
// derivative of the numerical solution on the recorded steps (Sec. 2.3).
#pragma once
#include "gs_stepper.cuh"

namespace gs {

// SLAB: the main step's stages leave their Jacobian factors in shared memory (from shared-window
// byte address sl, the float4s st bytes apart)
// and the stage VJPs read them back instead of re-evaluating the right-hand side's position factors;
// only for FP32 modes of systems that provide f_save / vjp_saved (the kernel supplies the memory).
// CK: the tape has a checkpoint stride S > 1 (gs_stepper.cuh, Tape); each segment of S steps is
// replayed forward from its checkpoint into this thread's segment buffer (local memory) before its
// steps are reversed, and outputs are attributed to steps through the tape's emit array.
template <template <class> class SysT, class Tab, int PM, bool SLAB = false, bool CK = false>
struct Adjoint {
  using T = Traj<SysT, Tab, PM>;
  static constexpr bool F32 = T::F32, DF = T::DF, DD = T::DD;
  using R = typename T::R;
  using Sys = typename T::Sys;
  static constexpr int D = T::D, NP = T::NP, S = Tab::S, NPA = T::NPA;
  static constexpr int Q = SaveQ<Sys>::value;
  // Nystrom form (the forward's stages of second-order systems in the FP32 modes): the stage
  // cotangents are those of the accelerations, abar_j = kbar_j's velocity part, over DH components
  static constexpr bool RKN = T::RKN;
  static constexpr int DH = T::DH;
  static constexpr int KD = RKN ? DH : D;
  using NY = Nystrom<Tab>;
  static_assert(!SLAB || (Q > 0 && F32 && !DD), "saved stage factors need an FP32 mode and f_save");
  static_assert(!CK || !DD, "checkpoint strides above 1 are not built for the df64 mode");
  static constexpr int kSegMax = kChunk;  // largest checkpoint stride

  struct PAcc {  // accumulator of theta-bar: FP64, or a compensated FP32 pair
    R s[NPA], c[NPA];
    __device__ void zero() {
#pragma unroll
      for (int q = 0; q < NPA; q++) { s[q] = R(0); c[q] = R(0); }
    }
    __device__ void add(int q, R v) {
      if constexpr (F32) {
        R ns, e;
        two_sum(s[q], v, ns, e);
        s[q] = ns;
        c[q] += e;
      } else {
        s[q] += v;
      }
    }
    __device__ double get(int q) const { return to_f64(s[q]) + to_f64(c[q]); }
  };

  // Reverse through stages 0..jmax-1 of a step of length hh whose stage states are Y and whose
  // stage cotangents are kbar (consumed). Adds to ybar and pacc: the stages' contributions to
  // theta-bar are summed in R first and enter the (compensated) accumulator once per step.
  template <bool USE_SLAB = false>
  __device__ static void reverse_stages(const T& tr, double tt, double hh, R (*Y)[D], R (*kbar)[D], int jmax,
                                        R* ybar, PAcc& pacc, unsigned sl = 0, unsigned st = 0) {
    const R hr = T::cvt(hh);
    R gsum[NPA];
#pragma unroll
    for (int q = 0; q < NPA; q++) gsum[q] = R(0);
#pragma unroll
    for (int j = S - 1; j >= 0; j--) {
      if (j < jmax) {
        R gy[D], gp[NPA];
        if constexpr (USE_SLAB) Sys::vjp_saved(tr.stage_time(tt + Tab::c(j) * hh), Y[j], tr.p, kbar[j], gy, gp,
                                               sl + unsigned(j * Q) * st, st);
        else Sys::vjp(tr.stage_time(tt + Tab::c(j) * hh), Y[j], tr.p, kbar[j], gy, gp);
#pragma unroll
        for (int i = 0; i < D; i++) ybar[i] += gy[i];
#pragma unroll
        for (int q = 0; q < NP; q++) gsum[q] += gp[q];
#pragma unroll
        for (int l = 0; l < j; l++) {
          if (Tab::a(j, l) != 0.0) {
            const R c = hr * R(Tab::a(j, l));
#pragma unroll
            for (int i = 0; i < D; i++) kbar[l][i] += c * gy[i];
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NP; q++) pacc.add(q, gsum[q]);
  }

  // reverse_stages in Nystrom form. With kbar_j = (xbar_j, abar_j) the general sweep's cotangents
  // of k_j = (V_j, a_j), substituting xbar_j = init + h sum_i a_ij Xbar_i leaves
  //   abar_l = (its initial value) + h^2 sum_i (A^2)_il Xbar_i,   Xbar_i = J_a(X_i)^T abar_i,
  //   ybar_x += sum_i Xbar_i,   ybar_v += h sum_i c'_i Xbar_i,
  // the initial values (b-terms and dense outputs) already carrying h A^T of their position parts
  // (step(), inject()). The same cotangents as the general sweep, over three components.
  template <bool USE_SLAB = false>
  __device__ static void reverse_stages_nystrom(const T& tr, double tt, double hh, R (*Y)[D], R (*abar)[KD], int jmax,
                                                R* ybar, PAcc& pacc, unsigned sl = 0, unsigned st = 0) {
    const R hr = T::cvt(hh);
    const R hr2 = hr * hr;
    R gsum[NPA];
#pragma unroll
    for (int q = 0; q < NPA; q++) gsum[q] = R(0);
#pragma unroll
    for (int j = S - 1; j >= 0; j--) {
      if (j < jmax) {
        R w[D], gy[D], gp[NPA];
#pragma unroll
        for (int i = 0; i < DH; i++) { w[i] = R(0); w[DH + i] = abar[j][i]; }
        if constexpr (USE_SLAB) Sys::vjp_saved(tr.stage_time(tt + Tab::c(j) * hh), Y[j], tr.p, w, gy, gp,
                                               sl + unsigned(j * Q) * st, st);
        else Sys::vjp(tr.stage_time(tt + Tab::c(j) * hh), Y[j], tr.p, w, gy, gp);
        const R hc = hr * R(NY::row(j));
#pragma unroll
        for (int i = 0; i < DH; i++) {
          ybar[i] += gy[i];
          ybar[DH + i] += hc * gy[i];
        }
#pragma unroll
        for (int q = 0; q < NP; q++) gsum[q] += gp[q];
#pragma unroll
        for (int l = 0; l < j - 1; l++) {
          if (NY::aa(j, l) != 0.0) {
            const R c = hr2 * R(NY::aa(j, l));
#pragma unroll
            for (int i = 0; i < DH; i++) abar[l][i] += c * gy[i];
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NP; q++) pacc.add(q, gsum[q]);
  }
  // the b-terms of the new state's cotangent ybar, before the stage sweep: general form
  // kbar_j += h b_j ybar; Nystrom form abar_j += h b_j ybar_v + h^2 (bA)_j ybar_x and
  // ybar_v += h ybar_x (x+ = x + h v + ...; sum_j b_j = 1)
  __device__ static void seed_b(R hr, R (*kbar)[KD], R* ybar) {
    if constexpr (RKN) {
      const R hr2 = hr * hr;
#pragma unroll
      for (int j = 0; j < S; j++)
#pragma unroll
        for (int i = 0; i < DH; i++) {
          R v = kbar[j][i];
          if (Tab::b(j) != 0.0) v += hr * R(Tab::b(j)) * ybar[DH + i];
          if (NY::ba(j) != 0.0) v += hr2 * R(NY::ba(j)) * ybar[i];
          kbar[j][i] = v;
        }
#pragma unroll
      for (int i = 0; i < DH; i++) ybar[DH + i] += hr * ybar[i];
    } else {
#pragma unroll
      for (int j = 0; j < S; j++)
        if (Tab::b(j) != 0.0)
#pragma unroll
          for (int i = 0; i < D; i++) kbar[j][i] += hr * R(Tab::b(j)) * ybar[i];
    }
  }

  struct SlotView {
    double t, tc, h;
    float th, tl, hf;  // PM 2: the time pair and FP32 step as recorded
    bool last;
  };

  __device__ static const unsigned char* slot_ptr(const Problem& pb, int32_t chunk, int o) {
    return pb.tape.pool + (long long)chunk * pb.tape.chunk_bytes + kChunkHeader + (long long)o * T::kSlotBytes;
  }
  __device__ static int32_t prev_chunk(const Problem& pb, int32_t chunk) {
    return int32_t(*reinterpret_cast<const long long*>(pb.tape.pool + (long long)chunk * pb.tape.chunk_bytes));
  }
  // A slot's words as loaded, before any arithmetic consumes them: the next step's slot is fetched
  // one step ahead into this, so the loads overlap a whole step of arithmetic, and decoded when used.
  struct Raw {
    R y[D];          // the state at the step's start (FP32 modes: its high part; the low part is
                     // not recorded, the stages are recomputed from the high part as in the forward)
    float4 tf;       // PM 2 tail: th, tl, h, flag
    double tt, tc, hs;  // PM 0, 1 tail: t, tc, h (negative for the last step)
  };
  __device__ static void fetch(const unsigned char* s, Raw& r) {
    if constexpr (F32) {
      if constexpr (D % 4 == 0) {
        const float4* f4 = reinterpret_cast<const float4*>(s);
#pragma unroll
        for (int q = 0; q < D / 4; q++) {
          const float4 a = f4[q];
          r.y[4 * q] = a.x; r.y[4 * q + 1] = a.y; r.y[4 * q + 2] = a.z; r.y[4 * q + 3] = a.w;
        }
      } else if constexpr (D % 2 == 0) {
        const float2* f2 = reinterpret_cast<const float2*>(s);
#pragma unroll
        for (int q = 0; q < D / 2; q++) { const float2 a = f2[q]; r.y[2 * q] = a.x; r.y[2 * q + 1] = a.y; }
      } else {
        const float* f = reinterpret_cast<const float*>(s);
#pragma unroll
        for (int i = 0; i < D; i++) r.y[i] = f[i];
      }
    } else if constexpr (DD) {
      // (hi, lo) per component: two components per 16-byte load
      const float4* f4 = reinterpret_cast<const float4*>(s);
#pragma unroll
      for (int q = 0; q < D / 2; q++) {
        const float4 a = f4[q];
        r.y[2 * q] = F2::pair(a.x, a.y);
        r.y[2 * q + 1] = F2::pair(a.z, a.w);
      }
      if constexpr (D % 2 == 1) {
        const float2 a = reinterpret_cast<const float2*>(s)[D - 1];
        r.y[D - 1] = F2::pair(a.x, a.y);
      }
    } else {
      const double2* f2 = reinterpret_cast<const double2*>(s);
#pragma unroll
      for (int q = 0; q < D / 2; q++) { const double2 a = f2[q]; r.y[2 * q] = a.x; r.y[2 * q + 1] = a.y; }
      if constexpr (D % 2 == 1) r.y[D - 1] = reinterpret_cast<const double*>(s)[D - 1];
    }
    if constexpr (DF) {
      r.tf = *reinterpret_cast<const float4*>(s + T::kTailOff);
    } else {
      if constexpr (T::kTailOff % 16 == 0) {
        const double2 a = *reinterpret_cast<const double2*>(s + T::kTailOff);
        r.tt = a.x; r.tc = a.y;
        r.hs = *reinterpret_cast<const double*>(s + T::kTailOff + 16);
      } else {
        r.tt = *reinterpret_cast<const double*>(s + T::kTailOff);
        const double2 a = *reinterpret_cast<const double2*>(s + T::kTailOff + 8);
        r.tc = a.x; r.hs = a.y;
      }
    }
  }
  __device__ static SlotView decode(const Raw& r) {
    SlotView v;
    if constexpr (DF) {
      v.th = r.tf.x; v.tl = r.tf.y; v.hf = r.tf.z; v.last = r.tf.w != 0.0f;
      v.t = double(v.th) + double(v.tl);
      v.tc = 0.0;
      v.h = double(v.hf);
    } else {
      v.t = r.tt; v.tc = r.tc;
      v.last = signbit_f64_bits(r.hs);  // (h > 0: the sign marks the last step)
      v.h = abs_f64_bits(r.hs);
    }
    return v;
  }

  // the forward's test for an output inside a step, in the same arithmetic
  __device__ static bool inside(const SlotView& v, double sv) {
    if constexpr (DF) {
      float svh, svl;
      split_df(sv, svh, svl);
      return v.last || ((svh - v.th) + (svl - v.tl)) <= v.hf;
    } else {
      return v.last || ((sv - v.t) + v.tc) <= v.h;
    }
  }
  __device__ static R sigma(const SlotView& v, double sv) {
    if constexpr (DD) {  // as the forward: df64 fraction from the time pairs and the step's exact length
      float svh, svl;
      split_df(sv, svh, svl);
      R sg = ((R(svh) + R(svl)) - (R(v.th) + R(v.tl))) / R(v.h);
      if (val(sg) > 1.0f) sg = R(1.0f);
      if (val(sg) < 0.0f) sg = R(0.0f);
      return sg;
    } else if constexpr (DF) {
      float svh, svl;
      split_df(sv, svh, svl);
      return fminf(fmaxf(__fdividef((svh - v.th) + (svl - v.tl), v.hf), 0.0f), 1.0f);
    } else {
      double sg = ((sv - v.t) + v.tc) / v.h;
      if (sg > 1.0) sg = 1.0;
      if (sg < 0.0) sg = 0.0;
      return R(sg);
    }
  }

  // ---- reverse sweep of one trajectory as a state machine: init(), step() per recorded step,
  // finish(); the plain kernel runs it per thread, the persistent one refills lanes.
  T tr;
  R ybar[D];
  PAcc pacc;
  const double* W;
  int kk, a;
  int32_t chunk;
  bool done;
  Raw nraw;  // the slot of step a, then (once step a has started) of step a - 1
  unsigned sl = 0, st = 0;  // SLAB: this thread's stage factors, stage j at shared address sl + j * Q * st
  // CK: start states (FP32 modes: their high parts, from which the stages are recomputed) and times
  // (t, tc, or the FP32 pair th, tl) of the steps seg_lo .. seg_lo + S - 1 of the current segment
  using TT = typename std::conditional<DF, float, double>::type;
  R sy[CK ? kSegMax : 1][D];
  TT sta[CK ? kSegMax : 1], stb[CK ? kSegMax : 1];
  int seg_lo;
  // CK self-check (tape.verify): the checkpoint loaded last (the start of the next newer segment)
  R vy[CK ? D : 1], vlo[CK ? D : 1];
  bool vhave;

  __device__ void write_const(const Problem& pb, double v_y, double v_p, bool sum_w, bool only_t0) {
    const long long n = tr.n;
    double* gy0 = pb.dLdy0 + n * D;
#pragma unroll
    for (int i = 0; i < D; i++) {
      double acc = v_y;
      if (sum_w) {
        acc = 0.0;
        for (int k = 0; k < pb.K; k++)
          if (!only_t0 || (save_valid(pb, n, k, tr.t0, tr.t1) && save_at(pb, n, k) == tr.t0)) acc += W[k * D + i];
      }
      gy0[i] = acc;
    }
#pragma unroll
    for (int q = 0; q < NP; q++) pb.dLdp[n * NP + q] = v_p;
  }

  __device__ void init(const Problem& pb, long long n) {
    done = false;
    tr.n = n;
    tr.t0 = pb.t0[n];
    tr.t1 = pb.t1[n];
    W = pb.dLdy + n * (long long)pb.K * D;
    const int32_t st = pb.status[n];
    const int32_t nrec = pb.tape.n_rec[n];
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);
    if ((st & ST_FAILED) || nrec < 0) { write_const(pb, nanv, nanv, false, false); done = true; return; }
    if (st & ST_EMPTY) { write_const(pb, 0.0, 0.0, true, false); done = true; return; }  // outputs are y0
    if (nrec == 0) { write_const(pb, 0.0, 0.0, true, true); done = true; return; }
#pragma unroll
    for (int q = 0; q < NP; q++) tr.p[q] = T::cvt(pb.params[n * NP + q]);
    if (NP == 0) tr.p[0] = R(0);
    prep_params<Sys>(tr.p);
#pragma unroll
    for (int i = 0; i < D; i++) ybar[i] = R(0);
    pacc.zero();
    kk = pb.K - 1;
    a = nrec - 1;
    chunk = pb.tape.head[n];
#pragma unroll
    for (int i = 0; i < T::DL; i++) tr.ylo[i] = R(0);
    if constexpr (CK) {
      // a chunk index outside the pool means the tape was recorded with other options (gs_vjp with
      // reuse_tape needs the recording's options): NaN gradients rather than a read outside the pool
      if (chunk < 0 || chunk >= pb.tape.pool_chunks) { write_const(pb, nanv, nanv, false, false); done = true; return; }
      seg_lo = nrec;  // no segment buffered
      vhave = false;
      // outputs emitted after the final step (the interval closed without a clipped last step)
      const int32_t* em = pb.tape.emit + n * pb.K;
      while (kk >= 0 && (em[kk] == kEmitUnused || em[kk] == nrec)) {
        if (em[kk] == nrec)
#pragma unroll
          for (int i = 0; i < D; i++) ybar[i] += R(W[kk * D + i]);
        kk--;
      }
      return;
    }
    fetch(slot_ptr(pb, chunk, a % kChunk), nraw);
    const SlotView last = decode(nraw);
    // outputs emitted after the final step when the interval closed without a clipped last step
    while (kk >= 0) {
      if (!save_valid(pb, n, kk, tr.t0, tr.t1)) { kk--; continue; }
      const double sv = save_at(pb, n, kk);
      if (sv == tr.t0 || inside(last, sv)) break;
#pragma unroll
      for (int i = 0; i < D; i++) ybar[i] += R(W[kk * D + i]);
      kk--;
    }
  }

  // CK: replay the segment holding step a from its checkpoint (in the current chunk: S divides the
  // chunk length, so a segment never spans two chunks) and keep the start state and time of each
  // of its steps up to a.
  __device__ void load_segment(const Problem& pb) {
    if constexpr (CK) {
      const int S = pb.tape.stride;
      seg_lo = (a / S) * S;
      const int o0 = seg_lo % kChunk;
      const unsigned char* base = pb.tape.pool + (long long)chunk * pb.tape.chunk_bytes;
      const uint4* c4 = reinterpret_cast<const uint4*>(base + T::kCkOff + (long long)(o0 / S) * T::kCkBytes);
      uint32_t w[T::kCkWords];
#pragma unroll
      for (int q = 0; q < T::kCkWords / 4; q++) {
        const uint4 v = c4[q];
        w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
      }
      if constexpr (F32) {
#pragma unroll
        for (int i = 0; i < D; i++) {
          tr.y[i] = __uint_as_float(w[i]);
          tr.ylo[i] = __uint_as_float(w[D + i]);
          tr.k1[i] = __uint_as_float(w[2 * D + i]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < D; i++) {
          tr.y[i] = __hiloint2double(int(w[2 * i + 1]), int(w[2 * i]));
          tr.k1[i] = __hiloint2double(int(w[2 * D + 2 * i + 1]), int(w[2 * D + 2 * i]));
        }
      }
      constexpr int T0 = T::kCkTimeOff / 4;
      if constexpr (DF) {
        tr.th = __uint_as_float(w[T0]);
        tr.tl = __uint_as_float(w[T0 + 1]);
      } else {
        tr.t = __hiloint2double(int(w[T0 + 1]), int(w[T0]));
        tr.tc = __hiloint2double(int(w[T0 + 3]), int(w[T0 + 2]));
      }
      const int m = a - seg_lo;  // steps to replay before step a
      const bool verify = pb.tape.verify != nullptr;
      R cy[CK ? D : 1], clo[CK ? D : 1];
      if (verify) {
#pragma unroll
        for (int q = 0; q < D; q++) {
          cy[q] = tr.y[q];
          if constexpr (F32) clo[q] = tr.ylo[q];
        }
      }
      for (int i = 0;; i++) {
#pragma unroll
        for (int q = 0; q < D; q++) sy[i][q] = tr.y[q];
        if constexpr (DF) { sta[i] = tr.th; stb[i] = tr.tl; }
        else { sta[i] = tr.t; stb[i] = tr.tc; }
        if (i >= m) break;
        tr.replay_step(step_length(base, o0 + i));
      }
      if (verify) {
        // a full segment's last step, replayed, must land bit for bit on the newer segment's checkpoint
        if (vhave && m == S - 1) {
          tr.replay_step(step_length(base, o0 + m));
          bool same = true;
#pragma unroll
          for (int q = 0; q < D; q++) {
            same = same && bits_equal(tr.y[q], vy[q]);
            if constexpr (F32) same = same && bits_equal(tr.ylo[q], vlo[q]);
          }
          atomicAdd(pb.tape.verify, 1u);
          if (!same) atomicAdd(pb.tape.verify + 1, 1u);
        }
#pragma unroll
        for (int q = 0; q < D; q++) {
          vy[q] = cy[q];
          if constexpr (F32) vlo[q] = clo[q];
        }
        vhave = true;
      }
    }
  }
  __device__ static double step_length(const unsigned char* base, int o) {
    if constexpr (DF) return double(reinterpret_cast<const float*>(base + kChunkHeader)[o]);
    else return reinterpret_cast<const double*>(base + kChunkHeader)[o];
  }
  __device__ static bool bits_equal(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
  __device__ static bool bits_equal(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }

  // Reverse of step a of a checkpointed tape (CK), a step of the segment load_segment() buffered: as
  // step(), with the step's start state and time from the segment buffer, its length from the chunk,
  // and its outputs from the emit array.
  __device__ void step_ck(const Problem& pb) {
    const long long n = tr.n;
    const double t1 = tr.t1;
    const int o = a % kChunk;
    const int i0 = a - seg_lo;
    const unsigned char* base = pb.tape.pool + (long long)chunk * pb.tape.chunk_bytes;
    SlotView cur;
    if constexpr (DF) {
      const float hv = reinterpret_cast<const float*>(base + kChunkHeader)[o];
      cur.last = hv < 0.0f;
      cur.hf = fabsf(hv);
      cur.h = double(cur.hf);
      cur.th = sta[i0];
      cur.tl = stb[i0];
      cur.t = double(cur.th) + double(cur.tl);
      cur.tc = 0.0;
    } else {
      const double hv = reinterpret_cast<const double*>(base + kChunkHeader)[o];
      cur.last = signbit_f64_bits(hv);  // (the sign marks the last step; h > 0)
      cur.h = abs_f64_bits(hv);
      cur.t = sta[i0];
      cur.tc = stb[i0];
    }
#pragma unroll
    for (int q = 0; q < D; q++) tr.y[q] = sy[i0][q];
    if constexpr (SLAB) Sys::f_save(tr.stage_time(cur.t), tr.y, tr.p, tr.k1, sl, st);
    else Sys::f(tr.stage_time(cur.t), tr.y, tr.p, tr.k1);
    const int32_t* em = pb.tape.emit + n * pb.K;
    // does an output of this step use the dense polynomial (which needs the last, FSAL stage)?
    bool dense_here = false;
    if constexpr (Tab::DENSE_POLY) {
      for (int q = kk; q >= 0; q--) {
        if (em[q] == kEmitUnused) continue;
        if (em[q] != a) break;
        if (!(cur.last && save_at(pb, n, q) == t1)) { dense_here = true; break; }
      }
    }
    R k[S][D], Y[S][D], kbar[S][KD];
    tr.template stages<SLAB>(cur.t, cur.h, k, Y, dense_here ? S : Tab::NREV, sl, st);
#pragma unroll
    for (int j = 0; j < S; j++)
#pragma unroll
      for (int i = 0; i < KD; i++) kbar[j][i] = R(0);
    R ydir[D];
#pragma unroll
    for (int i = 0; i < D; i++) ydir[i] = R(0);
    bool used_last_stage = false;
    const R hr = T::cvt(cur.h);
    while (kk >= 0) {
      if (em[kk] == kEmitUnused) { kk--; continue; }
      if (em[kk] != a) break;
      inject(pb, cur, save_at(pb, n, kk), k, kbar, ydir, used_last_stage, hr);
      kk--;
    }
    seed_b(hr, kbar, ybar);
#pragma unroll
    for (int i = 0; i < D; i++) ybar[i] += ydir[i];
    if constexpr (RKN)
      reverse_stages_nystrom<SLAB>(tr, cur.t, cur.h, Y, kbar, used_last_stage ? S : Tab::NREV, ybar, pacc, sl, st);
    else
      reverse_stages<SLAB>(tr, cur.t, cur.h, Y, kbar, used_last_stage ? S : Tab::NREV, ybar, pacc, sl, st);
    if (o == 0 && a > 0) {
      chunk = prev_chunk(pb, chunk);
      if (chunk < 0 || chunk >= pb.tape.pool_chunks) {  // as in init(): not this tape's layout
        const double nanv = __longlong_as_double(0x7ff8000000000000LL);
        write_const(pb, nanv, nanv, false, false);
        done = true;
        return;
      }
    }
    a -= 1;
    if (a < 0) finish(pb);
  }

  // The cotangent W[kk] of output time sv, emitted by the step cur: directly on the new state for
  // an output at t1 after the last step, else through the dense-output weights (Tsit5, Dopri5) or
  // a shortened step (Verner 7).
  __device__ void inject(const Problem& pb, const SlotView& cur, double sv, R (*k)[D], R (*kbar)[KD], R* ydir,
                         bool& used_last_stage, R hr) {
    R w[D];
#pragma unroll
    for (int i = 0; i < D; i++) w[i] = R(W[kk * D + i]);
    if (cur.last && sv == tr.t1) {
#pragma unroll
      for (int i = 0; i < D; i++) ybar[i] += w[i];  // y(t1) is the new state itself
      return;
    }
    const R sig = sigma(cur, sv);
    if constexpr (Tab::DENSE_POLY) {
      // y(t_k) = y + h sum_j b_j(sig) k_j
      R wd[S];
      Tab::dense(sig, wd);
      if constexpr (RKN) {
        // Nystrom form: abar_l += h wd_l w_v + h^2 (wd A)_l w_x; the position part also reaches v
        // through x(t_k) = x + h (sum_j wd_j) v + ...
        const R hr2 = hr * hr;
        R ws = R(0);
#pragma unroll
        for (int j = 0; j < S; j++) ws = ws + wd[j];
#pragma unroll
        for (int l = 0; l < S; l++) {
          R wa = R(0);
#pragma unroll
          for (int j = l + 1; j < S; j++)
            if (Tab::a(j, l) != 0.0) wa = wa + wd[j] * R(Tab::a(j, l));
#pragma unroll
          for (int i = 0; i < DH; i++) kbar[l][i] += hr * wd[l] * w[DH + i] + hr2 * wa * w[i];
        }
#pragma unroll
        for (int i = 0; i < DH; i++) {
          ydir[i] += w[i];
          ydir[DH + i] += w[DH + i] + hr * ws * w[i];
        }
      } else {
#pragma unroll
        for (int j = 0; j < S; j++)
#pragma unroll
          for (int i = 0; i < D; i++) kbar[j][i] += hr * wd[j] * w[i];
#pragma unroll
        for (int i = 0; i < D; i++) ydir[i] += w[i];
      }
      used_last_stage = true;
    } else {
      // Verner 7: y(t_k) = shortened step of length sig*h from (t, y)
      const double hs = to_f64(sig) * cur.h;
      R ks[S][D], Ys[S][D], kbs[S][D];
      tr.stages(cur.t, hs, ks, Ys, Tab::NREV);
      const R hsr = R(hs);
#pragma unroll
      for (int j = 0; j < S; j++)
#pragma unroll
        for (int i = 0; i < D; i++) kbs[j][i] = (j < Tab::NREV) ? hsr * R(Tab::b(j)) * w[i] : R(0);
#pragma unroll
      for (int i = 0; i < D; i++) ydir[i] += w[i];
      reverse_stages(tr, cur.t, hs, Ys, kbs, Tab::NREV, ydir, pacc);
    }
  }

  // Reverse of recorded step a (ybar holds the cotangent of the state after it).
  __device__ void step(const Problem& pb) {
    static_assert(!CK, "a checkpointed tape is reversed segment by segment (load_segment, step_ck)");
    const long long n = tr.n;
    const double t0 = tr.t0, t1 = tr.t1;
    const int o = a % kChunk;
    SlotView cur = decode(nraw);
    // df64: the last step spanned the exact remainder t1 - t (exact in FP64 for the time pairs)
    if constexpr (DD)
      if (cur.last) cur.h = tr.t1 - cur.t;
#pragma unroll
    for (int i = 0; i < D; i++) tr.y[i] = nraw.y[i];
    const int32_t pchunk = (o == 0 && a > 0) ? prev_chunk(pb, chunk) : chunk;
    // fetch step a - 1 now; its times are decoded only where an output may belong to it
    if (a > 0) fetch(slot_ptr(pb, pchunk, o == 0 ? kChunk - 1 : o - 1), nraw);
    if constexpr (SLAB) Sys::f_save(tr.stage_time(cur.t), tr.y, tr.p, tr.k1, sl, st);
    else Sys::f(tr.stage_time(cur.t), tr.y, tr.p, tr.k1);
    // does an output inside this step use the dense polynomial (which needs the last, FSAL stage)?
    bool dense_here = false;
    if constexpr (Tab::DENSE_POLY) {
      for (int q = kk; q >= 0; q--) {
        if (!save_valid(pb, n, q, t0, t1)) continue;
        const double sq = save_at(pb, n, q);
        if (sq == t0 || !inside(cur, sq) || (a > 0 && inside(decode(nraw), sq))) break;
        if (!(cur.last && sq == t1)) { dense_here = true; break; }
      }
    }
    R k[S][D], Y[S][D], kbar[S][KD];
    tr.template stages<SLAB>(cur.t, cur.h, k, Y, dense_here ? S : Tab::NREV, sl, st);
#pragma unroll
    for (int j = 0; j < S; j++)
#pragma unroll
      for (int i = 0; i < KD; i++) kbar[j][i] = R(0);
    // cotangents reaching the step's start state directly (identity term of an output inside it)
    R ydir[D];
#pragma unroll
    for (int i = 0; i < D; i++) ydir[i] = R(0);
    bool used_last_stage = false;
    const R hr = T::cvt(cur.h);
    // output cotangents of this step, latest first
    while (kk >= 0) {
      if (!save_valid(pb, n, kk, t0, t1)) { kk--; continue; }
      const double sv = save_at(pb, n, kk);
      if (sv == t0) break;
      if (!inside(cur, sv)) break;
      if (a > 0 && inside(decode(nraw), sv)) break;
      inject(pb, cur, sv, k, kbar, ydir, used_last_stage, hr);
      kk--;
    }
    // the step itself: kbar_j += h b_j ybar, then the stages in reverse
    seed_b(hr, kbar, ybar);
#pragma unroll
    for (int i = 0; i < D; i++) ybar[i] += ydir[i];
    if constexpr (RKN)
      reverse_stages_nystrom<SLAB>(tr, cur.t, cur.h, Y, kbar, used_last_stage ? S : Tab::NREV, ybar, pacc, sl, st);
    else
      reverse_stages<SLAB>(tr, cur.t, cur.h, Y, kbar, used_last_stage ? S : Tab::NREV, ybar, pacc, sl, st);
    chunk = pchunk;
    a -= 1;
    if (a < 0) finish(pb);
  }

  __device__ void finish(const Problem& pb) {
    const long long n = tr.n;
    // outputs at t0 are y0 itself
    while (kk >= 0) {
      if (save_valid(pb, n, kk, tr.t0, tr.t1) && save_at(pb, n, kk) == tr.t0) {
#pragma unroll
        for (int i = 0; i < D; i++) ybar[i] += R(W[kk * D + i]);
      }
      kk--;
    }
    double* gy0 = pb.dLdy0 + n * D;
#pragma unroll
    for (int i = 0; i < D; i++) gy0[i] = to_f64(ybar[i]);
#pragma unroll
    for (int q = 0; q < NP; q++) pb.dLdp[n * NP + q] = pacc.get(q) * VjpParamScale<Sys>::of(q);
    done = true;
  }
};

}  // namespace gs
