/* gs.h — C ABI of the GB300 ensemble Runge-Kutta library (libgs.so).
 *
 * The library integrates n independent initial-value problems dy_i/dt = f(t, y_i, theta_i),
 * y_i(t0_i) = y0_i (the ensemble problem, Sec. 2.1, Eq. ivp) with adaptive explicit Runge-Kutta
 * pairs (Sec. 2.2; Appendix A, Eqs. rk, errnorm, controller, dense), one trajectory per GPU thread,
 * and returns the gradient of a scalar loss through the solve by a discrete adjoint of the
 * accepted step sequence (the reverse-mode counterpart of Appendix A, Eqs. adjoint, stage-sens).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers to caller-owned memory, in row-major (C) order, FP64
 *    unless stated. The library allocates no device memory; scratch space is the caller's
 *    `workspace`. Nothing is freed by the library.
 *  - Calls are asynchronous and ordered on `cuda_stream` (a cudaStream_t; NULL = legacy default
 *    stream). Per-trajectory failures are reported in the `status` array, never by a trap.
 *  - Return value: GS_OK (0) or a GS_ERR_* code; on a non-zero return nothing was launched and no
 *    output was written. gs_last_error() then gives a message (thread-local).
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Systems (right-hand sides f):
 *  GS_SYS_ISOCHRONE    d=6, p=0: test particle in Phi = -1/(1+sqrt(1+r^2)), G = M = b = 1.
 *  GS_SYS_MW           d=6, p=4: Miyamoto-Nagai disc + Hernquist bulge + z-flattened NFW halo;
 *                      theta = (M_disc, M_bulge, M_halo [1e10 Msun], q_halo); kpc, Myr units.
 *  GS_SYS_PRECESSION   d=9, p=3: orbit-averaged spin precession in v (Sec. 5, Eqs. prec-spins,
 *                      prec-L, prec-omega, prec-rr with 2PN b_k); theta = (q, chi1, chi2).
 *  GS_SYS_QUINTESSENCE d=3, p=4: thawing quintessence in N = ln a (Sec. 4.1, Eq. de-model;
 *                      Appendix C, Eq. de-rhs); y = (phi, u, I), theta = (a0, lambda, Om, Or).
 *  GS_SYS_LOGHALO      d=6, p=3: flattened logarithmic halo (Sec. 3, Eq. loghalo);
 *                      theta = (v_c, R_c, q).
 */
typedef enum {
  GS_SYS_ISOCHRONE = 0,
  GS_SYS_MW = 1,
  GS_SYS_PRECESSION = 2,
  GS_SYS_QUINTESSENCE = 3,
  GS_SYS_LOGHALO = 4
} gs_system;

/* Runge-Kutta pairs (Sec. 2.2): Tsit5 and Dopri5 (order 5, FSAL, dense-output polynomial),
 * Verner's 7(6) pair (order 7; outputs inside a step by a shortened step, Appendix A). */
typedef enum { GS_TSIT5 = 0, GS_DOPRI5 = 1, GS_VERN7 = 2 } gs_method;

/* GS_FP64: every operation in FP64.
 * GS_FP32_STAGES: stage and right-hand-side arithmetic in FP32, the state kept as a compensated
 *   FP32 pair, the error-norm accumulation, the time (compensated summation) and the step-size
 *   controller in FP64. For the orbit systems (isochrone, Milky Way, log halo: y = (x, v),
 *   f = (v, a(x))) with GS_TSIT5 or GS_DOPRI5, both FP32 modes evaluate the pair's stages, dense
 *   output and reverse sweep in Nystrom form: the same stages, with sums over the positions only
 *   (A^2 and the row sums of A), and no difference of velocity-sized terms in the position error.
 * GS_FP32_DF: as GS_FP32_STAGES, but the time is an unevaluated FP32 pair (>= 48 significant bits,
 *   advanced error-free), the step length is the FP32 number the stages use, and the norm
 *   accumulation and controller run in FP32: the attempt loop issues no FP64 instruction.
 * GS_DF64: the state, the stages, the stage times, the error estimate and the dense outputs in
 *   double-FP32 arithmetic (unevaluated pairs of FP32 numbers, ~48 significant bits, built from
 *   error-free transformations), time and controller as GS_FP32_DF: tolerances near FP64's reach
 *   without the FP64 pipe. Systems GS_SYS_ISOCHRONE, GS_SYS_PRECESSION and GS_SYS_LOGHALO (their
 *   right-hand sides need only arithmetic and square roots); gs_solve and gs_vjp. */
typedef enum { GS_FP64 = 0, GS_FP32_STAGES = 1, GS_FP32_DF = 2, GS_DF64 = 3 } gs_precision;

/* GS_KERNEL_PLAIN: one thread per trajectory for its whole solve (a warp waits for its slowest
 *   member, Appendix A, Eq. cost). GS_KERNEL_PERSISTENT: persistent CTAs whose lanes take the next
 *   trajectory from a device work queue as soon as their own one finishes. */
typedef enum { GS_KERNEL_AUTO = 0, GS_KERNEL_PLAIN = 1, GS_KERNEL_PERSISTENT = 2 } gs_kernel;

/* Per-trajectory status bits (status[n]). */
#define GS_ST_OK 0
#define GS_ST_MAX_STEPS 1       /* more than max_steps attempts; outputs NaN            */
#define GS_ST_H_UNDERFLOW 2     /* h < 16 eps max(|t|,|t1|); outputs NaN                */
#define GS_ST_NONFINITE 4       /* non-finite y0, theta, t0 or t1; outputs NaN          */
#define GS_ST_EMPTY_INTERVAL 8  /* t1 <= t0: every output is y0, no step taken          */
#define GS_ST_SAVEAT_OUTSIDE 16 /* an output time outside [t0,t1] or decreasing: NaN there */
#define GS_ST_TAPE_OVERFLOW 32  /* gs_vjp: the step tape did not fit; gradients NaN     */
#define GS_ST_NO_CONVERGENCE 64 /* gs_solve_flat: |g| > gtol after max_newton steps, or
                                   the last output is not at t1 (then outputs NaN)       */

/* Return codes. */
#define GS_OK 0
#define GS_ERR_INVALID 1   /* bad argument (null pointer, size, enum)        */
#define GS_ERR_CUDA 2      /* a CUDA runtime call failed                     */
#define GS_ERR_WORKSPACE 3 /* workspace missing or too small                 */

typedef struct {
  int32_t method;       /* gs_method                                                  */
  int32_t precision;    /* gs_precision                                               */
  int32_t kernel;       /* gs_kernel                                                  */
  int32_t max_steps;    /* attempts per trajectory before GS_ST_MAX_STEPS (1e6)       */
  double safety;        /* controller safety factor (0.9)                             */
  double alpha_min;     /* smallest step ratio (0.2)                                  */
  double alpha_max;     /* largest step ratio (5)                                     */
  double beta1, beta2;  /* PI gains: h*clamp(safety*err^-beta1*err_prev^beta2);
                           beta1 = 0 selects 1/nu and beta2 = 0 gives Eq. controller  */
  double h0;            /* initial step; 0 = Hairer-Norsett-Wanner starting step      */
  int32_t per_traj_saveat; /* saveat is [N,K] instead of [K]                          */
  int32_t block_size;      /* threads per block; 0 = library default                  */
  int32_t record_tape;     /* gs_solve: record the accepted steps into the workspace  */
  int32_t reuse_tape;      /* gs_vjp: reverse the tape recorded by the preceding
                              gs_solve (same inputs and options) instead of re-solving */
  int32_t tape_capacity;   /* max accepted steps recorded per trajectory (1e6); a
                              trajectory with more gets GS_ST_TAPE_OVERFLOW            */
  int32_t sm_limit;        /* persistent kernels launch at most this many SMs' worth of
                              resident blocks (0 = every SM), so that kernels launched
                              concurrently on other streams share the GPU              */
  int32_t graph_safe;      /* gs_solve_flat / gs_profile_fit: no host synchronisation;
                              every Newton iteration is launched (max_newton of them)
                              and work-list lengths stay on the device, so the calls
                              can be captured into a CUDA graph                        */
  int32_t order;           /* order in which the forward kernels take trajectories:
                              GS_ORDER_AUTO (0): by cost_hint if given, else by the
                              estimate for N >= 32768, else as stored; GS_ORDER_NATURAL
                              (1): as stored, in gs_vjp's reverse pass too (otherwise
                              ordered by the recorded step counts); GS_ORDER_ESTIMATE
                              (2): longest first by the estimate
                              (t1 - t0) ||f(t0, y0)/s|| / ||y0/s||, s = atol + rtol|y0|
                              (one f evaluation per trajectory, the time-scale ratio of
                              the starting-step heuristic); GS_ORDER_HINT (3): longest
                              first by cost_hint. Results do not depend on the order  */
  const int32_t* cost_hint;  /* [N] device array, e.g. the attempt counts of a previous
                              solve of similar inputs (may be NULL)                    */
  int32_t ckpt_stride;     /* step tape (gs_vjp, gs_solve with record_tape): S = 1 (or 0)
                              records every accepted step's start state; S in {2, 4, 8,
                              16, 32} records the full integrator state every S accepted
                              steps plus every step's length, and the reverse pass
                              re-runs each segment of S steps from its checkpoint
                              (bit-identical to the forward, so the gradient equals
                              S = 1's). The tape shrinks about S-fold (a discrete form of
                              the checkpointing trade-off of Appendix A, Eq. disc-modes)
                              for one more forward step per reversed step. S > 1 needs
                              the persistent kernel and is not available in GS_DF64.
                              The library does not pick S; the Python autotuner does  */
  int32_t ckpt_verify;     /* with ckpt_stride > 1: gs_vjp's reverse pass also replays the
                              last step of every full segment and compares the state it
                              reaches with the next segment's checkpoint bit for bit,
                              adding the comparisons and the mismatches to the uint32
                              words at workspace bytes 16 and 20 (zeroed by the call that
                              records the tape). A self-check of the replay: one more
                              forward step per segment                                 */
  int32_t warp_lanes;      /* persistent kernels: how many lanes of each warp take
                              trajectories (1..32; 0 = 32). Fewer spread a small ensemble
                              over more warps, and so over more of the SMs' schedulers
                              and their FP64 units, at the price of idle lanes          */
} gs_options;

#define GS_ORDER_AUTO 0
#define GS_ORDER_NATURAL 1
#define GS_ORDER_ESTIMATE 2
#define GS_ORDER_HINT 3

/* Fill *opt with the defaults above (Tsit5, FP64, auto kernel). */
void gs_default_options(gs_options* opt);

/* State and parameter dimensions of a system. Returns GS_ERR_INVALID for an unknown id. */
int gs_dims(int32_t system, int32_t* d, int32_t* p);

/* Adaptive ensemble solve (Sec. 2.1-2.2; Appendix A, Eqs. rk, errnorm, controller, dense).
 *  y0 [N,d], params [N,p] (may be NULL when p = 0), t0 [N], t1 [N]: inputs.
 *  saveat [K] non-decreasing output times shared by all trajectories, or [N,K] if
 *    opt->per_traj_saveat. An output at t0 is y0 exactly; an output at t1 is the final state.
 *  y_out [N,K,d]: the solution at the output times (dense output inside steps).
 *  status [N], n_accept [N], n_reject [N] (int32): per-trajectory status bits and step-attempt
 *    counts (rejected attempts included in N_i = n_accept + n_reject, Sec. 2.2).
 *  workspace / workspace_bytes: needed for the persistent kernel (work-queue counter) and for
 *    opt->record_tape; size from gs_workspace_bytes. May be NULL otherwise.
 */
int gs_solve(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
             const double* t1, double rtol, double atol, int32_t K, const double* saveat,
             const gs_options* opt, double* y_out, int32_t* status, int32_t* n_accept,
             int32_t* n_reject, void* workspace, size_t workspace_bytes, void* cuda_stream);

/* Gradient of a scalar loss L through the solve, by the discrete adjoint of the accepted step
 * sequence (the steps are held fixed, so the result is the exact derivative of the numerical
 * solution on that sequence, Sec. 2.3 and Appendix A, Eq. stage-sens).
 *  Inputs as gs_solve, plus dLdy [N,K,d], the cotangent of y_out.
 *  dLdy0 [N,d], dLdparams [N,p] (may be NULL when p = 0): per-trajectory gradients; for
 *    parameters shared by all members the caller sums over n (Appendix A, Eq. chain).
 *  status [N]: as gs_solve, plus GS_ST_TAPE_OVERFLOW. Failed trajectories get NaN gradients.
 *  y_out [N,K,d]: the forward solution of the internal re-solve (may be NULL with reuse_tape).
 *  With opt->reuse_tape, status, n_accept and n_reject are INPUTS: the arrays written by the
 *  recording gs_solve (status gains GS_ST_TAPE_OVERFLOW there); the forward solve is not re-run.
 *  The workspace holds the step tape: per accepted step the state at its start, its time and
 *  its length, in chunks taken from a pool by an atomic counter. Layout: a 256-byte header, int32
 *  head[N], n_rec[N] and order[N] (the longest-first work list), 4096 bucket counters and the
 *  FP32 cost estimates cost[N] (each array padded to 256 bytes), with opt->ckpt_stride > 1 the
 *  int32 output attribution emit[N, K] (the accepted step that produced each output), then chunks;
 *  a trajectory with n accepted steps uses ceil(n / 32) chunks. A chunk is a 16-byte header holding
 *  the previous chunk's index, then
 *  - stride 1: 32 slots. GS_FP64: the state (8 d bytes), GS_FP32_STAGES: its FP32 high part (4 d
 *    bytes, from which the stages are recomputed); then, from the next 8-byte boundary, t, tc and h
 *    as FP64 (h negative for the last, clipped step), the slot padded to 16 bytes:
 *    roundup16(roundup8(state) + 24), 48 bytes for six FP32 components. GS_FP32_DF: roundup16(4 d)
 *    + 16 (time pair, h, flag as FP32); GS_DF64: roundup16(8 d) + 16 (df64 pairs, then as GS_FP32_DF);
 *  - stride S > 1: the 32 step lengths (FP64; FP32 in GS_FP32_DF; the last, clipped step negative),
 *    then 32 / S checkpoints of roundup16(state) + 16 bytes: GS_FP64 state = y and the first stage
 *    (16 d bytes), the FP32 modes its high part, low part and first stage (12 d bytes); then the
 *    time (t, tc as FP64, or the FP32 pair).
 */
int gs_vjp(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
           const double* t1, double rtol, double atol, int32_t K, const double* saveat,
           const gs_options* opt, const double* dLdy, double* dLdy0, double* dLdparams,
           double* y_out, int32_t* status, int32_t* n_accept, int32_t* n_reject, void* workspace,
           size_t workspace_bytes, void* cuda_stream);

/* Size of the built-in scratch array of gs_vjp_noalloc (64 MiB). */
#define GS_NOALLOC_SCRATCH_BYTES (64u << 20)

/* gs_vjp for callers that cannot allocate device memory or pass a workspace (code inside another
 * framework's memory pool, plug-ins whose host owns all device allocations, loops where an
 * allocation could stall). The paper has no counterpart. Same arguments and results as gs_vjp
 * without the workspace; opt->reuse_tape must be 0 (the forward solve is always re-run).
 * The scratch (work counters and step tape) is a GS_NOALLOC_SCRATCH_BYTES array inside the library,
 * present on every GPU that loads it until the process exits; nothing is allocated or freed.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and caches
 * it: make that first call before any stream capture. Calls share the array and it keeps the last
 * call's contents (the call clears what must start at zero); calls that overlap on the GPU race, so
 * issue them one after another. An ensemble whose part before the tape pool
 * (gs_workspace_bytes(system, N, K, opt, 1, 0): 16 N bytes of per-trajectory arrays and the
 * prepared-start rows of the persistent forward (112 to 256 bytes per trajectory by system and
 * precision), padded, the 256-byte header, 16 KB of counters, and 4 N K bytes with a checkpoint
 * stride above 1) plus one
 * tape chunk (gs_tape_chunk_bytes) exceeds the array is rejected with GS_ERR_WORKSPACE (an unknown
 * system with GS_ERR_INVALID first); trajectories whose steps do not fit in the rest of the array
 * get GS_ST_TAPE_OVERFLOW and NaN gradients. A checkpoint stride above 1 fits about S times more
 * steps. */
int gs_vjp_noalloc(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
                   const double* t1, double rtol, double atol, int32_t K, const double* saveat,
                   const gs_options* opt, const double* dLdy, double* dLdy0, double* dLdparams,
                   double* y_out, int32_t* status, int32_t* n_accept, int32_t* n_reject, void* cuda_stream);

/* Workspace bytes for N trajectories. for_vjp = 0: the work counters, the longest-first work list
 * (order[N], bucket counters, cost[N]) and the prepared starts of the persistent forward (one row
 * per trajectory: its state after start-up, written by a one-thread-per-trajectory pass so that a
 * lane of a persistent warp that takes a new trajectory loads it instead of starting it while the
 * other lanes wait; not for GS_DF64). A smaller workspace runs GS_ORDER_AUTO in stored order and
 * starts trajectories in place, and rejects GS_ORDER_ESTIMATE and GS_ORDER_HINT with
 * GS_ERR_WORKSPACE.
 * for_vjp != 0: room for a step tape of `steps_hint` accepted steps per trajectory on average
 * (rounded up to whole chunks per trajectory, plus one), in the chunk size of opt->precision and
 * opt->ckpt_stride (FP64, stride 1 when opt is NULL). With steps_hint = 0: the part before the tape
 * pool (with a checkpoint stride above 1 it includes the int32 output attribution [N, K]); a tape
 * for exactly n_i accepted steps per trajectory then needs (sum_i ceil(n_i / 32) + 1) chunks of
 * gs_tape_chunk_bytes more. A smaller workspace is accepted; trajectories whose steps no longer
 * fit get GS_ST_TAPE_OVERFLOW. Returns 0 for an unknown system, N < 0 or K < 0. */
size_t gs_workspace_bytes(int32_t system, int64_t N, int32_t K, const gs_options* opt, int32_t for_vjp,
                          double steps_hint);

/* Bytes of one step-tape chunk (32 accepted steps of one trajectory) for opt's precision and
 * checkpoint stride (FP64, stride 1 when opt is NULL); 0 for an unknown system or stride. */
size_t gs_tape_chunk_bytes(int32_t system, const gs_options* opt);

/* Forward sensitivities (Sec. 2.3, Eq. sens; Appendix A, Eq. stage-sens): the solve of gs_solve carrying
 * m tangent directions, S = dy/d(direction), integrated with the same Runge-Kutta steps as y (step
 * control on y alone), so S is the exact derivative of the numerical solution on those steps.
 *  dy0 [N,d,m]: S(t0), the direction of the initial state (NULL = 0).
 *  dparams [N,p,m]: the parameter direction (NULL = 0); e.g. unit vectors give dy/dtheta_q.
 *  y_out [N,K,d] as gs_solve; S_out [N,K,d,m]: the sensitivities at the output times.
 *  Precision GS_FP64 or GS_FP32_DF; persistent kernel; the workspace holds its work counter
 *  (gs_workspace_bytes(..., for_vjp = 0, ...)). Directions are processed up to 4 per launch
 *  (1 for GS_VERN7), so m > 4 repeats the solve per group. */
int gs_jvp(int32_t system, int64_t N, const double* y0, const double* params, const double* t0,
           const double* t1, double rtol, double atol, int32_t K, const double* saveat,
           const gs_options* opt, int32_t m, const double* dy0, const double* dparams, double* y_out,
           double* S_out, int32_t* status, int32_t* n_accept, int32_t* n_reject, void* workspace,
           size_t workspace_bytes, void* cuda_stream);

/* Quintessence cosmologies (system GS_SYS_QUINTESSENCE) with the amplitude a0 fixed by spatial flatness
 * (Sec. 4.1, Eq. de-flat): Newton's method on g(a0) = E(0)^2 - 1 = 0, each step one gs_jvp integration
 * to t1 (N = 0, today) carrying S_a0 = dy/da0 and S_Om = dy/dOm; then the derivative along the flat
 * models (Eq. de-ift): da0/dOm = -(dg/dOm)/(dg/da0) and dy/dOm = S_Om + (da0/dOm) S_a0.
 *  params [N,4] (a0, lambda, Om, Or): IN/OUT. params[n,0] is the starting amplitude (the paper starts
 *    from 1 - Om - Or, exact for a field at rest) and is replaced by the solution.
 *  saveat [K] (or [N,K]): output e-folds; the last one must equal t1, where g is evaluated.
 *  y_out [N,K,3]: the solution at the returned a0. dydOm [N,K,3], da0dOm [N], g_out [N] (final E(0)^2 - 1):
 *    may be NULL.
 *  status [N]: as gs_jvp, plus GS_ST_NO_CONVERGENCE. n_accept, n_reject [N]: of the last integration.
 *  n_newton [N]: integrations used until |g| <= gtol (gtol > 0; the residual cannot fall below the
 *    integration's own error, so gtol is usually of the order of rtol).
 *  opt: precision GS_FP64 or GS_FP32_DF, as gs_jvp. workspace: gs_flat_workspace_bytes(N, K) bytes,
 *    256-byte aligned. By default the call synchronises the stream once per Newton iteration (it
 *    reads how many cosmologies are still moving and stops when none is); with opt->graph_safe it
 *    launches all max_newton iterations, the later ones over device-side work lists that may be
 *    empty, and never synchronises, so it can be captured into a CUDA graph. */
int gs_solve_flat(int64_t N, const double* y0, double* params, const double* t0, const double* t1, double rtol,
                  double atol, int32_t K, const double* saveat, const gs_options* opt, int32_t max_newton,
                  double gtol, double* y_out, double* dydOm, double* da0dOm, double* g_out, int32_t* status,
                  int32_t* n_accept, int32_t* n_reject, int32_t* n_newton, void* workspace, size_t workspace_bytes,
                  void* cuda_stream);

/* Workspace bytes of gs_solve_flat for N cosmologies and K outputs (0 for N < 0 or K < 1). */
size_t gs_flat_workspace_bytes(int64_t N, int32_t K);

/* Profile-likelihood fits of the quintessence model (Sec. 4.3, Appendix C, Eq. de-gn): many damped
 * Gauss-Newton minimisations of chi^2 over psi = (Om, H0) at fixed lambda, each on one mock data set.
 * Every iteration is one gs_solve_flat of all fits at n_nodes output redshifts (the flat model and
 * dy/dOm along flat models), then one kernel that forms chi^2, J^T r and J^T J and takes the step. */
typedef struct {
  int32_t method, precision;  /* of the flatness solves (GS_FP64 or GS_FP32_DF) */
  double rtol, atol, gtol;    /* their tolerances and the flatness residual */
  int32_t max_newton;         /* Newton steps per flatness solve (8) */
  int32_t n_iter;             /* Gauss-Newton iterations (20); chi^2 is recomputed after the last */
  double mu;                  /* damping of Eq. de-gn (1e-3) */
  double trust_om, trust_h0;  /* trust region: the step is scaled so |dOm| <= 0.02, |dH0| <= 2 */
  double start_om, start_h0;  /* starting point (0.30, 70 km/s/Mpc) */
  double orad, omega_b, omega_nu; /* Omega_r (9e-5); baryon and neutrino densities in r_d */
  double conv_dchi2, conv_decrement; /* convergence test: |Delta chi^2| < 1e-4, decrement < 1e-6 */
  int32_t graph_safe;         /* flatness solves without host synchronisation (gs_options) */
  int32_t sm_limit;           /* SM budget of the flatness solves' persistent kernels (gs_options) */
} gs_profile_options;

void gs_profile_default_options(gs_profile_options* opt);

/* Bytes of the prepared-data buffer (0 for unsupported sizes: 4 <= n_nodes <= 64, n_bao <= 32). */
size_t gs_profile_prep_bytes(int32_t n_nodes, int32_t n_bao, int32_t n_sn, int32_t n_mocks);

/* One-time preparation of the data (device pointers, row-major):
 *  z_nodes [n_nodes]: output redshifts, ascending, z_nodes[0] = 0, uniform or not in x = ln(1+z);
 *    distances at the data redshifts come from a not-a-knot cubic spline in x of ln(D_M/z), ln D_H.
 *  bao_z, bao_kind [n_bao]: redshift and kind of each BAO point (0 D_V/r_d, 1 D_M/r_d, 2 D_H/r_d);
 *    L_bao [n_bao x n_bao]: lower Cholesky factor of their covariance; d_bao [n_mocks x n_bao].
 *  z_sn [n_sn], L_sn [n_sn x n_sn] (lower Cholesky factor), d_sn [n_mocks x n_sn]: supernova
 *    magnitudes; their absolute magnitude is marginalised (projection orthogonal to L_sn^{-1} 1).
 * The supernova part is reduced to n_nodes x n_nodes quadratic forms in the spline's node values
 * (exact: the spline is linear in them), so the fits never touch n_sn again. */
int gs_profile_prepare(int32_t n_nodes, const double* z_nodes, int32_t n_bao, const double* bao_z,
                       const int32_t* bao_kind, const double* L_bao, int32_t n_sn, const double* z_sn,
                       const double* L_sn, int32_t n_mocks, const double* d_bao, const double* d_sn, void* prep,
                       size_t prep_bytes, void* cuda_stream);

/* Workspace bytes of gs_profile_fit for n_fits fits (0 for unsupported n_nodes). */
size_t gs_profile_workspace_bytes(int64_t n_fits, int32_t n_nodes);

/* n_fits minimisations: lam [n_fits] the fixed slope, mock [n_fits] the data set of each.
 * Outputs [n_fits]: om, H0 at the returned parameters, a0 (flat amplitude there), chi2 recomputed
 * there, decrement = g^T (J^T J)^{-1} g (g = J^T r) there, converged (the test of opt), status
 * (flatness-solve status bits, or GS_ST_NONFINITE for a mock index outside [0, n_mocks); non-zero
 * stops the fit with NaN chi2). Dimensions as prepared. */
int gs_profile_fit(int64_t n_fits, const double* lam, const int32_t* mock, const void* prep, int32_t n_nodes,
                   int32_t n_bao, int32_t n_sn, int32_t n_mocks, const gs_profile_options* opt, double* om, double* H0,
                   double* a0, double* chi2, double* decrement, int32_t* converged, int32_t* status, void* workspace,
                   size_t workspace_bytes, void* cuda_stream);

/* Evaluate f (Eq. ivp) and its vector-Jacobian products for M states, as the solver does:
 *  f [M,d] = f(t, y, theta);  gy [M,d] = J_y^T w;  gp [M,p] = J_theta^T w  (gy, gp may be NULL).
 *  precision selects the FP64 (GS_FP64) or FP32 (the two FP32 modes) instantiation. */
int gs_rhs(int32_t system, int32_t precision, int64_t M, const double* t, const double* y,
           const double* params, const double* w, double* f, double* gy, double* gp, void* cuda_stream);

/* Plain-ALU throughput probe (the paper has no counterpart; the benchmark's roofline denominators):
 * one launch of blocks_per_sm (1..8) blocks of 256 threads per SM, every thread running `iters`
 * rounds of 8 independent multiply-add chains; kind 0: FP32, 1: FP64, 2: FP32 on the packed
 * two-lane multiply-add of sm_100 and later (float2 chains). sink: device array of at least
 * 8 x (multiprocessor count) doubles, one sum per block written (so the work is kept).
 * *fma_count (host) receives the number of multiply-adds launched; time the launch with CUDA events
 * on cuda_stream: FLOP/s = 2 * fma_count / time. */
int gs_alu_probe(int32_t kind, int64_t iters, int32_t blocks_per_sm, double* sink, int64_t* fma_count,
                 void* cuda_stream);

/* Device self-test of the bit-level FP64 helpers the kernels use instead of FP64-pipe instructions
 * (the paper has no counterpart; a GB300 cost, not a method step): FP64 -> FP32 rounding, FP32 -> FP64
 * widening, FP64 <= and ==, NaN and finiteness tests, sign operations (bit for bit on numbers; a NaN
 * gives a NaN), the order of non-negative numbers, log2 to FP32 accuracy (within 2^-20 +
 * 2^-23 |log2 x|) and the step-size floor 16 eps max(|x|, |y|) of finite x, y (bit for bit where it
 * is a normal number), each compared on the device with the instruction or FP64 expression it
 * replaces. n inputs per check from SplitMix64 on the counters seed .. seed + 4n - 1: raw 64-bit
 * patterns, numbers in and around the FP32 range, rounding ties and their neighbours, and a fixed
 * list of edge cases. counts: device array of 2 x GS_SELFTEST_CHECKS entries, set by the call
 * (stream-ordered on cuda_stream): counts[c] the mismatches of check c, counts[GS_SELFTEST_CHECKS + c]
 * the bit pattern of one mismatching input (0 if none). */
#define GS_SELFTEST_CHECKS 9
int gs_selftest(int64_t n, uint64_t seed, unsigned long long* counts, void* cuda_stream);

/* Message for the last non-zero return on this host thread ("" if none). */
const char* gs_last_error(void);

/* Library version string. */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
