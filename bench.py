"""Benchmark: ensemble solves/s and forward+gradient solves/s at a fixed error budget, against the
plain one-thread-per-trajectory FP64 kernel on the same GPU.

Headline workload: 1,048,576 test-particle orbits in the Milky-Way-like potential (Miyamoto-Nagai
disc + Hernquist bulge + z-flattened NFW halo, q ~ U[0.8, 1.2]), seeded ICs with R ~ U[4, 20] kpc,
|z| < 2 kpc, near-circular velocities plus 20 km/s dispersion, integrated 0-3 Gyr with Tsit5; gradient
of L = 1/2 sum ||y(t1) - y_tgt||^2 with respect to y0 and the 4 potential parameters.

Headline arithmetic: the precision split of the build's design, precision mode "fp32": stages and
right-hand sides in FP32 with the state as a compensated FP32 pair, while the accumulation of the
error norm (Eq. errnorm), the time (Kahan-compensated) and the step-size controller (Eq. controller)
stay FP64. The same line reports the FP64 persistent kernel and the FP64 plain kernel (the paper's
one-thread-per-trajectory form in its precision) as top-level entries, and the FP32-pair mode
("fp32df", time and control in FP32 pairs as well: beyond the split) among the variants.

One step = one pass of the whole hot path over the ensemble: the adaptive forward solve recording its
step tape, the loss cotangent, and the discrete-adjoint reverse sweep. Runs use the loosest tolerance
of the quarter-decade grid meeting the budgets (Eq. accept): P99 <= 1e-4 for the orbit state
(Eq. st-fwderr) and, for forward+gradient runs, P99 <= 1e-3 for the sensitivity matrix (Eq.
st-graderr). Every reported error is against the CPU oracle (FP64 Verner 7 at rtol = atol = 1e-13)
on a seeded sample of the same members, computed on the host cores outside the timed regions; a GPU
FP64 Verner 7 solve at rtol 1e-12 of a larger sample is kept as a cross-check.

The default run appends `workloads`: the other configurations (isochrone, spin precession on both
intervals, quintessence distances, flatness shooting, profile-likelihood fits, log-halo streams, the
mixed serving batch), each with its solves/s, errors against the oracle and ALU-roofline fraction.
`--workload NAME` runs one of them alone (fuller variant list). Prints one JSON line (rank 0).
`--impl reference` times the CPU oracle instead.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble solves/s and fwd+grad solves/s at fixed error budget vs plain FP64 on GB300"
N_ORBITS = 1 << 20
T1_MYR = 3000.0
BUDGET = 1e-4       # orbit state, Eq. st-fwderr (Sec. 3)
GRAD_BUDGET = 1e-3  # sensitivity matrix, Eq. st-graderr (Sec. 3, Appendix A)
# Loosest quarter-decade tolerances meeting the budgets on this workload (the tolerance search of
# Appendix A on a 4096-orbit draw; the achieved errors are re-measured on every run below):
# the state budget alone allows 3.16e-8 (FP32 stages) and 5.62e-8 (FP64); the derivative budget
# needs 1e-8 in every precision.
RTOL_FWD_F32 = 3.16e-8
RTOL_FWD_F64 = 5.62e-8
RTOL_GRAD = 1e-8
RTOL_CONFIG = 3e-7  # the tolerance the workload is quoted at; it misses the budget here
HEAD_PREC = "fp32"  # FP32 stages; FP64 norm accumulation, time and controller
ORACLE_RTOL = 1e-13  # the converged reference (Appendix A: the paper's references at 1e-13)

# Algorithmic flops (sqrt, div, log counted as one op each), Tsit5 on the MW system:
#   f:   ~70 add/mul + 4 sqrt + 1 log + 3 div = 78;  VJP of f: ~2.5 f = 195
#   forward attempt: 6 f (FSAL) + 2d (nnz A + nnz(b - bhat)) + ~40 (error norm, controller)
#                    = 468 + 2*6*(21+7) + 40 = 844
#   reverse accepted step: the 6 stages the new state depends on (b_7 = 0): 6 f (k1 included)
#                          + 2d (nnz of A among them + the 5 state updates) = 2*6*(15+5),
#                          6 VJPs, and the cotangent algebra 2d (15 a_lj + 6 b_j) = 2130
# Of the ~40 flops of error norm and controller, the precision split keeps 2d + 5 in FP64: the d
# squares accumulated (2d), the compensated time (4) and the step-size update (1).
# The FP32 modes take the stages of second-order systems (y = (x, v), f = (v, a(x))) in Nystrom form:
# the stage positions from the coefficients (A^2)_jm (zero for m >= j - 1) and the row sums of A,
# over the d/2 position components only, and the position error from ((b - bhat) A)_m. Counted the
# same way, a forward attempt is (S - 1) f + d (nnz A^2 + S - 1) + d (nnz((b - bhat) A) + nnz(b - bhat))
# + 40 = 468 + 6*(15+6) + 6*(6+7) + 40 = 712. A reversed step recomputes its stages with
# d (nnz A^2 among the 6 + 2*5) = 6*(10+10) instead of 2d (15 + 5), and its cotangent algebra, over
# the accelerations' cotangents, is d (nnz A^2 among the 6 + 6 c' terms + nnz b + nnz bA) =
# 6*(10+6+6+5) instead of 2d (15 + 6): 1920.
F_RHS_MW = 78
F_ATT_FWD = 6 * F_RHS_MW + 2 * 6 * (21 + 7) + 40
F_STEP_REV = 6 * F_RHS_MW + 2 * 6 * (15 + 5) + 6 * int(2.5 * F_RHS_MW) + 2 * 6 * (15 + 6)
F_ATT_FWD_NY = 6 * F_RHS_MW + 6 * (15 + 6) + 6 * (6 + 7) + 40
F_STEP_REV_NY = 6 * F_RHS_MW + 6 * (10 + 2 * 5) + 6 * int(2.5 * F_RHS_MW) + 6 * (10 + 6 + 6 + 5)
F64_ATT_SPLIT = 2 * 6 + 5
# Forward flops of the other workloads, the same count for any system and tableau: per attempt
# (S - 1) f + 2d (nnz A + nnz(b - bhat)) + 40, plus 2d nnz b for the new state and one f per accepted
# step (the next step's first stage) when the pair is not FSAL. f counts as written: MW 78, spin
# precession 172 (after the per-binary constants), isochrone 14, log halo 30, quintessence 40.
# Nonzeros of the published tableaux (S, FSAL, nnz A, nnz b, nnz(b - bhat)):
F_RHS = {"mw": 78, "precession": 172, "isochrone": 14, "loghalo": 30, "quintessence": 40}
TABLEAU_NNZ = {"tsit5": (7, True, 21, 6, 7), "dopri5": (7, True, 20, 5, 6), "vern7": (10, False, 36, 7, 8)}
# Nystrom form (FP32 modes, second-order systems, the 7-stage FSAL pairs): nnz A^2 over stages 2..S,
# nnz A^2 over the first 6 stages, nnz((b - bhat) A), nnz(b A)
NYSTROM_NNZ = {"tsit5": (15, 10, 6, 5), "dopri5": (14, 10, 5, 4)}
SECOND_ORDER = ("mw", "isochrone", "loghalo")


def nystrom(system, method, prec):
    return prec in ("fp32", "fp32df") and system in SECOND_ORDER and method in NYSTROM_NNZ


def forward_flops(system, method, d, attempts, accepted, prec="fp64"):
    S, fsal, n_a, n_b, n_e = TABLEAU_NNZ[method]
    f = F_RHS[system]
    if nystrom(system, method, prec):
        n_aa, _, n_ea, _ = NYSTROM_NNZ[method]
        return attempts * ((S - 1) * f + d * (n_aa + S - 1) + d * (n_ea + n_e) + 40)
    per_attempt = (S - 1) * f + 2 * d * (n_a + (0 if fsal else n_b) + n_e) + 40
    return attempts * per_attempt + (0 if fsal else accepted * f)


def reverse_flops(system, method, d, accepted, prec="fp64"):
    """Per accepted step: the stages recomputed (S - 1 f + 2d nnz A), S VJPs at 2.5 f, and the
    cotangent algebra 2d (nnz A + nnz b); in Nystrom form the recomputation d (nnz A^2 among the
    first 6 stages + 2*5) and the algebra d (nnz A^2 among them + 6 + nnz b + nnz bA)."""
    S, fsal, n_a, n_b, n_e = TABLEAU_NNZ[method]
    f = F_RHS[system]
    if nystrom(system, method, prec):
        _, n_aa6, _, n_ba = NYSTROM_NNZ[method]
        recompute, algebra = d * (n_aa6 + 10), d * (n_aa6 + 6 + n_b + n_ba)
    else:
        recompute, algebra = 2 * d * n_a, 2 * d * (n_a + n_b)
    return accepted * ((S - 1) * f + recompute + S * int(2.5 * f) + algebra)


def att_flops(prec):
    """Flops of one Milky-Way Tsit5 forward attempt and one reversed step in precision prec."""
    return (F_ATT_FWD_NY, F_STEP_REV_NY) if nystrom("mw", "tsit5", prec) else (F_ATT_FWD, F_STEP_REV)


# DRAM bytes per accepted step of the headline's kernels (forward recording the tape, reverse), from
# one-pass ncu captures (dram__bytes_read.sum + dram__bytes_write.sum) of the 262,144-orbit, 750-Myr
# case (a tape of a few GB; profiles/), divided by that launch's accepted steps; the traffic is
# proportional to the accepted steps, so it scales to the full launch. None: not captured for that
# kernel, or the kernel changed since.
FWD_DRAM_BYTES_PER_STEP = {"fp32": 58.5, "fp32df": 61.7, "fp64": None}
REV_DRAM_BYTES_PER_STEP = {"fp32": None, "fp32df": None, "fp64": None}  # not re-taken after the Nystrom-form adjoint
# Fallback peaks when the probe cannot run: FP32 from unit counts and clock (152 SMs x 128 FP32
# lanes x 2 flop x 2.07 GHz); FP64 the nominal GB300 rate
PEAK_FP32_DERIVED = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_NOMINAL = 1.25


def log(*a):
    print(*a, file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.strip()]
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_hbm_gbs():
    """The machine's measured HBM copy bandwidth (MEASURED_PEAKS.json beside this file), or None."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


# ------------------------------------------------------------------------------------------------
# CPU oracle: the converged references of every reported error, and the CPU baseline
def oracle_states(e, idx, method="vern7", rtol=ORACLE_RTOL):
    """The CPU oracle's converged solution of the members idx (all host cores): y [n, K, d]."""
    import oracle as O

    s = e.subset(idx)
    atol = 1e-15 if e.system == "quintessence" else rtol
    r = O.solve(e.system, s.y0, s.params if s.params.shape[1] else None, s.t0, s.t1, s.saveat, rtol, atol,
                method=method, max_steps=20_000_000)
    return r["y"], r["status"]


def oracle_sensitivities(e, idx, cols, rtol=ORACLE_RTOL):
    """The oracle's converged forward sensitivities of the final state to the parameter columns
    `cols`, with the final state: (y [n, d], S [n, d, len(cols)])."""
    import oracle as O

    s = e.subset(idx)
    d = s.y0.shape[1]
    r = O.sens(e.system, s.y0, s.params, s.t0, s.t1, s.saveat, rtol, rtol, method="vern7")
    return r["y"][:, -1], r["S"][:, -1][:, :, [d + c for c in cols]]


def cpu_oracle_rate(e, rtol, target_s=15.0, nmax=200000, n=None):
    """The CPU oracle (FP64 same-algorithm solve + forward-sensitivity gradient) on a bounded sample
    of the workload, all host cores: n orbits, or, when n is None, a 1024-orbit pilot sizes a sample
    of about target_s seconds. Returns (solves/s, cores, sample description, n)."""
    import oracle as O

    cores = O.max_threads()
    rng = np.random.default_rng(7)

    def run(n):
        idx = np.sort(rng.choice(e.n, n, replace=False))
        s = e.subset(idx)
        w = rng.normal(size=(n, 1, 6))
        t = time.perf_counter()
        O.grad("mw", s.y0, s.params, s.t0, s.t1, s.saveat, w, rtol=rtol, atol=rtol)
        return time.perf_counter() - t

    if n is None:
        n = min(1024, nmax, e.n)
        dt = run(n)
        if dt < target_s / 4:
            n = int(min(nmax, e.n, max(n, n * target_s / max(dt, 1e-9))))
            dt = run(n)
    else:
        dt = run(n)
    return n / dt, cores, "%d of %d orbits (fwd + forward-sensitivity gradient), %.1f s" % (n, e.n, dt), n


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2609_28458_gb300 import workloads as W

    e = W.mw(n=N_ORBITS, seed=1000, t1=T1_MYR, rtol=RTOL_GRAD)
    # one step: a sample of about 5 s of oracle work, sized once by the first warm-up step
    n_step = None
    for _ in range(max(args.warmup, 1)):
        _, _, _, n_step = cpu_oracle_rate(e, RTOL_GRAD, target_s=5.0, n=n_step)
    t = time.perf_counter()
    rates = []
    for _ in range(args.steps):
        r, cores, sample, _ = cpu_oracle_rate(e, RTOL_GRAD, n=n_step)
        rates.append(r)
    dt = time.perf_counter() - t
    value = float(np.median(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "mw_1048576_orbits_0_3gyr", "system": "mw", "method": "tsit5", "rtol": RTOL_GRAD,
                       "note": "CPU oracle, fwd + gradient by forward sensitivities, bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
class Ctx:
    """Device, timing helpers and the measured ALU peaks shared by the benchmark's parts."""

    def __init__(self, dev):
        import torch

        self.torch = torch
        self.dev = dev
        self.stream = torch.cuda.current_stream(dev)
        self.flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 129 MB L2
        self.flush_buf.fill_(1)  # its kernel loads on first use (a quarter of a second): not in a timed region
        self.peak32 = PEAK_FP32_DERIVED
        self.peak64 = PEAK_FP64_NOMINAL
        self.peak_source = "fallback: FP32 derived from unit counts and 2.07 GHz; FP64 nominal"

    def flush(self):
        self.flush_buf.fill_(1)

    def timed(self, fn, reps=3, warm=1):
        """Mean CUDA-event time (ms) of fn over `reps` runs, L2 flushed before each; and fn's last result."""
        torch = self.torch
        for _ in range(warm):
            self.flush()
            fn()
        torch.cuda.synchronize()
        ts, out = [], None
        for _ in range(reps):
            self.flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            out = fn()
            b.record(self.stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts)), out

    def measure_peaks(self, local):
        """The plain-ALU multiply-add peaks from gs_alu_probe (best of the block counts), with the SM
        clock sampled while it runs."""
        from paper_2609_28458_gb300 import api

        with ClockSampler(local) as clk:
            p32 = max(api.alu_peak(False, blocks_per_sm=b, device=self.dev) for b in (4, 8))
            p64 = max(api.alu_peak(True, blocks_per_sm=b, device=self.dev) for b in (4, 8))
        self.peak32, self.peak64 = p32, p64
        c = clk.summary()
        self.peak_source = ("measured: gs_alu_probe (8 independent FMA chains per thread, 4-8 blocks of 256 per SM), "
                            "best launch; SM clock %s MHz" % c.get("sm_mhz"))
        return {"fp32_tflops": p32, "fp64_tflops": p64, "fp32_derived_tflops": PEAK_FP32_DERIVED,
                "fp64_nominal_tflops": PEAK_FP64_NOMINAL, "clocks": c, "source": self.peak_source}

    def peak(self, prec):
        return self.peak64 if prec == "fp64" else self.peak32

    def frac(self, flops, ms, prec):
        a = flops / (ms / 1e3) / 1e12
        return {"tflops": a, "peak_tflops": self.peak(prec), "frac": a / self.peak(prec),
                "peak_kind": "FP64" if prec == "fp64" else "FP32"}


def _counts(r):
    att = int((r["n_accept"].long() + r["n_reject"].long()).sum().item())
    acc = int(r["n_accept"].long().sum().item())
    return att, acc


# ------------------------------------------------------------------------------------------------
def run_gpu(args):
    import torch

    from paper_2609_28458_gb300 import api, autotune
    from paper_2609_28458_gb300 import build as gsbuild
    from paper_2609_28458_gb300 import metrics as M
    from paper_2609_28458_gb300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        gsbuild.build()
    if world > 1:
        dist.barrier()
    gsbuild.build()
    ctx = Ctx(dev)

    # each rank integrates its own contiguous shard of a world x N-member ensemble (weak scaling: N
    # orbits per GPU; the ensemble is defined block by block, block r seeded 1000 + r, so a rank draws
    # only its own members)
    from paper_2609_28458_gb300 import sharding

    sh_start, sh_stop = sharding.shard_bounds(world * args.n, world, rank)
    assert sh_stop - sh_start == args.n
    e = W.mw(n=args.n, seed=1000 + sh_start // args.n, t1=T1_MYR, rtol=RTOL_GRAD)
    N = e.n
    y0 = torch.as_tensor(e.y0, device=dev)
    pr = torch.as_tensor(e.params, device=dev)
    t0 = torch.as_tensor(e.t0, device=dev)
    t1 = torch.as_tensor(e.t1, device=dev)
    sv = torch.as_tensor(e.saveat, device=dev)
    # target: the endpoint of the same orbits with potential parameters perturbed by 1% (seeded)
    rng = np.random.default_rng(77 + rank)
    ptgt = torch.as_tensor(e.params * (1 + 0.01 * rng.standard_normal(e.params.shape)), device=dev)
    y_tgt = api.solve("mw", y0, ptgt, t0, t1, sv, 1e-9, 1e-9, precision="fp64")["y"].clone()
    stream = ctx.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    free_bytes = torch.cuda.mem_get_info(dev)[0]

    def make(prec, rtol, kernel="persistent"):
        # the plain kernel is the paper's one-thread-per-trajectory form: trajectories in stored order
        order = "natural" if kernel == "plain" else "auto"
        ws = api.Workspace(dev)
        probe = api.solve("mw", y0, pr, t0, t1, sv, rtol, rtol, precision=prec, kernel=kernel, order=order)
        # checkpoint stride: every accepted step while the tape fits half of the free memory, else the
        # smallest stride that fits (the autotuner's memory rule)
        stride = autotune.pick_stride("mw", N, probe["n_accept"], prec, budget_bytes=free_bytes // 2,
                                      kernel=kernel)
        nbytes = api.tape_bytes("mw", N, n_accept=probe["n_accept"], precision=prec, ckpt_stride=stride)

        def step():  # forward with tape, loss cotangent, reverse
            s = api.solve("mw", y0, pr, t0, t1, sv, rtol, rtol, precision=prec, kernel=kernel, order=order,
                          record_tape=True, workspace=ws, tape_nbytes=nbytes, ckpt_stride=stride)
            ev[1].record(stream)
            w = s["y"] - y_tgt  # dL/dy of L = 1/2 ||y(t1) - y_tgt||^2
            ev[2].record(stream)
            g = api.vjp("mw", y0, pr, t0, t1, sv, rtol, rtol, w, precision=prec, kernel=kernel, reuse_tape=s,
                        workspace=ws, order=order, ckpt_stride=stride)
            return s, g

        def fwd():
            return api.solve("mw", y0, pr, t0, t1, sv, rtol, rtol, precision=prec, kernel=kernel, order=order)

        return step, fwd, ws, stride

    peaks = ctx.measure_peaks(local)

    # ---- references on the host cores (outside every timed region): the CPU oracle, converged
    ns_o = min(N, args.oracle_sample)
    idx_o = np.sort(np.random.default_rng(5).choice(N, ns_o, replace=False))
    t = time.perf_counter()
    yref_o, _ = oracle_states(e, idx_o)
    ns_s = min(N, args.oracle_sens_sample)
    idx_s = idx_o[np.random.default_rng(6).choice(ns_o, ns_s, replace=False)]
    idx_s.sort()
    ysref_o, S_ref_o = oracle_sensitivities(e, idx_s, cols=[0, 1, 2, 3])
    oracle_s = time.perf_counter() - t
    rE_o, vE_o = M.orbit_scales("mw", e.y0[idx_o], e.params[idx_o])
    rE_s, vE_s = M.orbit_scales("mw", e.y0[idx_s], e.params[idx_s])
    # cross-check: a GPU FP64 Verner 7 solve at rtol 1e-12 of a larger sample
    ns = min(N, args.acc_sample)
    idx_np = np.sort(np.random.default_rng(5).choice(N, ns, replace=False))
    idx = torch.as_tensor(idx_np, device=dev)
    rE, vE = M.orbit_scales("mw", e.y0[idx_np], e.params[idx_np])
    gref = api.solve("mw", y0[idx], pr[idx], t0[idx], t1[idx], sv, 1e-12, 1e-12, method="vern7", precision="fp64")
    io_t = torch.as_tensor(idx_o, device=dev)
    is_t = torch.as_tensor(idx_s, device=dev)

    def errors(y):
        """Orbit errors (Eq. st-fwderr) of the final states y [N, 1, 6] against the oracle and the
        GPU cross-check."""
        eo = M.orbit_error(y[io_t, -1].cpu().numpy(), yref_o[:, -1], rE_o, vE_o)
        eg = M.orbit_error(y[idx, -1].cpu().numpy(), gref["y"][:, -1].cpu().numpy(), rE, vE)
        return eo, eg

    def sens_err(prec, rtol, kernel="persistent"):
        """Eq. st-graderr of dy(t1)/dtheta by six vector-Jacobian products on the oracle's sample."""
        S = np.zeros((ns_s, 6, 4))
        for i in range(6):
            w = torch.zeros((ns_s, 1, 6), dtype=torch.float64, device=dev)
            w[:, 0, i] = 1.0
            g = api.vjp("mw", y0[is_t], pr[is_t], t0[is_t], t1[is_t], sv, rtol, rtol, w, precision=prec, kernel=kernel)
            S[:, i, :] = g["dLdparams"].cpu().numpy()
        return M.sensitivity_error(S, S_ref_o, rE_s, vE_s, e.params[idx_s])

    def acc_block(y, serr=None):
        eo, eg = errors(y)
        out = {"p99_orbit_err": M.p99(eo), "max_orbit_err": float(eo.max()), "orbit_accepted": M.accepted(eo, BUDGET),
               "gpu_vern7_crosscheck_p99": M.p99(eg)}
        if serr is not None:
            out.update(p99_sensitivity_err=M.p99(serr), max_sensitivity_err=float(serr.max()),
                       sensitivity_accepted=M.accepted(serr, GRAD_BUDGET))
        return out

    # ---------------- headline: fwd+grad in the precision split, persistent kernels ----------------
    step, fwd, ws, head_stride = make(HEAD_PREC, RTOL_GRAD)
    for _ in range(args.warmup):  # the warm-up steps as timed (the flush's kernel loads on first use)
        ctx.flush()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_fwd, t_rev = [], []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            ctx.flush()
            ev[0].record(stream)
            s, g = step()
            ev[3].record(stream)
            torch.cuda.synchronize()
            t_fwd.append(ev[0].elapsed_time(ev[1]))
            t_rev.append(ev[2].elapsed_time(ev[3]))
        stop.record(stream)
        torch.cuda.synchronize()
    total_ms = start.elapsed_time(stop)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = tt.item()
    ms_per_step = total_ms / args.steps
    value = world * N * args.steps / (total_ms / 1e3)
    n_att, n_acc = _counts(s)
    n_bad = int((s["status"] != 0).sum().item())
    acc_head = acc_block(s["y"], sens_err(HEAD_PREC, RTOL_GRAD))
    acc_head["failed_trajectories"] = n_bad
    tape_gb = ws.nbytes / 1e9
    del step, fwd, ws
    torch.cuda.empty_cache()

    # roofline of the dominant kernel of the headline step
    fk, rk = float(np.mean(t_fwd)), float(np.mean(t_rev))
    if rk >= fk:
        dom, flops, dur = "k_reverse_persist (discrete adjoint, %s)" % HEAD_PREC, n_acc * att_flops(HEAD_PREC)[1], rk
        bps = REV_DRAM_BYTES_PER_STEP.get(HEAD_PREC)
        traffic = bps * n_acc if bps else None
    else:
        dom, flops, dur = "k_persist (forward + tape record, %s)" % HEAD_PREC, n_att * att_flops(HEAD_PREC)[0], fk
        bps = FWD_DRAM_BYTES_PER_STEP.get(HEAD_PREC)
        traffic = bps * n_acc if bps else None
    achieved = flops / (dur / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": ctx.peak32, "unit": "TFLOP/s",
                "frac": achieved / ctx.peak32, "traffic": traffic, "peak_source": ctx.peak_source,
                "note": "algorithmic FP32 flops of the launch / its CUDA-event time, against the measured FP32 FMA peak"}
    if dom.startswith("k_persist"):
        # the precision split also keeps 2d + 5 FP64 flops per attempt: the kernel's attainable time is
        # the longer of its FP32 and FP64 work at their measured peaks
        t32 = n_att * att_flops(HEAD_PREC)[0] / (ctx.peak32 * 1e12)
        t64 = n_att * F64_ATT_SPLIT / (ctx.peak64 * 1e12)
        roofline["split_attainable_ms"] = 1e3 * max(t32, t64)
        roofline["frac_of_split_roofline"] = 1e3 * max(t32, t64) / dur
    if traffic is not None:
        roofline["dram_gbs"] = traffic / (dur / 1e3) / 1e9
        hbm = measured_hbm_gbs()
        if hbm:
            roofline["dram_frac_of_measured_hbm"] = roofline["dram_gbs"] / hbm

    # ---------------- forward-only at the state budget ----------------
    _, fwd_h, _, _ = make(HEAD_PREC, RTOL_FWD_F32)
    fwd_ms, sf = ctx.timed(fwd_h, args.steps, 2)
    acc_fwd = acc_block(sf["y"])
    hint = (sf["n_accept"] + sf["n_reject"]).clone()
    fwd_hint_ms, _ = ctx.timed(lambda: api.solve("mw", y0, pr, t0, t1, sv, RTOL_FWD_F32, RTOL_FWD_F32,
                                                 precision=HEAD_PREC, kernel="persistent", order="hint",
                                                 cost_hint=hint), args.steps, 2)
    fwd_att, fwd_acc = _counts(sf)

    # ---------------- end to end through the public API with host buffers ----------------
    host = {k: torch.as_tensor(v).pin_memory() for k, v in
            dict(y0=e.y0, p=e.params, t0=e.t0, t1=e.t1, sv=e.saveat, tgt=y_tgt.cpu().numpy()).items()}
    out_y0 = torch.empty((N, 6), dtype=torch.float64).pin_memory()
    out_p = torch.empty((N, 4), dtype=torch.float64).pin_memory()
    dbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    ws_e2e = api.Workspace(dev)
    tape_nb = api.tape_bytes("mw", N, n_accept=s["n_accept"], precision=HEAD_PREC, ckpt_stride=head_stride)

    def e2e_step():
        for k in host:
            dbuf[k].copy_(host[k], non_blocking=True)
        ss = api.solve("mw", dbuf["y0"], dbuf["p"], dbuf["t0"], dbuf["t1"], dbuf["sv"], RTOL_GRAD, RTOL_GRAD,
                       precision=HEAD_PREC, record_tape=True, workspace=ws_e2e, tape_nbytes=tape_nb,
                       ckpt_stride=head_stride)
        gg = api.vjp("mw", dbuf["y0"], dbuf["p"], dbuf["t0"], dbuf["t1"], dbuf["sv"], RTOL_GRAD, RTOL_GRAD,
                     ss["y"] - dbuf["tgt"], precision=HEAD_PREC, reuse_tape=ss, workspace=ws_e2e,
                     ckpt_stride=head_stride)
        out_y0.copy_(gg["dLdy0"], non_blocking=True)
        out_p.copy_(gg["dLdparams"], non_blocking=True)

    e2e_ms, _ = ctx.timed(e2e_step, args.steps, 1)
    del e2e_step, ws_e2e, dbuf
    torch.cuda.empty_cache()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_y0.numel() * 8 + out_p.numel() * 8

    kernels = [dict(kernel="k_persist (forward + tape record, %s)" % HEAD_PREC, ms=fk,
                    **ctx.frac(n_att * att_flops(HEAD_PREC)[0], fk, HEAD_PREC)),
               dict(kernel="k_reverse_persist (discrete adjoint, %s)" % HEAD_PREC, ms=rk,
                    **ctx.frac(n_acc * att_flops(HEAD_PREC)[1], rk, HEAD_PREC)),
               dict(kernel="k_persist (forward, %s, estimate order)" % HEAD_PREC, ms=fwd_ms,
                    **ctx.frac(fwd_att * att_flops(HEAD_PREC)[0], fwd_ms, HEAD_PREC))]

    # ---------------- FP64 anchors and the other variants, each at its own budget tolerance ----------------
    def arm(prec, kernel, rf, reps):
        stp, _, wsv, stride = make(prec, RTOL_GRAD, kernel)
        g_ms, (sg, _) = ctx.timed(stp, reps, 1)
        ga, gc = _counts(sg)
        acc_g = acc_block(sg["y"])
        del stp, wsv
        torch.cuda.empty_cache()
        _, fw, _, _ = make(prec, rf, kernel)
        f_ms, so = ctx.timed(fw, reps, 1)
        fa, fc = _counts(so)
        kf = dict(kernel="k_%s (forward, %s)" % ("plain" if kernel == "plain" else "persist", prec), ms=f_ms,
                  **ctx.frac(fa * att_flops(prec)[0], f_ms, prec))
        kg = dict(kernel="forward + tape and reverse, %s %s" % (kernel, prec), ms=g_ms,
                  **ctx.frac(ga * att_flops(prec)[0] + gc * att_flops(prec)[1], g_ms, prec))
        row = {"precision": prec, "kernel": kernel, "reps": reps, "ckpt_stride": stride,
               "fwd_rtol": rf, "fwd_ms": f_ms, "fwd_solves_per_s": world * N / (f_ms / 1e3),
               "fwd_accuracy": acc_block(so["y"]), "fwd_frac_of_peak": kf["frac"],
               "fwd_grad_rtol": RTOL_GRAD, "fwd_grad_ms": g_ms, "fwd_grad_solves_per_s": world * N / (g_ms / 1e3),
               "fwd_grad_accuracy": acc_g, "fwd_grad_frac_of_peak": kg["frac"], "peak_kind": kf["peak_kind"]}
        return row, [kf, kg]

    variants = {}
    anchors = {}
    if not args.skip_variants:
        for name, prec, kern, rf in (("fp64_persistent", "fp64", "persistent", RTOL_FWD_F64),
                                     ("fp64_plain", "fp64", "plain", RTOL_FWD_F64)):
            row, ks = arm(prec, kern, rf, args.anchor_reps)
            anchors[name] = row
            kernels += ks
            log(name, json.dumps(row))
        row, ks = arm("fp32df", "persistent", RTOL_FWD_F32, args.anchor_reps)
        row["note"] = "beyond the precision split: time as an FP32 pair, error norm and controller in FP32"
        variants["fp32df"] = row
        kernels += ks
        # the workload's quoted tolerance, for context (it misses the budget on this workload)
        _, fwc, _, _ = make(HEAD_PREC, RTOL_CONFIG)
        c_ms, sc = ctx.timed(fwc, 1, 1)
        eo, _ = errors(sc["y"])
        variants["quoted_rtol_3e-7"] = {"precision": HEAD_PREC, "fwd_rtol": RTOL_CONFIG, "fwd_ms": c_ms,
                                        "fwd_p99_orbit_err": M.p99(eo), "accepted": M.accepted(eo, BUDGET)}

    cpu = None
    if rank == 0 and not args.skip_cpu:
        r, cores, sample, _ = cpu_oracle_rate(e, RTOL_GRAD)
        cpu = {"value": r, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample}

    workloads = {}
    if rank == 0 and not args.skip_workloads:
        for name in ("isochrone", "precession", "precession_paper", "quintessence", "quintessence_flat",
                     "streams", "profile", "mixed"):
            t = time.perf_counter()
            try:
                workloads[name] = WORKLOADS[name](ctx, quick=True)
            except Exception as exc:  # a failing workload is reported, not fatal to the headline line
                workloads[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            workloads[name]["wall_s"] = time.perf_counter() - t
            log(name, json.dumps(workloads[name])[:2000])
            torch.cuda.empty_cache()

    if rank == 0:
        base = anchors.get("fp64_plain")
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "mw_1048576_orbits_0_3gyr", "N_per_gpu": N, "system": "mw", "method": "tsit5",
                       "precision": HEAD_PREC,
                       "arithmetic": "FP32 stages and right-hand sides, state as a compensated FP32 pair; FP64 "
                                     "error-norm accumulation, Kahan-compensated FP64 time, FP64 step-size controller",
                       "kernel": "persistent forward (tape) + persistent reverse", "ckpt_stride": head_stride,
                       "rtol": RTOL_GRAD, "atol": RTOL_GRAD, "t1_myr": T1_MYR,
                       "budgets": {"orbit_p99": BUDGET, "sensitivity_p99": GRAD_BUDGET},
                       "parallelism": ("replicas: rank %d of %d integrates members [%d, %d) of %d" %
                                       (rank, world, sh_start, sh_stop, world * N)) if world > 1 else "single GPU",
                       "l2": "L2 flushed (256 MB write) before every timed step; tape %.0f GB per step" % tape_gb},
            "fwd_solves_per_s": world * N / (fwd_ms / 1e3),
            "fwd": {"rtol": RTOL_FWD_F32, "ms": fwd_ms, "accuracy": acc_fwd,
                    "order": "longest first by the per-member estimate", "ms_hint_order": fwd_hint_ms,
                    "hint_solves_per_s": world * N / (fwd_hint_ms / 1e3)},
            "kernel_ms": {"forward_record": fk, "reverse": rk},
            "accuracy": dict(acc_head, reference="CPU oracle: FP64 Verner 7 at rtol = atol = %g, %d orbits for the "
                             "state and %d for the sensitivity matrix (%.1f s on the host cores); cross-check: GPU "
                             "FP64 Verner 7 at rtol 1e-12 on %d orbits" % (ORACLE_RTOL, ns_o, ns_s, oracle_s, ns)),
            "fp64_persistent_fwd_grad_solves_per_s": anchors.get("fp64_persistent", {}).get("fwd_grad_solves_per_s"),
            "fp64_persistent_fwd_solves_per_s": anchors.get("fp64_persistent", {}).get("fwd_solves_per_s"),
            "fp64_persistent_fwd_grad_frac_of_fp64_peak": anchors.get("fp64_persistent", {}).get("fwd_grad_frac_of_peak"),
            "fp64_plain_fwd_grad_solves_per_s": base["fwd_grad_solves_per_s"] if base else None,
            "fp64_plain_fwd_solves_per_s": base["fwd_solves_per_s"] if base else None,
            "fp64": anchors,
            "variants": variants,
            "speedup_vs_plain_fp64": ({"fwd": base["fwd_ms"] / fwd_ms, "fwd_grad": base["fwd_grad_ms"] / ms_per_step}
                                      if base else None),
            "step_attempts": {"mean": n_att / N, "accepted_mean": n_acc / N},
            "roofline": roofline,
            "peaks": peaks,
            "kernels": kernels,
            "workloads": workloads,
            "cpu_baseline": cpu,
            "e2e": {"value": world * N / (e2e_ms / 1e3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # per step: the forward's cost estimate, histogram, scan and scatter of its longest-first
            # work list and k_persist; the reverse's histogram, scan, scatter and k_reverse_persist
            "gpu_launches": (5 + 4) * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# The other configurations. Each returns a dict; quick=True is the reduced form the default run
# embeds (fewer variants, two timed repetitions), quick=False the fuller `--workload NAME` run.
def _solve_rows(ctx, system, e, rows, errfn, reps, grad_stride=None):
    """Times each (precision, kernel, method, rtol, atol, grad) row on ensemble e; errors by errfn."""
    import torch

    from paper_2609_28458_gb300 import api, autotune

    dev = ctx.dev
    d, p = e.y0.shape[1], e.params.shape[1]
    y0 = torch.as_tensor(e.y0, device=dev)
    pr = torch.as_tensor(e.params, device=dev) if p else None
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    K = e.saveat.shape[-1]
    out = []
    for row_spec in rows:
        prec, kern, meth, rtol, atol, grad = row_spec[:6]
        row_stride = row_spec[6] if len(row_spec) > 6 else grad_stride
        kw = dict(method=meth, precision=prec, kernel=kern, max_steps=2_000_000,
                  order="natural" if kern == "plain" else "auto")
        f_ms, s = ctx.timed(lambda: api.solve(system, y0, pr, t0, t1, sv, rtol, atol, **kw), reps, 1)
        att, acc = _counts(s)
        row = {"precision": prec, "kernel": kern, "method": meth, "rtol": rtol, "atol": atol, "fwd_ms": f_ms,
               "fwd_solves_per_s": e.n / (f_ms / 1e3), "us_per_solve": 1e3 * f_ms / e.n,
               "attempts_mean": att / e.n, "failed": int(((s["status"] & 7) != 0).sum().item())}
        row.update(errfn(s["y"]))
        if system in F_RHS and prec != "df64":
            row["fwd_frac_of_peak"] = ctx.frac(forward_flops(system, meth, d, att, acc, prec), f_ms, prec)["frac"]
            row["peak_kind"] = "FP64" if prec == "fp64" else "FP32"
        if grad:
            stride = row_stride or autotune.pick_stride(system, e.n, s["n_accept"], prec,
                                                         budget_bytes=torch.cuda.mem_get_info(dev)[0] // 2,
                                                         kernel=kern, K=K)
            ws = api.Workspace(dev)
            nb = api.tape_bytes(system, e.n, n_accept=s["n_accept"], precision=prec, K=K, ckpt_stride=stride)
            w = torch.ones_like(s["y"])

            def fg():
                ss = api.solve(system, y0, pr, t0, t1, sv, rtol, atol, record_tape=True, workspace=ws, tape_nbytes=nb,
                               ckpt_stride=stride, **kw)
                return api.vjp(system, y0, pr, t0, t1, sv, rtol, atol, w, reuse_tape=ss, workspace=ws,
                               ckpt_stride=stride, **kw)

            g_ms, _ = ctx.timed(fg, reps, 1)
            row.update(fwd_grad_ms=g_ms, fwd_grad_solves_per_s=e.n / (g_ms / 1e3), ckpt_stride=stride,
                       tape_gb=nb / 1e9)
            if system in F_RHS and prec != "df64":
                fl = forward_flops(system, meth, d, att, acc, prec) + reverse_flops(system, meth, d, acc, prec)
                row["fwd_grad_frac_of_peak"] = ctx.frac(fl, g_ms, prec)["frac"]
            del ws
        out.append(row)
        torch.cuda.empty_cache()
    return out


def wl_isochrone(ctx, quick=True):
    """Configuration 1: 4096 isochrone orbits, Tsit5 rtol 1e-10 atol 1e-12, 11 outputs on [0, 100]:
    same-algorithm parity with the oracle (the 1e-9 gate) and the error against its converged solve."""
    import oracle as O
    from paper_2609_28458_gb300 import metrics as M
    from paper_2609_28458_gb300 import workloads as W

    e = W.isochrone(n=4096, seed=0)
    same = O.solve("isochrone", e.y0, None, e.t0, e.t1, e.saveat, e.rtol, e.atol, method="tsit5")["y"]
    conv, _ = oracle_states(e, np.arange(e.n))
    rE, vE = M.orbit_scales("isochrone", e.y0, None)

    def errfn(y):
        y = y.cpu().numpy()
        rel = np.max(np.linalg.norm(y - same, axis=-1) / np.linalg.norm(same, axis=-1), axis=-1)
        er = M.orbit_error(y, conv, rE, vE)
        return {"parity_max_rel_vs_oracle": float(rel.max()), "parity_gate_1e-9": bool(rel.max() <= 1e-9),
                "p99_orbit_err": M.p99(er), "max_orbit_err": float(er.max())}

    rows = [("fp64", "plain", "tsit5", 1e-10, 1e-12, False), ("fp64", "persistent", "tsit5", 1e-10, 1e-12, True)]
    if not quick:
        rows += [("df64", "plain", "tsit5", 1e-10, 1e-12, False), ("df64", "persistent", "tsit5", 1e-10, 1e-12, True)]
    return {"config": "4096 isochrone orbits, t in [0, 100], 11 outputs, Tsit5 rtol 1e-10 atol 1e-12",
            "reference": "CPU oracle: same-algorithm solve (parity) and Verner 7 at 1e-13 (error), all 4096",
            "rows": _solve_rows(ctx, "isochrone", e, rows, errfn, 2 if quick else 3)}


def _wl_precession(ctx, quick=True, paper=False):
    from paper_2609_28458_gb300 import metrics as M
    from paper_2609_28458_gb300 import workloads as W

    e = W.precession(n=1_000_000, seed=2000, paper_interval=paper)
    ns = 2048
    idx = np.sort(np.random.default_rng(5).choice(e.n, ns, replace=False))
    ref, _ = oracle_states(e, idx)
    ok = e.t1[idx] > e.t0[idx]

    def errfn(y):
        er = M.precession_error(y.cpu().numpy()[idx][:, -1], ref[:, -1])[ok]
        return {"p99_angle_err": M.p99(er), "max_angle_err": float(er.max()), "accepted_2e-7": M.accepted(er, 2e-7)}

    rows = [("fp64", "persistent", "vern7", 3.16e-9, 3.16e-9, True), ("fp64", "plain", "vern7", 3.16e-9, 3.16e-9, False),
            ("fp64", "persistent", "tsit5", 5.62e-10, 5.62e-10, False)]
    if paper:  # the gradient also with checkpoint stride 16: its tape is a sixth of stride 1's
        rows = [("fp64", "persistent", "vern7", 3.16e-9, 3.16e-9, True),
                ("fp64", "persistent", "vern7", 3.16e-9, 3.16e-9, True, 16),
                ("fp64", "persistent", "tsit5", 5.62e-10, 5.62e-10, False)]
    if not quick:
        rows += [("fp64", "plain", "tsit5", 5.62e-10, 5.62e-10, False)]
    # the paper's interval takes ~4 s forward and ~12 s forward + gradient per 10^6 solves: one timed
    # repetition after the warm-up in the default run
    out = _solve_rows(ctx, "precession", e, rows, errfn, (1 if paper else 2) if quick else 3)
    return {"config": "10^6 binary spin-precession solves (state 9, FP64), %s" %
                      ("the paper's interval r = 100 M -> 10 M (v = 0.1 -> 10^-1/2)" if paper else
                       "f = 20 Hz (GW) to v = 0.3; binaries above ~87 Msun have an empty interval"),
            "empty_intervals": int((e.t1 <= e.t0).sum()), "budget_rad": 2e-7,
            "reference": "CPU oracle, Verner 7 at 1e-13, %d binaries" % ns, "rows": out}


def wl_precession(ctx, quick=True):
    return _wl_precession(ctx, quick, paper=False)


def wl_precession_paper(ctx, quick=True):
    return _wl_precession(ctx, quick, paper=True)


def wl_quintessence(ctx, quick=True):
    from paper_2609_28458_gb300 import metrics as M
    from paper_2609_28458_gb300 import workloads as W

    e = W.quintessence(n=10_000, seed=3000)
    ns = 2048
    idx = np.sort(np.random.default_rng(5).choice(e.n, ns, replace=False))
    ref, _ = oracle_states(e, idx)

    def errfn(y):
        er = M.distance_error(y.cpu().numpy()[idx], ref, e.params[idx], e.saveat)
        return {"p99_distance_err": M.p99(er), "max_distance_err": float(er.max()), "accepted_1e-4": M.accepted(er, 1e-4)}

    rows = [("fp32", "persistent", "dopri5", 1e-4, 1e-7, True), ("fp32df", "persistent", "dopri5", 1e-4, 1e-7, True),
            ("fp32df", "persistent", "tsit5", 1e-4, 1e-7, True), ("fp64", "plain", "tsit5", 1e-6, 1e-9, True)]
    if not quick:
        rows += [(p, "persistent", m, r, 1e-3 * r, True) for r in (1e-5, 1e-6) for m in ("dopri5", "tsit5")
                 for p in ("fp32", "fp32df")]
    return {"config": "10^4 quintessence cosmologies, z = 50 -> 0, distances at 7 redshifts and today",
            "reference": "CPU oracle, Verner 7 at rtol 1e-13, atol 1e-15, %d cosmologies" % ns,
            "rows": _solve_rows(ctx, "quintessence", e, rows, errfn, 3)}


def wl_quintessence_flat(ctx, quick=True):
    """NEXT-2: dark-energy distances for 10^6 cosmologies with the amplitude supplied, and with the
    flatness condition solved by Newton (Eq. de-flat) with da0/dOm and dy/dOm (Eq. de-ift)."""
    import torch

    import oracle.flat as OF
    from paper_2609_28458_gb300 import api
    from paper_2609_28458_gb300 import metrics as M
    from paper_2609_28458_gb300 import workloads as W

    dev = ctx.dev
    rtol, gtol = 1e-4, 1e-5
    rows = []
    for n in ((1_000_000,) if quick else (10_000, 100_000, 1_000_000)):
        e = W.quintessence(n=n, seed=3000, rtol=rtol)
        y0 = torch.as_tensor(e.y0, device=dev)
        t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
        start = torch.as_tensor(e.params, device=dev)
        kw = dict(method="tsit5", precision="fp32df")
        fl = api.solve_flat(y0, start, t0, t1, sv, rtol, 1e-3 * rtol, gtol=gtol, **kw)
        flat_params = fl["params"].clone()
        sup_ms, _ = ctx.timed(lambda: api.solve("quintessence", y0, flat_params, t0, t1, sv, rtol, 1e-3 * rtol,
                                                kernel="persistent", **kw), 3, 1)
        sol_ms, _ = ctx.timed(lambda: api.solve_flat(y0, start, t0, t1, sv, rtol, 1e-3 * rtol, gtol=gtol, **kw), 3, 1)
        ns = 256
        idx = np.sort(np.random.default_rng(5).choice(n, ns, replace=False))
        ref = OF.solve_flat(e.y0[idx], e.params[idx], e.t0[idx], e.t1[idx], e.saveat, 1e-12, 1e-14, method="vern7",
                            gtol=1e-12, max_newton=12)
        pg = flat_params.cpu().numpy()[idx]
        pr_ = e.params[idx].copy()
        pr_[:, 0] = ref["a0"]
        dm, dh = M.distances(fl["y"].cpu().numpy()[idx], pg, e.saveat)
        dmr, dhr = M.distances(ref["y"], pr_, e.saveat)
        err = np.maximum(np.abs(dm - dmr).max(1), np.abs(dh - dhr).max(1))
        st = fl["status"].cpu().numpy()
        rows.append({"n": n, "rtol": rtol, "gtol": gtol, "method": "tsit5", "precision": "fp32df",
                     "a0_supplied_ms": sup_ms, "a0_supplied_us_per_cosmology": 1e3 * sup_ms / n,
                     "a0_solved_ms": sol_ms, "a0_solved_us_per_cosmology": 1e3 * sol_ms / n,
                     "newton_mean": float(fl["n_newton"].double().mean()),
                     "unconverged": int(((st & 64) != 0).sum()), "failed": int(((st & 7) != 0).sum()),
                     "p99_distance_err": M.p99(err), "max_distance_err": float(err.max()),
                     "accepted_1e-4": M.accepted(err, 1e-4),
                     "a0_max_abs_err": float(np.abs(pg[:, 0] - ref["a0"]).max())})
        torch.cuda.empty_cache()
    return {"config": "flat quintessence cosmologies (Newton on a0), Tsit5 FP32-pair rtol 1e-4",
            "reference": "CPU oracle flatness solve (Verner 7, rtol 1e-12, |g| <= 1e-12) on 256 cosmologies",
            "rows": rows}


def wl_streams(ctx, quick=True):
    """NEXT-4: the paper's stream system (Sec. 3): orbits in the flattened logarithmic halo with the
    final state's sensitivity to (v_c, q) integrated in the same launch (gs_jvp), at the loosest
    quarter-decade tolerance meeting both budgets (1.78e-7, Appendix A search)."""
    import torch

    from paper_2609_28458_gb300 import api
    from paper_2609_28458_gb300 import metrics as M
    from paper_2609_28458_gb300 import workloads as W

    dev = ctx.dev
    n = 1_000_000
    e = W.loghalo(n=n, seed=4000)
    dp = np.zeros((n, 3, 2))
    dp[:, 0, 0] = 1.0
    dp[:, 2, 1] = 1.0
    T = dict(y0=torch.as_tensor(e.y0, device=dev), p=torch.as_tensor(e.params, device=dev),
             t0=torch.as_tensor(e.t0, device=dev), t1=torch.as_tensor(e.t1, device=dev),
             sv=torch.as_tensor(e.saveat, device=dev), dp=torch.as_tensor(dp, device=dev))
    ns = 1024
    idx = np.sort(np.random.default_rng(5).choice(n, ns, replace=False))
    yref, Sref = oracle_sensitivities(e, idx, cols=[0, 2])
    rE, vE = M.orbit_scales("loghalo", e.y0[idx], e.params[idx])
    Dm = e.params[idx][:, [0, 2]]
    it = torch.as_tensor(idx, device=dev)
    rows = []
    for prec in ("fp32df", "fp64"):
        rtol = 1.78e-7
        f_ms, s = ctx.timed(lambda: api.solve("loghalo", T["y0"], T["p"], T["t0"], T["t1"], T["sv"], rtol, rtol,
                                              precision=prec, kernel="persistent"), 3, 1)
        g_ms, j = ctx.timed(lambda: api.jvp("loghalo", T["y0"], T["p"], T["t0"], T["t1"], T["sv"], rtol, rtol,
                                            dparams=T["dp"], precision=prec), 3, 1)
        ey = M.orbit_error(j["y"][it, -1].cpu().numpy(), yref, rE, vE)
        eS = M.sensitivity_error(j["S"][it, -1].cpu().numpy(), Sref, rE, vE, Dm)
        rows.append({"precision": prec, "rtol": rtol, "fwd_us_per_orbit": 1e3 * f_ms / n,
                     "fwd_sens_us_per_orbit": 1e3 * g_ms / n, "fwd_orbits_per_s": n / (f_ms / 1e3),
                     "fwd_sens_orbits_per_s": n / (g_ms / 1e3), "p99_state_err": M.p99(ey),
                     "p99_sensitivity_err": M.p99(eS),
                     "accepted": M.accepted(ey, 1e-4) and M.accepted(eS, 1e-3)})
        del s, j
        torch.cuda.empty_cache()
    return {"config": "10^6 log-halo orbits (v_c, R_c, q) = (1, 0.2, 0.7), 3.7 periods, Tsit5, sensitivities to (v_c, q)",
            "reference": "CPU oracle forward sensitivities, Verner 7 at 1e-13, %d orbits" % ns, "rows": rows}


def wl_profile(ctx, quick=True):
    """NEXT-3: 100 slopes x 100 mock data sets = 10^4 Gauss-Newton minimisations of chi^2 over
    (Om, H0), 20 iterations each (Sec. 4.3, Appendix C), with FP64 flatness solves."""
    import torch

    import oracle.profile as OP
    from paper_2609_28458_gb300 import api
    from paper_2609_28458_gb300 import workloads as W

    n_lam, n_mock = 100, 100
    data = W.profile_data(n_lam=n_lam)
    bao, sn = W.profile_truth_lcdm(data)
    C_bao = W.bao_covariance(data, bao)
    mb = W.profile_mocks(bao, C_bao, n_mock, seed=5002)
    ms = W.profile_mocks(sn, data.sn_cov, n_mock, seed=5003)
    Lb, Ls = np.linalg.cholesky(C_bao), np.linalg.cholesky(data.sn_cov)
    t = time.time()
    pd = api.ProfileData(data.z_nodes, data.bao_z, data.bao_kind, Lb, data.z_sn, Ls, mb, ms, device=ctx.dev)
    torch.cuda.synchronize()
    prep_s = time.time() - t
    lam = np.repeat(data.lam_grid, n_mock)
    mock = np.tile(np.arange(n_mock), n_lam)
    n = len(lam)
    kw = dict(precision="fp64", rtol=1e-8, atol=1e-11, gtol=1e-10)
    fit_ms, r = ctx.timed(lambda: api.profile_fit(pd, lam, mock, n_iter=20, **kw), 1 if quick else 2, 1)
    r = {k: v.cpu().numpy() for k, v in r.items()}
    # the oracle's own Gauss-Newton fit (data-space whitening) of a few of the same minimisations
    pick = [0, 2525, 5050, 9999]
    d_om, d_h0 = [], []
    for i in pick:
        o = OP.gn_fit(lam[i], mb[mock[i]], ms[mock[i]], data, Lb, Ls, n_iter=20)
        d_om.append(abs(o["om"] - r["om"][i]))
        d_h0.append(abs(o["H0"] - r["H0"][i]))
    return {"config": "10^4 profile-likelihood fits (100 lambda x 100 mocks), 20 GN iterations, 1701 SNe, 13 BAO",
            "fits": n, "prepare_s": prep_s, "fit_ms": fit_ms, "us_per_iteration_per_fit": 1e3 * fit_ms / (20 * n),
            "converged_fraction": float(np.mean(r["converged"] == 1)), "failed": int(np.sum(r["status"] != 0)),
            "oracle_check": {"fits": len(pick), "max_abs_om_diff": float(max(d_om)), "max_abs_H0_diff": float(max(d_h0)),
                             "reference": "oracle Gauss-Newton fit with data-space whitening"}}


def wl_mixed(ctx, quick=True):
    """Configuration 5: the three pieces (10^4 fits, 2^18 orbit gradients, 2^17 precession gradients)
    in one CUDA graph on concurrent streams, against the same pieces one after another."""
    import torch

    from paper_2609_28458_gb300 import api, autotune, serving

    rows = []
    for variant, mw_prec in ((("fp32_stages", "fp32"),) if quick else (("fp32_stages", "fp32"), ("fp32df", "fp32df"),
                                                                        ("full_fp64", "fp64"))):
        P = serving.pieces(mw_precision=mw_prec)
        shares, alone = autotune.share_sms(P, reps=1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for f in P.values():
            f(0)
        b.record()
        torch.cuda.synchronize()
        seq = a.elapsed_time(b)
        mb = api.MixedBatch(P, sm_limits=shares)
        best, out = ctx.timed(mb.replay, 2, 1)
        rows.append({"variant": variant, "sm_limits": shares, "alone_ms": alone, "sequential_ms": seq, "graph_ms": best,
                     "fits_converged_fraction": float((out["fits"]["converged"] == 1).double().mean()),
                     "orbit_failures": int((out["orbits"]["status"] != 0).sum()),
                     "precession_failures": int(((out["precession"]["status"] & 7) != 0).sum()),
                     "throughput": {"fits_per_s": 10_000 / (best / 1e3), "orbit_grads_per_s": (1 << 18) / (best / 1e3),
                                    "precession_grads_per_s": (1 << 17) / (best / 1e3)}})
        del mb, P, out
        torch.cuda.empty_cache()
    return {"config": "mixed serving batch: 10^4 fits + 2^18 MW orbit gradients + 2^17 precession gradients",
            "rows": rows}


WORKLOADS = {"isochrone": wl_isochrone, "precession": wl_precession, "precession_paper": wl_precession_paper,
             "quintessence": wl_quintessence, "quintessence_flat": wl_quintessence_flat, "streams": wl_streams,
             "profile": wl_profile, "mixed": wl_mixed}


def run_workload(args):
    import torch

    from paper_2609_28458_gb300 import build as gsbuild

    gsbuild.build()
    _, _, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = Ctx(dev)
    peaks = ctx.measure_peaks(local)
    out = WORKLOADS[args.workload](ctx, quick=False)
    print(json.dumps({"metric": METRIC, "workload": args.workload, "peaks": peaks, **out}), flush=True)


def run_case(args):
    """Small profiling cases of the headline kernels (no JSON line): the seeded MW workload with
    --n orbits at --rtol, solved twice. 'fwd': persistent forward without a tape; 'fwdrev': forward
    recording its tape (checkpoint stride --ckpt-stride), then the persistent reverse sweep.
    --t1-myr shortens the orbits so that a case with several trajectories per lane keeps its tape to
    a few GB. 'prec': --n spin-precession solves, FP64 Verner 7 persistent forward. 'plain64': the
    FP64 plain-kernel baseline forward."""
    import torch

    from paper_2609_28458_gb300 import api
    from paper_2609_28458_gb300 import build as gsbuild
    from paper_2609_28458_gb300 import workloads as W

    gsbuild.build()
    dev = torch.device("cuda")
    if args.case == "plain64":  # the FP64 one-thread-per-trajectory baseline, stored order, no tape
        e = W.mw(n=args.n, seed=1000, t1=args.t1_myr)
        y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
        t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
        for _ in range(2):
            s = api.solve("mw", y0, pr, t0, t1, sv, RTOL_FWD_F64, RTOL_FWD_F64, precision="fp64", kernel="plain",
                          order="natural")
        torch.cuda.synchronize()
        log("case plain64: n=%d failed=%d mean attempts %.1f" % (args.n, int((s["status"] != 0).sum()),
                                                                float((s["n_accept"] + s["n_reject"]).double().mean())))
        return
    if args.case == "prec":  # spin precession, FP64 Verner 7, persistent forward (the workload's kernel)
        p = W.precession(n=args.n, seed=2000)
        py0, pp = torch.as_tensor(p.y0, device=dev), torch.as_tensor(p.params, device=dev)
        pt0, pt1, psv = (torch.as_tensor(x, device=dev) for x in (p.t0, p.t1, p.saveat))
        for _ in range(2):
            s = api.solve("precession", py0, pp, pt0, pt1, psv, 3.16e-9, 3.16e-9, method="vern7", precision="fp64",
                          kernel="persistent")
        torch.cuda.synchronize()
        log("case prec: n=%d status!=0 %d mean attempts %.1f" % (args.n, int((s["status"] != 0).sum()),
                                                                 float((s["n_accept"] + s["n_reject"]).double().mean())))
        return
    e = W.mw(n=args.n, seed=1000, t1=args.t1_myr)
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    kw = dict(precision=args.precision, kernel="persistent")
    if args.case == "fwd":
        for _ in range(2):
            s = api.solve("mw", y0, pr, t0, t1, sv, args.rtol, args.rtol, **kw)
    else:
        ws = api.Workspace(dev)
        probe = api.solve("mw", y0, pr, t0, t1, sv, args.rtol, args.rtol, **kw)
        nb = api.tape_bytes("mw", args.n, n_accept=probe["n_accept"], precision=args.precision,
                            ckpt_stride=args.ckpt_stride)
        for _ in range(2):
            s = api.solve("mw", y0, pr, t0, t1, sv, args.rtol, args.rtol, record_tape=True, workspace=ws,
                          tape_nbytes=nb, ckpt_stride=args.ckpt_stride, **kw)
            api.vjp("mw", y0, pr, t0, t1, sv, args.rtol, args.rtol, s["y"] - 0.0, reuse_tape=s, workspace=ws,
                    ckpt_stride=args.ckpt_stride, **kw)
    torch.cuda.synchronize()
    log("case %s: n=%d failed=%d mean accepted steps %.1f" % (args.case, args.n, int((s["status"] != 0).sum()),
                                                              float(s["n_accept"].double().mean())))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_ORBITS)
    ap.add_argument("--acc-sample", type=int, default=16384)
    ap.add_argument("--oracle-sample", type=int, default=4096)
    ap.add_argument("--oracle-sens-sample", type=int, default=256)
    ap.add_argument("--anchor-reps", type=int, default=3, help="timed repetitions of the FP64 anchors")
    ap.add_argument("--skip-variants", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-workloads", action="store_true")
    ap.add_argument("--case", choices=["fwd", "fwdrev", "prec", "plain64"], help="run a small profiling case instead")
    ap.add_argument("--t1-myr", type=float, default=T1_MYR, help="orbit length of a --case run")
    ap.add_argument("--workload", default="mw", choices=["mw"] + sorted(WORKLOADS))
    ap.add_argument("--precision", default=HEAD_PREC)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--ckpt-stride", type=int, default=1)
    args = ap.parse_args()
    if args.case:
        run_case(args)
    elif args.workload != "mw":
        run_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
