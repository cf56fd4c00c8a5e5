"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances:
* FP64, isochrone workload (4096 orbits, Tsit5, rtol 1e-10, atol 1e-12, 11 outputs): every output
  of every trajectory within 1e-9 relative of the oracle's same-algorithm solve.
* FP64, other systems: trajectories whose accepted/rejected step counts equal the oracle's (the
  same step sequence) agree to 1e-10 relative; a trajectory whose sequence differs (a rounding-level
  difference flipped one accept test) still agrees to 50 x rtol, and such flips must be rare.
* FP32 stages: the error against the converged oracle (Verner 7, rtol 1e-12) meets the paper's
  budget in the paper's measure (Eq. accept): P99 <= 1e-4 for orbits (Eq. st-fwderr) and for
  distances in c/H0 (Sec. 4.2).
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import gpu_solve, rel_err
from paper_2609_28458_gb300 import metrics as M
from paper_2609_28458_gb300 import workloads as W
from paper_2609_28458_gb300.workloads import Ensemble

pytestmark = pytest.mark.gpu


def oracle_solve(e, method=None, rtol=None, atol=None, **kw):
    return O.solve(e.system, e.y0, e.params, e.t0, e.t1, e.saveat, e.rtol if rtol is None else rtol,
                   e.atol if atol is None else atol, method=method or e.method, **kw)


@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_isochrone_workload_fp64_within_1e9(kernel):
    e = W.isochrone(n=4096, seed=0)
    ref = oracle_solve(e)
    g = gpu_solve(e, kernel=kernel)
    assert np.all(g["status"] == 0) and np.all(ref["status"] == 0)
    err = rel_err(g["y"], ref["y"])
    assert err.max() <= 1e-9, (err.max(), np.argmax(err))
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"])
    assert same.mean() > 0.99


CASES = [
    ("mw", lambda: W.mw(n=256, seed=21, t1=1500.0, rtol=1e-8), "tsit5"),
    ("mw", lambda: W.mw(n=256, seed=22, t1=1500.0, rtol=1e-8), "dopri5"),
    ("mw", lambda: W.mw(n=128, seed=23, t1=1500.0, rtol=1e-8), "vern7"),
    ("precession", lambda: W.precession(n=128, seed=24, paper_interval=True, rtol=1e-9), "vern7"),
    ("precession", lambda: W.precession(n=256, seed=25, method="tsit5", rtol=1e-9), "tsit5"),
    ("quintessence", lambda: W.quintessence(n=256, seed=26, rtol=1e-8), "tsit5"),
    ("quintessence", lambda: W.quintessence(n=256, seed=27, rtol=1e-8, dense=True), "dopri5"),
    ("quintessence", lambda: W.quintessence(n=128, seed=28, rtol=1e-8), "vern7"),
    ("loghalo", lambda: W.loghalo(n=256, seed=29, rtol=1e-8), "tsit5"),
    ("isochrone", lambda: W.isochrone(n=256, seed=30), "vern7"),
]


@pytest.mark.parametrize("system,gen,method", CASES)
@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_fp64_same_algorithm_parity(system, gen, method, kernel):
    e = gen()
    ref = oracle_solve(e, method=method)
    g = gpu_solve(e, method=method, kernel=kernel)
    assert np.array_equal(g["status"], ref["status"])
    ok = (ref["status"] & O.ST_EMPTY_INTERVAL) == 0
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"])
    err = rel_err(g["y"], ref["y"])
    assert same[ok].mean() >= 0.9, same.mean()
    assert err[same & ok].max() <= 1e-10, err[same & ok].max()
    assert err[ok].max() <= 50 * e.rtol, err[ok].max()
    empty = ~ok
    assert np.array_equal(g["y"][empty], ref["y"][empty])


PI_CASES = [
    ("mw", lambda: W.mw(n=256, seed=41, t1=1500.0, rtol=1e-8), "tsit5"),
    ("precession", lambda: W.precession(n=128, seed=42, paper_interval=True, rtol=1e-9), "vern7"),
    ("isochrone", lambda: W.isochrone(n=256, seed=43), "dopri5"),
]


@pytest.mark.parametrize("system,gen,method", PI_CASES)
@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_fp64_pi_controller_parity(system, gen, method, kernel):
    """The PI form of Eq. controller with Gustafsson's gains (beta1, beta2) = (0.7/nu, 0.4/nu):
    err_prev carried across accepted steps and reset to 1 by a rejection, in both kernels.

    Tolerance. The PI controller carries rounding noise of the error estimate (which cancels its
    leading terms: ~eps h|f| / (rtol |y|), 1e-8 relative at rtol 1e-8) from step to step instead of
    resetting it each step, so its step sequence depends on the order of rounding far more than
    Eq. controller's: the oracle's own source compiled with multiply-add contraction against without
    it, on the Milky-Way case here, differs by up to 8.7e-9 relative on members with equal step
    counts (P90 1.2e-10) under the PI gains, and by 1.3e-12 under Eq. controller. The GPU fuses
    multiply-adds and the oracle does not, so the bar is that spread: members with the oracle's step
    counts within 5 rtol and their median within 1e-10; every member within 50 rtol."""
    e = gen()
    nu = 7 if method == "vern7" else 5
    kw = dict(beta1=0.7 / nu, beta2=0.4 / nu)
    ref = oracle_solve(e, method=method, **kw)
    g = gpu_solve(e, method=method, kernel=kernel, **kw)
    assert np.array_equal(g["status"], ref["status"])
    ok = (ref["status"] & O.ST_EMPTY_INTERVAL) == 0
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"])
    err = rel_err(g["y"], ref["y"])
    assert same[ok].mean() >= 0.9, same[ok].mean()
    assert err[same & ok].max() <= 5 * e.rtol, err[same & ok].max()
    assert np.median(err[same & ok]) <= 1e-10, np.median(err[same & ok])
    assert err[ok].max() <= 50 * e.rtol, err[ok].max()
    # the gains reached the kernel (the step sequences differ from Eq. controller's) and the
    # rejection branch, which resets err_prev, was taken
    i_ctrl = oracle_solve(e, method=method)
    assert np.any(i_ctrl["n_accept"][ok] != ref["n_accept"][ok])
    assert ref["n_reject"][ok].sum() > 0


def test_persistent_kernel_matches_plain():
    """Same per-trajectory algorithm in both kernels. FP64: the compiler may fuse multiply-adds
    differently in the two, so results agree to rounding and step counts almost always. FP32 modes:
    the FP32 rounding noise of the error estimate is a sizeable fraction of the tolerance, so the
    two codegens flip borderline accept tests and the step sequences diverge; the results then agree
    to the tolerance level, judged in the orbit error measure (Eq. st-fwderr) against the budget."""
    e = W.mw(n=3000, seed=31, t1=1000.0)
    a = gpu_solve(e, precision="fp64", kernel="plain")
    b = gpu_solve(e, precision="fp64", kernel="persistent")
    assert np.array_equal(a["status"], b["status"])
    same = (a["n_accept"] == b["n_accept"]) & (a["n_reject"] == b["n_reject"])
    assert same.mean() > 0.95, same.mean()
    assert rel_err(a["y"], b["y"])[same].max() <= 1e-10
    rE, vE = M.orbit_scales("mw", e.y0, e.params)
    for prec in ("fp32", "fp32df"):
        a = gpu_solve(e, precision=prec, kernel="plain")
        b = gpu_solve(e, precision=prec, kernel="persistent")
        assert np.array_equal(a["status"], b["status"])
        err = M.orbit_error(a["y"][:, -1], b["y"][:, -1], rE, vE)
        assert M.p99(err) <= 1e-4, (prec, M.p99(err))
        assert abs(a["n_accept"].mean() / b["n_accept"].mean() - 1) < 0.02


def test_repeated_launches_are_bitwise_reproducible():
    for prec in ("fp64", "fp32", "fp32df"):
        for kernel in ("plain", "persistent"):
            e = W.mw(n=2000, seed=38, t1=800.0)
            a = gpu_solve(e, precision=prec, kernel=kernel)
            b = gpu_solve(e, precision=prec, kernel=kernel)
            for k in ("y", "status", "n_accept", "n_reject"):
                assert np.array_equal(a[k], b[k]), (prec, kernel, k)


def _converged(e, method="vern7"):
    return oracle_solve(e, method=method, rtol=1e-12, atol=1e-12 if e.system != "quintessence" else 1e-14)


@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_mw_meets_orbit_budget_at_searched_tolerance(kernel):
    """Over 3 Gyr the workload's quoted rtol 3e-7 gives P99 ~ 1e-3 (outside the 1e-4 budget); the
    quarter-decade search of Appendix A selects 3.16e-8 (FP32 stages) and 5.62e-8 (FP64). Checked
    here one grid step tighter, on another draw."""
    e = W.mw(n=1024, seed=32)
    ref = _converged(e)
    rE, vE = M.orbit_scales("mw", e.y0, e.params)
    for prec, rtol in (("fp32", 1.78e-8), ("fp32df", 1.78e-8), ("fp64", 3.16e-8)):
        g = gpu_solve(e, precision=prec, kernel=kernel, rtol=rtol, atol=rtol)
        assert np.all(g["status"] == 0)
        err = M.orbit_error(g["y"][:, -1], ref["y"][:, -1], rE, vE)
        assert M.accepted(err, 1e-4), (prec, M.p99(err), err.max())


@pytest.mark.parametrize("t0, span", [(-1500.0, 750.0), (1e7, 750.0), (1e9, 1.0), (0.0, 1e-3)])
def test_fp32_stages_time_arithmetic_on_shifted_intervals(t0, span):
    """The precision split keeps the time as a Kahan-compensated FP64 sum and decides the last step
    by an FP32 lower bound of the remaining interval wherever that bound settles it (the FP64 tests
    elsewhere). Intervals that are negative, far from 0, short against their offset or tiny end on
    t1 and give, at five outputs each, the oracle's FP64 same-algorithm solve within the orbit budget
    (Eq. st-fwderr). The Milky-Way field is autonomous, so shifting the interval changes only the
    rounding of the time: each member takes the step sequence of the same solve on [0, span] (the
    last step's length apart) and reaches the same outputs."""
    base = W.mw(n=512, seed=41, t1=span)

    def on(t_start):
        t0v = np.full(base.n, t_start)
        t1v = t0v + span
        sv = t0v[:, None] + span * np.linspace(0.0, 1.0, 5)[None, :]
        sv[:, -1] = t1v
        return Ensemble("mw", base.y0, base.params, t0v, t1v, sv, 1e-8, 1e-8, "tsit5")

    e, e0 = on(t0), on(0.0)
    ref = oracle_solve(e)
    g = gpu_solve(e, precision="fp32", kernel="persistent")
    g0 = gpu_solve(e0, precision="fp32", kernel="persistent")
    assert np.all(g["status"] == 0) and np.all(ref["status"] == 0) and np.all(g0["status"] == 0)
    rE, vE = M.orbit_scales("mw", e.y0, e.params)
    for k in range(e.saveat.shape[1]):
        err = M.orbit_error(g["y"][:, k], ref["y"][:, k], rE, vE)
        assert M.p99(err) <= 1e-4, (k, M.p99(err))
        assert M.p99(M.orbit_error(g["y"][:, k], g0["y"][:, k], rE, vE)) <= 1e-6, k
    assert np.array_equal(g["y"][:, 0], e.y0)
    d = g["n_accept"].astype(np.int64) - g0["n_accept"]
    assert np.abs(d).max() <= 1 and np.mean(d == 0) >= 0.98, (np.abs(d).max(), np.mean(d == 0))


@pytest.mark.parametrize("prec", ["fp32", "fp32df"])
def test_fp32_modes_close_to_fp64_at_same_tolerance(prec):
    """An FP32-stage solve differs from the FP64 solve of the same tolerance by much less than the
    budget: precision adds at most a small fraction to the truncation error."""
    e = W.mw(n=2048, seed=37)
    rE, vE = M.orbit_scales("mw", e.y0, e.params)
    a = gpu_solve(e, precision=prec, kernel="persistent", rtol=3.16e-8, atol=3.16e-8)
    b = gpu_solve(e, precision="fp64", kernel="persistent", rtol=3.16e-8, atol=3.16e-8)
    err = M.orbit_error(a["y"][:, -1], b["y"][:, -1], rE, vE)
    assert M.p99(err) <= 1e-4, M.p99(err)


def test_fp32df_dense_outputs_and_time_pair():
    """FP32-pair time: outputs at 11 times over 100 time units (isochrone) stay within the FP32 stage
    accuracy of the FP64 oracle, and the output at t1 comes from the clipped last step."""
    e = W.isochrone(n=512, seed=39)
    ref = oracle_solve(e, rtol=1e-12, atol=1e-12, method="vern7")
    g = gpu_solve(e, precision="fp32df", kernel="persistent", rtol=1e-8, atol=1e-8)
    assert np.all(g["status"] == 0)
    assert rel_err(g["y"], ref["y"]).max() <= 2e-4
    assert np.array_equal(g["y"][:, 0], e.y0)


def test_quintessence_fp32_stages_meet_distance_budget():
    e = W.quintessence(n=1024, seed=33, rtol=1e-6)
    ref = _converged(e, method="tsit5")
    for method, prec in (("tsit5", "fp32"), ("dopri5", "fp32"), ("tsit5", "fp32df"), ("dopri5", "fp32df")):
        g = gpu_solve(e, method=method, precision=prec)
        assert np.all(g["status"] == 0)
        err = M.distance_error(g["y"], ref["y"], e.params, e.saveat)
        assert M.accepted(err, 1e-4), (method, prec, M.p99(err))


def test_precession_fp64_meets_angle_budget():
    e = W.precession(n=512, seed=34)
    ref = _converged(e)
    g = gpu_solve(e, kernel="persistent")
    err = M.precession_error(g["y"][:, -1], ref["y"][:, -1])
    assert M.accepted(err, 2e-7), M.p99(err)


def test_status_codes_and_edge_cases():
    e = W.isochrone(n=6, seed=17)
    e.y0[1, 2] = np.nan
    e.t1[2] = 0.0
    sv = np.stack([e.saveat] * 6)
    sv[3, 10] = 150.0
    sv[4, 6] = 45.0
    e.saveat = sv
    for kernel in ("plain", "persistent"):
        ref = oracle_solve(e, rtol=1e-8, atol=1e-8)
        g = gpu_solve(e, rtol=1e-8, atol=1e-8, kernel=kernel)
        assert np.array_equal(g["status"], ref["status"])
        assert np.array_equal(np.isnan(g["y"]), np.isnan(ref["y"]))
        assert np.array_equal(g["y"][2], ref["y"][2])
        ref = oracle_solve(e, rtol=1e-8, atol=1e-8, max_steps=20)
        g = gpu_solve(e, rtol=1e-8, atol=1e-8, kernel=kernel, max_steps=20)
        assert np.array_equal(g["status"], ref["status"])
        assert np.array_equal(g["n_accept"] + g["n_reject"], ref["n_accept"] + ref["n_reject"])


def test_outputs_at_t0_and_t1_are_exact_states():
    e = W.isochrone(n=64, seed=35)
    g = gpu_solve(e)
    assert np.array_equal(g["y"][:, 0], e.y0)
    ref = oracle_solve(e)
    assert rel_err(g["y"][:, -1:], ref["y"][:, -1:]).max() <= 1e-9


def test_empty_ensemble_and_no_outputs():
    e = W.mw(n=8, seed=36, t1=100.0)
    e0 = e.subset(np.arange(0))
    g = gpu_solve(e0)
    assert g["y"].shape == (0, 1, 6)
    e.saveat = np.zeros(0)
    g = gpu_solve(e)
    ref = oracle_solve(e)
    assert g["y"].shape == (8, 0, 6)
    assert np.array_equal(g["n_accept"], ref["n_accept"]) or np.all(np.abs(g["n_accept"] - ref["n_accept"]) <= 1)
