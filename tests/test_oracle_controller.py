"""Pins of the oracle's error norm and step-size controller (Appendix A, Eqs. errnorm and controller,
and the PI form of the controller) against things other than the oracle itself (CPU only).

1. SciPy's RK45 is an independent implementation of the Dormand-Prince 5(4) pair with the norm and
   controller that Appendix A prescribes for an embedded pair of order 5: the scaled RMS norm with
   scale atol + rtol max(|y|, |y+|), accept when the norm is at most 1, next step
   h * clamp(0.9 ||e||^(-1/5), 0.2, ceiling) after accepts and rejects alike. Its ceiling is 10, and
   after a rejection it caps the next accepted step's factor at 1, which Eq. controller does not.
   So the oracle's Dopri5, run with alpha_max = 10 from the same state and first step, must take
   SciPy's accepted steps, with the rejections at the same attempts, up to and including the
   accepted retry after a rejection. Each trajectory is cut into such windows: every window
   restarts both integrators from SciPy's state and SciPy's proposed step, so every accepted step
   and every rejection of whole trajectories of four workloads is compared.
   Tolerance: the embedded error estimate sum_j (b_j - bhat_j) k_j cancels its leading terms, so
   rounding perturbs it by about eps h|f| / (rtol |y|) relative (1e-10 at rtol 1e-6); the step ratio
   takes its 1/5 power and the trajectories drift apart by rounding over hundreds of steps. The
   worst window measured differs by 5e-10; the bound is 1e-8, while any of the plausible misreadings
   (a scale on |y| alone, exponent -1/(nu+1), a missing mean in the RMS, no safety factor) changes
   step sizes by 1e-3 or more.

2. On Dahlquist's test equation y' = lambda y a step of any explicit Runge-Kutta pair multiplies y
   by its stability polynomial R(z), z = h lambda, and the embedded solution by Rhat(z), so the
   error estimate is exactly (R(z) - Rhat(z)) y with R(z) - Rhat(z) = z (b - bhat)^T (I - zA)^(-1) 1.
   The tests evaluate that closed form in exact rational arithmetic from the tableau (itself pinned
   by the order conditions) and drive Eq. controller with it: every accept/reject decision, every
   accepted step and the counts must equal the oracle's, for decay (scale set by |y|) and growth
   (scale set by |y+|), a tiny first step (step ratios at the ceiling alpha_max = 5 of the paper's
   controller), a huge one (ratios at the floor 0.2, repeated rejections), and the PI gains
   (beta1, beta2) = (0.7/nu, 0.4/nu) with err_prev = max(err, 1e-4) after accepts and 1 after
   rejects. Tolerance: the oracle's estimate carries the same cancellation as above, and from a tiny
   first step it is mostly rounding noise (its exact value, of order z^(nu+1) y, lies below
   eps z y): about 1e-10 z / ||e|| relative. The I-controller sits at its ceiling there, but the PI
   controller acts on these estimates and sums their relative errors, times beta1, into h: measured
   up to 6e-7 (order-5 pairs). Bound 1e-5; the misreadings change steps by 1e-2 or more, or change
   an accept/reject decision.

tests/test_oracle_mutations.py plants each misreading in a copy of the oracle and checks that one of
these pins fails.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2609_28458_gb300 import workloads as W

SCIPY_RTOL = 1e-8
LINEAR_RTOL = 1e-5


# ---------------------------------------------------------------------------------------------
def scipy_windows(system, y0, p, t0, t1, rtol, atol):
    """Compare the oracle's Dopri5 with SciPy's RK45 window by window over one trajectory.
    Returns (worst relative step difference, windows, accepted steps, rejections)."""
    RK45 = pytest.importorskip("scipy.integrate").RK45

    def fun(t, y):
        return O.rhs(system, t, y, p)

    t, y = t0, np.array(y0, dtype=np.float64)
    h = O.initial_step(system, "dopri5", t0, t1, y0, p, rtol, atol)
    worst, nwin, nsteps, nrej = 0.0, 0, 0, 0
    while True:
        s = RK45(fun, t, y, t1, rtol=rtol, atol=atol, first_step=min(h, t1 - t))
        hs, att = [], []
        while True:
            t_old, nf = s.t, s.nfev
            s.step()
            hs.append(s.t - t_old)
            att.append((s.nfev - nf) // 6)  # six evaluations of f per attempt (FSAL)
            if s.status != "running" or att[-1] > 1:
                break
        finished = s.status != "running"
        assert s.status in ("running", "finished"), s.message
        if finished:  # the step that reached t1 was clipped to it; the oracle clips differently
            hs, att = hs[:-1], att[:-1]
        if hs:
            hs, att = np.array(hs), np.array(att)
            r = O.solve(system, y[None], None if p is None else p[None], t, t1, np.array([t1]), rtol, atol,
                        method="dopri5", record=True, alpha_max=10.0, h0=min(h, t1 - t), max_steps=int(att.sum()))
            assert r["n_accept"][0] == len(hs) and r["n_reject"][0] == int((att - 1).sum()), \
                (system, t, r["n_accept"][0], len(hs), r["n_reject"][0], att)
            th = r["tape"][0, : r["ntape"][0]]
            worst = max(worst, float(np.max(np.abs(th / hs - 1.0))))
            nwin += 1
            nsteps += len(hs)
            nrej += int((att - 1).sum())
        if finished:
            return worst, nwin, nsteps, nrej
        t, y, h = s.t, s.y.copy(), s.h_abs


SCIPY_CASES = [
    ("isochrone", lambda: W.isochrone(n=4, seed=3), 1e-6, 1e-6),
    ("mw", lambda: W.mw(n=3, seed=4, t1=1500.0), 1e-6, 1e-6),
    ("quintessence", lambda: W.quintessence(n=4, seed=5, rtol=1e-6), 1e-6, 1e-9),
    ("precession", lambda: W.precession(n=2, seed=6, paper_interval=True), 1e-6, 1e-6),
]


def check_scipy_rk45(cases=SCIPY_CASES):
    total_rej = 0
    for system, gen, rtol, atol in cases:
        e = gen()
        for i in range(e.n):
            p = e.params[i] if e.params.shape[1] else None
            t0, t1 = float(np.ravel(e.t0)[i]), float(np.ravel(e.t1)[i])
            worst, nwin, nsteps, nrej = scipy_windows(system, e.y0[i], p, t0, t1, rtol, atol)
            assert worst <= SCIPY_RTOL, (system, i, worst)
            assert nsteps > 20, (system, i, nsteps)
            total_rej += nrej
    assert total_rej >= 1, total_rej  # the reject branch is exercised


@pytest.mark.parametrize("case", SCIPY_CASES, ids=[c[0] for c in SCIPY_CASES])
def test_accepted_steps_match_scipy_rk45(case):
    check_scipy_rk45([case])


# ---------------------------------------------------------------------------------------------
def _stability(tab, z):
    """(R(z), R(z) - Rhat(z)) exactly, for the tableau's double coefficients and the double z."""
    s, A, b, bh = tab["s"], tab["A"], tab["b"], tab["bh"]
    zf = Fraction(z)
    g = []  # g = (I - zA)^(-1) 1 by forward substitution (A strictly lower triangular)
    for j in range(s):
        acc = Fraction(0)
        for l in range(j):
            if A[j, l] != 0.0:
                acc += Fraction(A[j, l]) * g[l]
        g.append(1 + zf * acc)
    R = 1 + zf * sum(Fraction(b[j]) * g[j] for j in range(s))
    E = zf * sum((Fraction(b[j]) - Fraction(bh[j])) * g[j] for j in range(s))
    return R, E


def controller_on_closed_form(method, lam, h0, n_att, rtol, atol, beta1=0.0, beta2=0.0):
    """Eq. controller (PI form) driven by the exact error estimate on y' = lambda y, y(0) = 1, for
    n_att attempts: the paper's (safety, alpha_min, alpha_max) = (0.9, 0.2, 5), exponent -1/nu."""
    tab = O.tableau(method)
    b1 = beta1 if beta1 > 0.0 else 1.0 / tab["order"]
    y, h, err_prev = 1.0, h0, 1.0
    accepted, nrej = [], 0
    for _ in range(n_att):
        R, E = _stability(tab, h * lam)
        y_new = float(R) * y
        sc = atol + rtol * max(abs(y), abs(y_new))
        err = float(abs(E)) * abs(y) / sc
        fac = 0.9 * err ** (-b1) * (err_prev ** beta2 if beta2 != 0.0 else 1.0)
        fac = min(max(fac, 0.2), 5.0)
        if err <= 1.0:
            accepted.append(h)
            y = y_new
            err_prev = max(err, 1e-4)
        else:
            nrej += 1
            err_prev = 1.0
        h = h * fac
    return np.array(accepted), nrej


def _nu(method):
    return O.tableau(method)["order"]


LINEAR_CASES = [
    # (lambda, first step, PI gains as multiples of 1/nu, attempts, methods)
    (-1.0, 1e-4, None, 50, "all"),   # decay from a tiny step: ratios at the ceiling, scale set by |y|
    (0.5, 1e-4, None, 50, "all"),    # growth: scale set by |y+|
    (-3.0, 10.0, None, 50, "all"),   # a huge first step: ratios at the floor, rejections in a row
    (0.5, 3.0, None, 50, "all"),     # growth with rejections
    (-1.0, 0.5, None, 150, "all"),   # y decays below atol: steps limited by stability, rejections
                                     # after accepted steps
    (-2.0, 5.0, (0.7, 0.4), 50, "all"),  # PI gains: rejections at the start
    (0.3, 2.0, (0.7, 0.4), 50, "all"),
    (-1.0, 0.5, (0.7, 0.4), 150, "all"),  # PI in the stability-limited regime: err_prev carried
    (-5.0, 0.1, (0.7, 0.4), 150, "all"),  # across accepts and reset by a rejection between them
    # PI from a tiny step: estimates below 1e-4, so err_prev sits at its floor. Verner 7's estimate
    # (of order z^8) is rounding noise there, which the PI controller would sum into h: Runge-Kutta
    # pairs of order 5 only.
    (-1.0, 1e-4, (0.7, 0.4), 50, ("tsit5", "dopri5")),
    (0.5, 1e-4, (0.7, 0.4), 50, ("tsit5", "dopri5")),
]


def check_linear(methods=("tsit5", "dopri5", "vern7"), cases=LINEAR_CASES, rtol=1e-6, atol=1e-9):
    for method in methods:
        for lam, h0, pi, n_att, only in cases:
            if only != "all" and method not in only:
                continue
            kw = {}
            if pi:
                kw = dict(beta1=pi[0] / _nu(method), beta2=pi[1] / _nu(method))
            hs, nrej = controller_on_closed_form(method, lam, h0, n_att, rtol, atol, **kw)
            T = 1e4 if lam < 0 else 1e3  # never reached within n_att attempts
            r = O.solve("linear", np.array([[1.0]]), np.array([[lam]]), 0.0, T, np.array([T]), rtol, atol,
                        method=method, record=True, h0=h0, max_steps=n_att, **kw)
            assert r["status"][0] == O.ST_MAX_STEPS, r["status"]
            assert r["n_accept"][0] == len(hs) and r["n_reject"][0] == nrej, \
                (method, lam, h0, r["n_accept"][0], len(hs), r["n_reject"][0], nrej)
            th = r["tape"][0, : r["ntape"][0]]
            rel = float(np.max(np.abs(th / hs - 1.0)))
            assert rel <= LINEAR_RTOL, (method, lam, h0, rel)


@pytest.mark.parametrize("method", ["tsit5", "dopri5", "vern7"])
def test_controller_on_linear_test_equation(method):
    check_linear(methods=(method,))


def test_linear_cases_exercise_both_clamps_and_rejections():
    """The closed-form cases do reach the ceiling, the floor and rejections (else they pin less)."""
    for method in ("tsit5", "vern7"):
        hs, nrej = controller_on_closed_form(method, -1.0, 1e-4, 50, 1e-6, 1e-9)
        assert np.any(np.isclose(hs[1:] / hs[:-1], 5.0, rtol=1e-14))
        hs, nrej = controller_on_closed_form(method, -3.0, 10.0, 50, 1e-6, 1e-9)
        assert nrej >= 2
        hs, nrej = controller_on_closed_form(method, -1.0, 0.5, 150, 1e-6, 1e-9, beta1=0.7 / _nu(method),
                                             beta2=0.4 / _nu(method))
        assert nrej >= 1 and len(hs) > 100


def test_oracle_default_controller_is_the_papers():
    """Eq. controller's constants as the oracle's wrapper passes them by default (readings 1-2)."""
    o = O.opts()
    assert (o.safety, o.alpha_min, o.alpha_max, o.beta1, o.beta2) == (0.9, 0.2, 5.0, 0.0, 0.0)
