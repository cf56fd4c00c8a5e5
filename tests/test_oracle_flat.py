"""Pins of the oracle's flatness shooting (Sec. 4.1, Eqs. de-flat and de-ift) and of its full
sensitivity matrix, against what the mathematics fixes independently of the code under test:

* the sensitivity matrix contracted with any cotangent is the oracle's adjoint-free gradient, and
  matches central finite differences of the adaptive solve;
* at lambda = 0 the field never moves, so the flat amplitude is 1 - Om - Or exactly, da0/dOm = -1,
  and dI/dOm along the flat models is a one-dimensional integral (Gauss-Legendre quadrature);
* for lambda > 0 the Newton root equals the root found by bisection on g from plain solves (no
  sensitivities), and da0/dOm and dy/dOm equal central differences of bisection roots and of plain
  solves along the flat models.
"""
import numpy as np
import pytest

import oracle as O
from oracle import flat as F

T0 = -np.log(51.0)          # z = 50
OR = 9e-5
RTOL, ATOL = 1e-12, 1e-15


def _saveat():
    z = np.expm1(np.linspace(np.log(1.3), np.log(3.4), 7))
    return np.unique(np.concatenate([np.sort(-np.log1p(z)), [0.0]]))


def _theta(lam, om, a0=None):
    lam, om = np.atleast_1d(lam).astype(float), np.atleast_1d(om).astype(float)
    a0 = 1.0 - om - OR if a0 is None else np.atleast_1d(a0).astype(float)
    return np.stack([a0, lam, om, np.full(len(lam), OR)], axis=1)


def _plain(theta, sv=None):
    n = theta.shape[0]
    sv = _saveat() if sv is None else sv
    return O.solve("quintessence", np.zeros((n, 3)), theta, np.full(n, T0), np.zeros(n), sv, RTOL, ATOL)["y"]


def _g_plain(lam, om, a0):
    th = _theta([lam], [om], [a0])
    return F.g_flat(_plain(th, np.array([0.0]))[:, -1], th)[0]


def _bisect_a0(lam, om):
    lo, hi = 0.2, 1.5
    glo, ghi = _g_plain(lam, om, lo), _g_plain(lam, om, hi)
    assert glo < 0 < ghi
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _g_plain(lam, om, mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _flat(lam, om, **kw):
    th = _theta(lam, om)
    n = th.shape[0]
    return F.solve_flat(np.zeros((n, 3)), th, np.full(n, T0), np.zeros(n), _saveat(), RTOL, ATOL, **kw)


def test_sens_matrix_contracts_to_gradient_and_matches_finite_differences():
    th = _theta([0.4, 1.2], [0.3, 0.33])
    sv = _saveat()
    n = th.shape[0]
    y0 = np.zeros((n, 3))
    r = O.sens("quintessence", y0, th, np.full(n, T0), np.zeros(n), sv, RTOL, ATOL)
    assert r["S"].shape == (n, len(sv), 3, 7) and np.all(r["status"] == 0)
    w = np.random.default_rng(1).normal(size=(n, len(sv), 3))
    g = O.grad("quintessence", y0, th, np.full(n, T0), np.zeros(n), sv, w, rtol=RTOL, atol=ATOL)
    lhs = np.einsum("nki,nkim->nm", w, r["S"])
    assert np.allclose(lhs[:, 3:], g["dLdparams"], rtol=1e-12, atol=1e-15)
    assert np.allclose(lhs[:, :3], g["dLdy0"], rtol=1e-12, atol=1e-15)
    # d y / d theta_q by central differences of the adaptive solve
    for q, step in ((0, 1e-5), (1, 1e-5), (2, 1e-5)):
        tp, tm = th.copy(), th.copy()
        tp[:, q] += step
        tm[:, q] -= step
        fd = (_plain(tp) - _plain(tm)) / (2 * step)
        S = r["S"][..., 3 + q]
        assert np.max(np.abs(fd - S)) <= 1e-6 * (np.max(np.abs(S)) + 1e-3)
    # MW orbit: derivative with respect to the initial position
    e_y0 = np.array([[8.0, 0.5, 0.3, 0.01, 0.2, 0.02]])
    e_p = np.array([[6.8, 0.5, 54.0, 0.9]])
    r = O.sens("mw", e_y0, e_p, np.zeros(1), np.full(1, 200.0), np.array([200.0]), RTOL, ATOL)
    for m in (0, 4):
        yp, ym = e_y0.copy(), e_y0.copy()
        yp[0, m] += 1e-6
        ym[0, m] -= 1e-6
        f = lambda y: O.solve("mw", y, e_p, np.zeros(1), np.full(1, 200.0), np.array([200.0]), RTOL, ATOL)["y"]
        fd = (f(yp) - f(ym)) / 2e-6
        assert np.max(np.abs(fd[0, -1] - r["S"][0, -1, :, m])) <= 1e-5 * np.max(np.abs(r["S"][0, -1, :, m]))


def test_lambda_zero_flat_amplitude_is_closed_form():
    om = np.array([0.28, 0.31, 0.34])
    res = _flat(np.zeros(3), om)
    assert np.all(res["converged"]) and np.all(res["n_newton"] == 1)
    assert np.allclose(res["a0"], 1.0 - om - OR, rtol=0, atol=1e-15)
    assert np.allclose(res["da0dOm"], -1.0, rtol=0, atol=1e-12)
    assert np.all(res["dydOm"][:, :, :2] == 0.0)    # the field stays at rest along the flat models
    # dI(N_k)/dOm = -1/2 int_{N0}^{N_k} e^{-N} E^{-3} (e^{-3N} - 1) dN, E^2 = Om e^{-3N} + Or e^{-4N} + 1 - Om - Or
    x, wq = np.polynomial.legendre.leggauss(400)
    sv = _saveat()
    for n in range(3):
        for k, Nk in enumerate(sv):
            N = 0.5 * (Nk - T0) * x + 0.5 * (Nk + T0)
            E2 = om[n] * np.exp(-3 * N) + OR * np.exp(-4 * N) + 1 - om[n] - OR
            f = -0.5 * np.exp(-N) * E2 ** -1.5 * (np.exp(-3 * N) - 1.0)
            ref = 0.5 * (Nk - T0) * np.dot(wq, f)
            assert abs(res["dydOm"][n, k, 2] - ref) <= 1e-10 * max(1.0, abs(ref)), (n, k)


@pytest.mark.parametrize("lam,om", [(0.5, 0.30), (1.0, 0.33), (1.5, 0.28)])
def test_newton_root_equals_bisection_root(lam, om):
    res = _flat([lam], [om], gtol=1e-13)
    assert res["converged"][0] and res["n_newton"][0] <= 6       # quadratic convergence from 1 - Om - Or
    assert abs(res["g"][0]) <= 1e-13
    a0b = _bisect_a0(lam, om)
    assert abs(res["a0"][0] - a0b) <= 1e-10
    assert res["a0"][0] > 1.0 - om - OR                         # the moving field needs a larger amplitude


@pytest.mark.parametrize("lam,om", [(0.8, 0.31), (1.4, 0.29)])
def test_ift_derivative_equals_finite_differences_along_flat_models(lam, om):
    res = _flat([lam], [om], gtol=1e-13)
    d = 1e-4
    ap, am = _bisect_a0(lam, om + d), _bisect_a0(lam, om - d)
    fd = (ap - am) / (2 * d)
    assert abs(res["da0dOm"][0] - fd) <= 1e-6 * abs(fd)
    yp = _plain(_theta([lam], [om + d], [ap]))
    ym = _plain(_theta([lam], [om - d], [am]))
    fdy = (yp - ym)[0] / (2 * d)
    assert np.max(np.abs(res["dydOm"][0] - fdy)) <= 1e-5 * np.max(np.abs(fdy))


def test_newton_stops_at_max_iterations_unconverged():
    res = _flat([1.5], [0.3], max_newton=1, gtol=1e-13)
    assert not res["converged"][0] and res["n_newton"][0] == 1
    assert abs(res["g"][0]) > 1e-3           # the frozen-field start leaves E(0) < 1
    assert res["g"][0] < 0
