"""Spatial flatness of the quintessence cosmologies (TEST INFRASTRUCTURE; only the test suite and
the CPU-baseline leg of bench.py use it).

Sec. 4.1 (Eq. de-flat): a flat model has E(0) = 1, i.e.

    g(a0; lambda, Om) = (Om + Or + a0 exp(-lambda phi0)) / (1 - u0^2 / 6) - 1 = 0,

with (phi0, u0) the field and its velocity at N = 0, known only after integrating to today. The
amplitude a0 is found by Newton's method: each step is one integration to N = 0 carrying the
sensitivity S_a0 = dy/da0, which gives dg/da0 = (dg/dy) S_a0(0) + dg/da0|explicit.

Eq. de-ift: along the flat models a0 depends on Om, with da0/dOm = -(dg/dOm) / (dg/da0), each
total derivative being (dg/dy) S_theta(0) + dg/dtheta|explicit, and the state moves with
dy/dOm = S_Om + (da0/dOm) S_a0 at every output.

Plain NumPy over the oracle's full sensitivity matrix (``oracle.sens``); no step of this module is
shared with the GPU library.
"""
import numpy as np

from . import sens

# theta = (a0, lambda, Omega_m, Omega_r); state y = (phi, u, I)
IA0, ILAM, IOM, IOR = 0, 1, 2, 3
D = 3


def g_flat(y_today, theta):
    """Eq. de-flat: E(0)^2 - 1 from the state today and theta (arrays over cosmologies)."""
    phi, u = y_today[:, 0], y_today[:, 1]
    a0, lam, om, orad = theta[:, IA0], theta[:, ILAM], theta[:, IOM], theta[:, IOR]
    return (om + orad + a0 * np.exp(-lam * phi)) / (1.0 - u * u / 6.0) - 1.0


def dg_dy(y_today, theta):
    """Partial derivatives of g with respect to (phi0, u0, I0)."""
    phi, u = y_today[:, 0], y_today[:, 1]
    a0, lam, om, orad = theta[:, IA0], theta[:, ILAM], theta[:, IOM], theta[:, IOR]
    den = 1.0 - u * u / 6.0
    num = om + orad + a0 * np.exp(-lam * phi)
    out = np.zeros((len(phi), D))
    out[:, 0] = -lam * a0 * np.exp(-lam * phi) / den
    out[:, 1] = num * (u / 3.0) / (den * den)
    return out


def dg_dtheta(y_today, theta):
    """Explicit partial derivatives of g with respect to (a0, lambda, Om, Or) at fixed state."""
    phi, u = y_today[:, 0], y_today[:, 1]
    a0, lam = theta[:, IA0], theta[:, ILAM]
    den = 1.0 - u * u / 6.0
    out = np.zeros((len(phi), 4))
    out[:, IA0] = np.exp(-lam * phi) / den
    out[:, ILAM] = -phi * a0 * np.exp(-lam * phi) / den
    out[:, IOM] = 1.0 / den
    out[:, IOR] = 1.0 / den
    return out


def solve_flat(y0, params, t0, t1, saveat, rtol, atol, method="tsit5", max_newton=20, gtol=1e-12):
    """Newton's method on a0 (Eq. de-flat), started from params[:, 0], then Eq. de-ift.

    saveat: output e-folds, the last of which must be t1 = 0 (today). A cosmology stops at the
    first iteration whose residual satisfies |g| <= gtol; its outputs are those of that
    integration. Returns dict(a0, y [N,K,3], dydOm [N,K,3], da0dOm [N], g [N], n_newton [N],
    converged [N])."""
    theta = np.array(params, dtype=np.float64, copy=True)
    N = theta.shape[0]
    saveat = np.asarray(saveat, dtype=np.float64)
    K = saveat.shape[-1]
    res = dict(a0=np.full(N, np.nan), y=np.full((N, K, D), np.nan), dydOm=np.full((N, K, D), np.nan),
               da0dOm=np.full(N, np.nan), g=np.full(N, np.nan), n_newton=np.zeros(N, np.int32),
               converged=np.zeros(N, bool))
    todo = np.ones(N, bool)
    for it in range(max_newton):
        idx = np.nonzero(todo)[0]
        if len(idx) == 0:
            break
        sv = saveat[idx] if saveat.ndim == 2 else saveat
        r = sens("quintessence", np.asarray(y0)[idx], theta[idx], np.asarray(t0)[idx], np.asarray(t1)[idx], sv,
                 rtol, atol, method)
        yT = r["y"][:, -1]
        S_a0 = r["S"][..., D + IA0]   # [n, K, 3]
        S_om = r["S"][..., D + IOM]
        th = theta[idx]
        g = g_flat(yT, th)
        gy = dg_dy(yT, th)
        gt = dg_dtheta(yT, th)
        dg_da0 = np.einsum("ni,ni->n", gy, S_a0[:, -1]) + gt[:, IA0]
        dg_dom = np.einsum("ni,ni->n", gy, S_om[:, -1]) + gt[:, IOM]
        da0dom = -dg_dom / dg_da0
        conv = np.abs(g) <= gtol
        last = it == max_newton - 1
        done = conv | last
        sel = idx[done]
        res["a0"][sel] = th[done, IA0]
        res["y"][sel] = r["y"][done]
        res["dydOm"][sel] = S_om[done] + da0dom[done, None, None] * S_a0[done]
        res["da0dOm"][sel] = da0dom[done]
        res["g"][sel] = g[done]
        res["n_newton"][sel] = it + 1
        res["converged"][sel] = conv[done]
        upd = idx[~done]
        theta[upd, IA0] = th[~done, IA0] - g[~done] / dg_da0[~done]
        todo[sel] = False
    return res
