"""Per-trajectory error measures and the acceptance test (NumPy, host side).

* Orbits: Eq. st-scales and Eq. st-fwderr (Sec. 3): the error of an orbit is the larger of its
  position error in units of the zero-velocity radius r_E (Phi(r_E, 0) = E, in the plane) and its
  velocity error in units of v_E (v_E^2 / 2 + Phi(0) = E). Gradient error: Eq. st-graderr
  (Appendix A), the relative Frobenius error of the scaled sensitivity matrix.
* Precession: Eq. prec-err (Sec. 5), the largest angle between the final Lhat, S1hat, S2hat of an
  arm and of the reference.
* Dark energy: Sec. 4.2, the largest difference in D_M or D_H over the output redshifts, in c/H0,
  with D_M(z) = I(0) - I(N_z) and D_H(z) = 1/E(N_z) (Sec. 4.1).
* Acceptance, Eq. accept (Sec. 2.4): P99 of the errors at most eps_req and every error finite.

The potentials below are evaluated only to set the error units of an orbit.
"""
import numpy as np

from .workloads import G_KPC_MYR, MW_SCALES


def potential(system, x, params):
    """Phi at positions x [N, 3] (NumPy)."""
    x = np.asarray(x, dtype=np.float64)
    R2 = x[:, 0] ** 2 + x[:, 1] ** 2
    z2 = x[:, 2] ** 2
    if system == "isochrone":
        return -1.0 / (1.0 + np.sqrt(1.0 + R2 + z2))
    if system == "loghalo":
        vc, rc, q = params[:, 0], params[:, 1], params[:, 2]
        return 0.5 * vc * vc * np.log(rc * rc + R2 + z2 / (q * q))
    if system == "mw":
        G = G_KPC_MYR
        a, b, c, rs = MW_SCALES["a"], MW_SCALES["b"], MW_SCALES["c"], MW_SCALES["rs"]
        md, mb, mh, q = params[:, 0], params[:, 1], params[:, 2], params[:, 3]
        disc = -G * md / np.sqrt(R2 + (a + np.sqrt(z2 + b * b)) ** 2)
        bulge = -G * mb / (np.sqrt(R2 + z2) + c)
        rq = np.sqrt(R2 + z2 / (q * q))
        with np.errstate(invalid="ignore", divide="ignore"):
            halo = np.where(rq > 0, -G * mh * np.log1p(rq / rs) / np.where(rq > 0, rq, 1.0), -G * mh / rs)
        return disc + bulge + halo
    raise ValueError(system)


def orbit_scales(system, y0, params):
    """(r_E, v_E) per orbit from its energy (Eq. st-scales)."""
    y0 = np.asarray(y0, dtype=np.float64)
    n = y0.shape[0]
    if params is None or np.size(params) == 0:
        params = np.zeros((n, 4))
    E = 0.5 * np.sum(y0[:, 3:] ** 2, axis=1) + potential(system, y0[:, :3], params)
    phi0 = potential(system, np.zeros((n, 3)), params)
    vE = np.sqrt(np.maximum(2.0 * (E - phi0), 0.0))
    lo = np.zeros(n)
    hi = np.full(n, 1.0)
    for _ in range(200):  # bracket: grow hi until Phi(hi, 0) >= E
        ph = potential(system, np.stack([hi, 0 * hi, 0 * hi], 1), params)
        grow = ph < E
        if not grow.any():
            break
        hi = np.where(grow, hi * 2.0, hi)
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        ph = potential(system, np.stack([mid, 0 * mid, 0 * mid], 1), params)
        below = ph < E
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi), vE


def orbit_error(y, yref, rE, vE):
    """Eq. st-fwderr for y, yref [N, 6] (or [N, K, 6]; the max over outputs is taken)."""
    y = np.asarray(y)
    yref = np.asarray(yref)
    if y.ndim == 3:
        dx = np.linalg.norm(y[..., :3] - yref[..., :3], axis=-1) / rE[:, None]
        dv = np.linalg.norm(y[..., 3:] - yref[..., 3:], axis=-1) / vE[:, None]
        return np.max(np.maximum(dx, dv), axis=1)
    dx = np.linalg.norm(y[:, :3] - yref[:, :3], axis=1) / rE
    dv = np.linalg.norm(y[:, 3:] - yref[:, 3:], axis=1) / vE
    return np.maximum(dx, dv)


def sensitivity_error(S, Sref, rE, vE, D):
    """Eq. st-graderr: ||W (S - Sref) D||_F / ||W Sref D||_F with W = diag(1/r_E x3, 1/v_E x3)."""
    W = np.concatenate([np.repeat(1.0 / rE[:, None], 3, 1), np.repeat(1.0 / vE[:, None], 3, 1)], axis=1)
    A = W[:, :, None] * (S - Sref) * D[:, None, :]
    B = W[:, :, None] * Sref * D[:, None, :]
    return np.sqrt((A ** 2).sum((1, 2))) / np.sqrt((B ** 2).sum((1, 2)))


def _angle(a, b):
    c = np.cross(a, b)
    return np.arctan2(np.linalg.norm(c, axis=-1), np.sum(a * b, axis=-1))


def precession_error(y, yref):
    """Eq. prec-err for final states y, yref [N, 9]."""
    y = np.asarray(y).reshape(-1, 9)
    yref = np.asarray(yref).reshape(-1, 9)
    return np.max(np.stack([_angle(y[:, 3 * j:3 * j + 3], yref[:, 3 * j:3 * j + 3]) for j in range(3)]), axis=0)


def tilts(y):
    """Spin tilts theta_j = atan2(|S_j x L|, S_j . L) of final states [N, 9]."""
    y = np.asarray(y).reshape(-1, 9)
    L = y[:, :3]
    return np.stack([_angle(y[:, 3:6], L), _angle(y[:, 6:9], L)], axis=1)


def quintessence_E(N, y, params):
    """E(N) from the Friedmann equation (Eq. de-model, first line)."""
    a0, lam, om, orad = (params[:, k] for k in range(4))
    phi, u = y[..., 0], y[..., 1]
    if np.ndim(phi) == 2:
        a0, lam, om, orad = (v[:, None] for v in (a0, lam, om, orad))
    num = om * np.exp(-3.0 * N) + orad * np.exp(-4.0 * N) + a0 * np.exp(-lam * phi)
    return np.sqrt(num / (1.0 - u * u / 6.0))


def distances(y, params, saveat):
    """D_M and D_H (units c/H0) at every output except the last (today): y [N, K, 3], saveat [K]."""
    I0 = y[:, -1, 2]
    DM = I0[:, None] - y[:, :-1, 2]
    E = quintessence_E(np.asarray(saveat)[None, :-1], y[:, :-1, :], params)
    return DM, 1.0 / E


def distance_error(y, yref, params, saveat):
    dm, dh = distances(y, params, saveat)
    dmr, dhr = distances(yref, params, saveat)
    return np.maximum(np.abs(dm - dmr).max(1), np.abs(dh - dhr).max(1))


def p99(err):
    return float(np.percentile(err, 99))


def accepted(err, eps_req):
    """Eq. accept: P99 of the errors at most eps_req and every error finite."""
    err = np.asarray(err)
    return bool(np.all(np.isfinite(err)) and p99(err) <= eps_req)
