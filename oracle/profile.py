"""Profile-likelihood Gauss-Newton fits on mock data (TEST INFRASTRUCTURE; only the test suite and
the CPU-baseline leg of bench.py use it).

Sec. 4.3 and Appendix C, restated in the order they describe:

* the model: for (lambda, Om) the flat quintessence cosmology (a0 from Eq. de-flat by
  ``oracle.flat``), its state saved at 64 output redshifts, and its derivative along the flat models
  dy/dOm (Eq. de-ift);
* the distances at the data redshifts by a cubic spline in x = ln(1+z) through the 64 nodes. What is
  splined are the smooth distance functions f_M = ln(D_M / z) (its limit -ln E(0) at z = 0) and
  f_H = ln D_H, D in units of c/H0, with not-a-knot end conditions (scipy's CubicSpline);
* the observables: D_V/r_d, D_M/r_d, D_H/r_d (D_V = (z D_M^2 D_H)^(1/3)) with r_d from the fitting
  formula of Aubourg et al. (2015) at a fixed baryon density, and supernova magnitudes
  m = 5 log10(D_L / 10 pc) + M, D_L = (1+z) D_M;
* the residuals whitened by the lower Cholesky factors of the data covariances,
  r = C^{-1/2}(model - data), the supernova part projected orthogonally to C^{-1/2} 1 (equivalent
  to marginalising M with a flat prior), chi^2 = r^T r;
* the damped Gauss-Newton update psi <- psi - (J^T J + mu diag J^T J)^{-1} J^T r for
  psi = (Om, H0) (Eq. de-gn), the step shortened to a fixed trust region; J's H0 column analytic,
  its Om column from dy/dOm; the flatness solve of each iteration starts from the previous a0
  moved by da0/dOm times the Om step;
* a fixed number of iterations, then chi^2 recomputed at the returned parameters and the
  convergence test |Delta chi^2| < 1e-4 over the last step and Gauss-Newton decrement below 1e-6.

Readings (the paper gives no values): mu = 1e-3; trust region |dOm| <= 0.02, |dH0| <= 2 km/s/Mpc,
the step scaled by one factor so that both hold; the decrement is g^T (J^T J)^{-1} g, g = J^T r;
start (Om, H0) = (0.30, 70); omega_b = 0.02218 and omega_nu = 0.00064 in r_d, omega_cb = Om h^2 -
omega_nu. Plain NumPy/SciPy over the oracle's flatness solve; no step is shared with the GPU library.
"""
import numpy as np
from scipy.interpolate import CubicSpline

from . import flat as F

C_KMS = 299792.458
T0_EFOLDS = -np.log(51.0)    # z = 50
RD_A, RD_NU, RD_CB, RD_B = 55.154, 72.3, 0.25351, 0.12807
OMEGA_NU = 0.00064
MU_DAMP = 1e-3
TRUST = (0.02, 2.0)


def rd_aubourg(om, H0, omega_b):
    """Sound horizon at the drag epoch in Mpc (Aubourg et al. 2015, Eq. 16)."""
    h = H0 / 100.0
    wcb = om * h * h - OMEGA_NU
    return RD_A * np.exp(-RD_NU * (OMEGA_NU + 0.0006) ** 2) / (wcb ** RD_CB * omega_b ** RD_B)


def dlnrd(om, H0):
    """(d ln r_d / d Om, d ln r_d / d H0)."""
    h = H0 / 100.0
    wcb = om * h * h - OMEGA_NU
    return -RD_CB * h * h / wcb, -RD_CB * 2.0 * om * h * h / (wcb * H0)


def node_model(lam, om, a0_start, z_nodes, orad, rtol, atol, method="tsit5"):
    """Flat model at the nodes: f_M, f_H [64] and their derivatives along flat models, a0, da0/dOm."""
    N_nodes = -np.log1p(z_nodes[::-1])          # ascending e-folds, today last
    th = np.array([[a0_start, lam, om, orad]])
    r = F.solve_flat(np.zeros((1, 3)), th, np.array([T0_EFOLDS]), np.array([0.0]), N_nodes, rtol, atol,
                     method=method, gtol=1e-13, max_newton=30)
    assert r["converged"][0]
    y, dy = r["y"][0, ::-1], r["dydOm"][0, ::-1]  # back to z order (z = 0 first)
    a0, da0 = r["a0"][0], r["da0dOm"][0]
    N = -np.log1p(z_nodes)
    phi, u, I = y[:, 0], y[:, 1], y[:, 2]
    den = 1.0 - u * u / 6.0
    ev = np.exp(-lam * phi)
    num = om * np.exp(-3 * N) + orad * np.exp(-4 * N) + a0 * ev
    E2 = num / den
    dE2 = (np.exp(-3 * N) / den + ev / den * da0 - lam * a0 * ev / den * dy[:, 0] + num * (u / 3.0) / den ** 2 * dy[:, 1])
    fH, dfH = -0.5 * np.log(E2), -0.5 * dE2 / E2
    fM, dfM = np.empty_like(fH), np.empty_like(fH)
    fM[0], dfM[0] = fH[0], dfH[0]               # D_M / z -> 1 / E(0) at z = 0
    DM = I[0] - I[1:]
    fM[1:] = np.log(DM / z_nodes[1:])
    dfM[1:] = (dy[0, 2] - dy[1:, 2]) / DM
    return dict(fM=fM, fH=fH, dfM=dfM, dfH=dfH, a0=a0, da0dOm=da0)


def observables(nm, data, om, H0):
    """Model BAO and supernova observables (M = 0) with their (Om, H0) derivatives."""
    x_nodes = np.log1p(data.z_nodes)
    fM = CubicSpline(x_nodes, nm["fM"], bc_type="not-a-knot")
    fH = CubicSpline(x_nodes, nm["fH"], bc_type="not-a-knot")
    dfM = CubicSpline(x_nodes, nm["dfM"], bc_type="not-a-knot")
    dfH = CubicSpline(x_nodes, nm["dfH"], bc_type="not-a-knot")
    zb = data.bao_z
    xb = np.log1p(zb)
    lnDM = np.log(zb) + fM(xb)
    lnDH = fH(xb)
    dlnDM, dlnDH = dfM(xb), dfH(xb)
    kind = data.bao_kind
    lnX = np.where(kind == 0, (np.log(zb) + 2 * lnDM + lnDH) / 3.0, np.where(kind == 1, lnDM, lnDH))
    dlnX = np.where(kind == 0, (2 * dlnDM + dlnDH) / 3.0, np.where(kind == 1, dlnDM, dlnDH))
    rd = rd_aubourg(om, H0, data.fiducial["omega_b"])
    drd_om, drd_h = dlnrd(om, H0)
    bao = C_KMS / H0 * np.exp(lnX) / rd
    bao_om = bao * (dlnX - drd_om)
    bao_h = bao * (-1.0 / H0 - drd_h)
    zs = data.z_sn
    xs = np.log1p(zs)
    sn = 5.0 * np.log10((1 + zs) * zs) + 5.0 / np.log(10.0) * fM(xs) + 5.0 * np.log10(C_KMS / H0) + 25.0
    sn_om = 5.0 / np.log(10.0) * dfM(xs)
    sn_h = np.full_like(sn, -5.0 / (np.log(10.0) * H0))
    return bao, np.stack([bao_om, bao_h], 1), sn, np.stack([sn_om, sn_h], 1)


def whiten(bao, Jb, sn, Js, d_bao, d_sn, L_bao, L_sn):
    """r = C^{-1/2}(model - data) and J likewise; the supernova part projected orthogonally to C^{-1/2} 1."""
    from scipy.linalg import solve_triangular
    rb = solve_triangular(L_bao, bao - d_bao, lower=True)
    Jbw = solve_triangular(L_bao, Jb, lower=True)
    rs = solve_triangular(L_sn, sn - d_sn, lower=True)
    Jsw = solve_triangular(L_sn, Js, lower=True)
    u = solve_triangular(L_sn, np.ones(len(sn)), lower=True)
    u = u / np.linalg.norm(u)
    rs = rs - u * (u @ rs)
    Jsw = Jsw - np.outer(u, u @ Jsw)
    return np.concatenate([rb, rs]), np.concatenate([Jbw, Jsw])


def gn_fit(lam, d_bao, d_sn, data, L_bao, L_sn, n_iter=20, start=(0.30, 70.0), rtol=1e-8, atol=1e-11,
           method="tsit5"):
    """One minimisation of chi^2 over (Om, H0) at fixed lambda (Eq. de-gn). Returns dict with the
    parameter and chi^2 history, the final chi^2 recomputed at the returned parameters, the last
    Gauss-Newton decrement and the convergence flag."""
    om, H0 = start
    orad = data.fiducial["orad"]
    a0 = 1.0 - om - orad
    hist = []
    chi2_prev = None
    for it in range(n_iter + 1):
        nm = node_model(lam, om, a0, data.z_nodes, orad, rtol, atol, method)
        bao, Jb, sn, Js = observables(nm, data, om, H0)
        r, J = whiten(bao, Jb, sn, Js, d_bao, d_sn, L_bao, L_sn)
        chi2 = float(r @ r)
        JTJ = J.T @ J
        g = J.T @ r
        dec = float(g @ np.linalg.solve(JTJ, g))
        hist.append(dict(om=om, H0=H0, a0=nm["a0"], chi2=chi2, decrement=dec))
        if it == n_iter:
            break
        step = -np.linalg.solve(JTJ + MU_DAMP * np.diag(np.diag(JTJ)), g)
        s = min(1.0, TRUST[0] / max(abs(step[0]), 1e-300), TRUST[1] / max(abs(step[1]), 1e-300))
        step = s * step
        a0 = nm["a0"] + nm["da0dOm"] * step[0]
        om, H0 = om + step[0], H0 + step[1]
        chi2_prev = chi2
    final = hist[-1]
    conv = abs(final["chi2"] - chi2_prev) < 1e-4 and final["decrement"] < 1e-6
    return dict(om=final["om"], H0=final["H0"], a0=final["a0"], chi2=final["chi2"], decrement=final["decrement"],
                converged=conv, history=hist)


def truth_vectors(data, lam, om, H0, rtol=1e-10, atol=1e-13, method="tsit5"):
    """Model BAO and supernova observables at (lambda, Om, H0) with the fiducial absolute magnitude."""
    orad = data.fiducial["orad"]
    nm = node_model(lam, om, 1.0 - om - orad, data.z_nodes, orad, rtol, atol, method)
    bao, _, sn, _ = observables(nm, data, om, H0)
    return bao, sn + data.fiducial["M_abs"]
