"""Pins of the oracle's profile-likelihood Gauss-Newton fit (Sec. 4.3, Appendix C, Eq. de-gn):

* r_d from the Aubourg et al. (2015) fitting formula reproduces the Planck 2018 sound horizon at
  Planck's densities (tests/golden/planck2018_sound_horizon.txt, two parameter sets);
* the projection of the whitened supernova residuals equals the analytic minimum over the absolute
  magnitude M of (v - M 1)^T C^{-1} (v - M 1);
* the spline through the 64 nodes gives the BAO distances and supernova magnitudes of a direct
  dense-output solve at the data redshifts;
* the Jacobian columns equal central differences of the whitened residuals along flat models;
* on noiseless data the fit returns the generating (Om, H0) with chi^2 ~ 0, and on a noisy mock it
  ends at a stationary point (decrement < 1e-6) that passes the paper's convergence test.
"""
import os

import numpy as np
import pytest

import oracle as O
from oracle import profile as P
from paper_2609_28458_gb300 import workloads as W


@pytest.fixture(scope="module")
def setup():
    data = W.profile_data(n_sn=400)
    fid = data.fiducial
    bao, sn = P.truth_vectors(data, fid["lam"], fid["om"], fid["H0"])
    C_bao = W.bao_covariance(data, bao)
    return data, bao, sn, np.linalg.cholesky(C_bao), np.linalg.cholesky(data.sn_cov)


def test_sound_horizon_matches_planck():
    # tests/golden/planck2018_sound_horizon.txt: Planck 2018 VI, Table 2 (densities and r_drag);
    # 0.1 Mpc is three times the formula's stated 0.02% accuracy
    path = os.path.join(os.path.dirname(__file__), "golden", "planck2018_sound_horizon.txt")
    rows = np.loadtxt(path, comments="#", ndmin=2)
    assert rows.shape == (2, 5)
    for wb, wc, h, rd, _ in rows:
        om = (wb + wc + P.OMEGA_NU) / h ** 2
        assert abs(P.rd_aubourg(om, 100 * h, wb) - rd) < 0.1


def test_projection_is_marginalisation_over_M():
    rng = np.random.default_rng(3)
    n = 50
    A = rng.normal(size=(n, n))
    C = A @ A.T + n * np.eye(n)
    L = np.linalg.cholesky(C)
    v = rng.normal(size=n) + 3.0
    r, _ = P.whiten(np.zeros(1), np.zeros((1, 2)), v, np.zeros((n, 2)), np.zeros(1), np.zeros(n), np.eye(1), L)
    Ci = np.linalg.inv(C)
    one = np.ones(n)
    M = one @ Ci @ v / (one @ Ci @ one)
    ref = (v - M) @ Ci @ (v - M)
    assert abs(r @ r - ref) <= 1e-10 * ref


def test_spline_matches_direct_dense_output(setup):
    data = setup[0]
    lam, om, H0 = 1.1, 0.33, 67.0
    orad = data.fiducial["orad"]
    nm = P.node_model(lam, om, 1 - om - orad, data.z_nodes, orad, 1e-10, 1e-13)
    bao, _, sn, _ = P.observables(nm, data, om, H0)
    # direct: the flat model saved at the data redshifts themselves
    zs = np.unique(np.concatenate([data.bao_z, data.z_sn]))
    N = np.sort(-np.log1p(zs))
    th = np.array([[nm["a0"], lam, om, orad]])
    y = O.solve("quintessence", np.zeros((1, 3)), th, np.array([P.T0_EFOLDS]), np.zeros(1), np.append(N, 0.0),
                1e-10, 1e-13)["y"][0]
    I0 = y[-1, 2]
    zout = np.expm1(-N)                                  # redshift of each output, same order as y[:-1]
    key = lambda z: int(np.argmin(np.abs(zout - z)))
    rd = P.rd_aubourg(om, H0, data.fiducial["omega_b"])
    for i, (z, k) in enumerate(zip(data.bao_z, data.bao_kind)):
        if k == 1:                                       # D_M/r_d
            ref = P.C_KMS / H0 * (I0 - y[key(z), 2]) / rd
            assert abs(bao[i] / ref - 1) < 1e-8, (z, bao[i], ref)
    DMs = np.array([I0 - y[key(z), 2] for z in data.z_sn])
    ref_sn = 5 * np.log10((1 + data.z_sn) * DMs) + 5 * np.log10(P.C_KMS / H0) + 25
    assert np.max(np.abs(sn - ref_sn)) < 1e-7            # magnitudes


def test_jacobian_matches_finite_differences(setup):
    data, bao_t, sn_t, Lb, Ls = setup
    lam, om, H0 = 0.9, 0.30, 69.0
    orad = data.fiducial["orad"]

    def res(om_, H0_):
        nm = P.node_model(lam, om_, 1 - om_ - orad, data.z_nodes, orad, 1e-11, 1e-14)
        b, Jb, s, Js = P.observables(nm, data, om_, H0_)
        return P.whiten(b, Jb, s, Js, bao_t, sn_t, Lb, Ls)

    r, J = res(om, H0)
    d = 1e-5
    fd_om = (res(om + d, H0)[0] - res(om - d, H0)[0]) / (2 * d)
    fd_h = (res(om, H0 + 1e-3)[0] - res(om, H0 - 1e-3)[0]) / 2e-3
    assert np.max(np.abs(fd_om - J[:, 0])) <= 1e-5 * np.max(np.abs(J[:, 0]))
    assert np.max(np.abs(fd_h - J[:, 1])) <= 1e-6 * np.max(np.abs(J[:, 1]))


def test_noiseless_fit_recovers_truth(setup):
    data, bao_t, sn_t, Lb, Ls = setup
    fid = data.fiducial
    f = P.gn_fit(fid["lam"], bao_t, sn_t, data, Lb, Ls)
    assert f["converged"]
    assert abs(f["om"] - fid["om"]) < 1e-6 and abs(f["H0"] - fid["H0"]) < 1e-4
    assert f["chi2"] < 1e-8


def test_noisy_mock_fit_is_stationary(setup):
    data, bao_t, sn_t, Lb, Ls = setup
    mb = W.profile_mocks(bao_t, W.bao_covariance(data, bao_t), 1, seed=11)[0]
    ms = W.profile_mocks(sn_t, data.sn_cov, 1, seed=12)[0]
    f = P.gn_fit(0.5, mb, ms, data, Lb, Ls)
    assert f["converged"] and f["decrement"] < 1e-6
    chi = [h["chi2"] for h in f["history"]]
    assert chi[-1] <= min(chi) + 1e-6
    n_dof = len(mb) + len(ms) - 1 - 2
    assert 0.5 * n_dof < f["chi2"] < 1.5 * n_dof
