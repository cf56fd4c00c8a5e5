"""Seeded synthetic ensembles for the four workloads (inputs only; no integration arithmetic).

Each generator returns NumPy FP64 arrays: y0 [N, d], params [N, p], t0 [N], t1 [N], saveat [K]
(or [N, K]), plus the tolerances and method the workload is run with. The same arrays feed the
GPU library and the CPU oracle; neither side's arithmetic lives here. Seeds follow
``seed = workload index * 1000 + repetition``.

Workloads (shapes and distributions of the paper's ensembles, Sec. 3-5, with the potentials and
sizes of the benchmark configurations):

* ``isochrone``: test particles in Phi = -1/(1+sqrt(1+r^2)) (G = M = b = 1); r ~ U[0.5, 5],
  isotropic position and velocity directions, speed U[0.3, 0.9] x v_circ(r); t in [0, 100],
  11 equally spaced outputs; Tsit5, rtol 1e-10, atol 1e-12.
* ``mw``: Milky-Way-like potential (Miyamoto-Nagai disc + Hernquist bulge + flattened NFW halo),
  units kpc, Myr, 1e10 Msun; R ~ U[4, 20] kpc, phi ~ U[0, 2pi), z ~ U[-2, 2] kpc, velocity
  v_circ(R, 0) phi-hat plus N(0, (20 km/s)^2) per component; q_halo ~ U[0.8, 1.2];
  t in [0, 3000] Myr, endpoint output; Tsit5, rtol = atol = 3e-7.
* ``precession``: binary black holes, M ~ U[10, 100] Msun, q ~ U[0.1, 1], chi_j ~ U[0, 1],
  isotropic spin directions, Lhat = z-hat; integrated in v from the 20 Hz gravitational-wave
  frequency to v = 0.3 (or, paper-faithful, from r = 100 M to 10 M); endpoint output.
* ``quintessence``: lambda ~ U[0, 1.5], Omega_m ~ U[0.28, 0.34], Omega_r = 9e-5, amplitude
  a0 = 1 - Omega_m - Omega_r (supplied); field at rest at z = 50; outputs at 7 redshifts spread
  uniformly in ln(1+z) over [0.3, 2.4] plus today (or 64 nodes over [0, 3]); rtol 1e-4..1e-6,
  atol = 1e-3 rtol.
"""
from dataclasses import dataclass, field

import numpy as np

# units: kpc, Myr, 1e10 Msun. G from GM_sun = 1.3271244e20 m^3/s^2, kpc = 3.0856775814913673e19 m,
# Myr = 3.15576e13 s.
_GM_SUN, _KPC, _MYR = 1.3271244e20, 3.0856775814913673e19, 3.15576e13
G_KPC_MYR = 1e10 * _GM_SUN * _MYR * _MYR / (_KPC ** 3)
KMS_IN_KPC_MYR = 1e3 * _MYR / _KPC
MW_PARAMS = (6.8, 0.5, 54.0, 1.0)  # (M_disc, M_bulge, M_halo in 1e10 Msun, q_halo)
MW_SCALES = dict(a=3.0, b=0.28, c=1.0, rs=15.6)
T_SUN_S = 4.925490947641267e-6  # G Msun / c^3 in seconds


@dataclass
class Ensemble:
    system: str
    y0: np.ndarray
    params: np.ndarray
    t0: np.ndarray
    t1: np.ndarray
    saveat: np.ndarray
    rtol: float
    atol: float
    method: str = "tsit5"
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.y0.shape[0]

    def subset(self, idx):
        idx = np.asarray(idx)
        sv = self.saveat[idx] if self.saveat.ndim == 2 else self.saveat
        return Ensemble(self.system, self.y0[idx].copy(), self.params[idx].copy(), self.t0[idx].copy(),
                        self.t1[idx].copy(), sv.copy(), self.rtol, self.atol, self.method, dict(self.extra))


def _isotropic(rng, n):
    u = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2 * np.pi, n)
    s = np.sqrt(1.0 - u * u)
    return np.stack([s * np.cos(ph), s * np.sin(ph), u], axis=1)


def isochrone(n=4096, seed=0):
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.5, 5.0, n)
    xhat = _isotropic(rng, n)
    s = np.sqrt(1.0 + r * r)
    vcirc = np.sqrt(r * r / ((1.0 + s) ** 2 * s))
    speed = rng.uniform(0.3, 0.9, n) * vcirc
    vhat = _isotropic(rng, n)
    y0 = np.concatenate([xhat * r[:, None], vhat * speed[:, None]], axis=1)
    return Ensemble("isochrone", y0, np.zeros((n, 0)), np.zeros(n), np.full(n, 100.0),
                    np.linspace(0.0, 100.0, 11), 1e-10, 1e-12, "tsit5")


def mw_vcirc(R, params=MW_PARAMS):
    """Circular speed in the plane z = 0 from the radial forces of the three components."""
    G = G_KPC_MYR
    a, b, c, rs = MW_SCALES["a"], MW_SCALES["b"], MW_SCALES["c"], MW_SCALES["rs"]
    md, mb, mh = params[0], params[1], params[2]
    dphi_disc = G * md * R / (R * R + (a + b) ** 2) ** 1.5
    dphi_bulge = G * mb / (R + c) ** 2
    dphi_halo = G * mh * (np.log1p(R / rs) / R ** 2 - 1.0 / (R * (rs + R)))
    return np.sqrt(R * (dphi_disc + dphi_bulge + dphi_halo))


def mw(n=1 << 20, seed=1000, t1=3000.0, rtol=3e-7):
    rng = np.random.default_rng(seed)
    R = rng.uniform(4.0, 20.0, n)
    ph = rng.uniform(0.0, 2 * np.pi, n)
    z = rng.uniform(-2.0, 2.0, n)
    vc = mw_vcirc(R)
    sig = 20.0 * KMS_IN_KPC_MYR
    dv = rng.normal(0.0, sig, (n, 3))
    x = np.stack([R * np.cos(ph), R * np.sin(ph), z], axis=1)
    v = np.stack([-vc * np.sin(ph), vc * np.cos(ph), np.zeros(n)], axis=1) + dv
    q = rng.uniform(0.8, 1.2, n)
    params = np.tile(np.array(MW_PARAMS[:3]), (n, 1))
    params = np.concatenate([params, q[:, None]], axis=1)
    return Ensemble("mw", np.concatenate([x, v], axis=1), params, np.zeros(n), np.full(n, t1),
                    np.array([t1]), rtol, rtol, "tsit5")


def precession(n=1_000_000, seed=2000, method="vern7", rtol=None, paper_interval=False):
    rng = np.random.default_rng(seed)
    M = rng.uniform(10.0, 100.0, n)
    q = rng.uniform(0.1, 1.0, n)
    chi1 = rng.uniform(0.0, 1.0, n)
    chi2 = rng.uniform(0.0, 1.0, n)
    c1 = rng.uniform(-1.0, 1.0, n)
    c2 = rng.uniform(-1.0, 1.0, n)
    dphi = rng.uniform(0.0, 2 * np.pi, n)
    s1, s2 = np.sqrt(1 - c1 * c1), np.sqrt(1 - c2 * c2)
    L = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    S1 = np.stack([s1, np.zeros(n), c1], axis=1)
    S2 = np.stack([s2 * np.cos(dphi), s2 * np.sin(dphi), c2], axis=1)
    y0 = np.concatenate([L, S1, S2], axis=1)
    params = np.stack([q, chi1, chi2], axis=1)
    if paper_interval:
        t0 = np.full(n, 0.1)
        t1v = 10.0 ** -0.5
    else:
        # v = (pi M T_sun f)^(1/3) at gravitational-wave frequency f = 20 Hz
        t0 = (np.pi * M * T_SUN_S * 20.0) ** (1.0 / 3.0)
        t1v = 0.3
    if rtol is None:
        rtol = 3.16e-9 if method == "vern7" else 5.62e-10
    return Ensemble("precession", y0, params, t0, np.full(n, t1v), np.array([t1v]), rtol, rtol, method,
                    dict(M=M))


def quintessence_redshifts(dense=False):
    if dense:
        return np.expm1(np.linspace(0.0, np.log(4.0), 64))
    return np.expm1(np.linspace(np.log(1.3), np.log(3.4), 7))


def quintessence(n=10_000, seed=3000, rtol=1e-6, method="tsit5", dense=False, omega_r=9e-5):
    rng = np.random.default_rng(seed)
    lam = rng.uniform(0.0, 1.5, n)
    om = rng.uniform(0.28, 0.34, n)
    a0 = 1.0 - om - omega_r
    params = np.stack([a0, lam, om, np.full(n, omega_r)], axis=1)
    z = quintessence_redshifts(dense)
    Nz = np.sort(-np.log1p(z))
    saveat = np.unique(np.concatenate([Nz, [0.0]]))
    return Ensemble("quintessence", np.zeros((n, 3)), params, np.full(n, -np.log(51.0)), np.zeros(n), saveat,
                    rtol, 1e-3 * rtol, method, dict(z=z))


def loghalo(n=10_000, seed=4000, rtol=3.16e-7):
    """Flattened logarithmic halo of Sec. 3 with (v_c, R_c, q) = (1, 0.2, 0.7): orbits started in
    and out of the plane, from near-circular to nearly radial, run for about four periods."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.5, 2.0, n)
    xhat = _isotropic(rng, n)
    speed = rng.uniform(0.3, 1.0, n)
    vhat = _isotropic(rng, n)
    y0 = np.concatenate([xhat * r[:, None], vhat * speed[:, None]], axis=1)
    period = 2 * np.pi * r
    params = np.tile(np.array([1.0, 0.2, 0.7]), (n, 1))
    t1 = 3.7 * period
    return Ensemble("loghalo", y0, params, np.zeros(n), t1, t1[:, None].copy(), rtol, rtol, "tsit5")


def by_name(name, **kw):
    return dict(isochrone=isochrone, mw=mw, precession=precession, quintessence=quintessence,
                loghalo=loghalo)[name](**kw)


# ---------------------------------------------------------------------------------------------
# Profile-likelihood data (Sec. 4.3, Appendix C): synthetic stand-ins for the DESI DR2 BAO distances
# and the Pantheon+ supernova magnitudes, which are not available. Shapes only: 7 BAO redshift bins
# (the first with D_V/r_d alone, the others with correlated D_M/r_d and D_H/r_d), 1701 supernovae
# with a dense covariance (statistical diagonal plus smooth systematic modes), 64 solver output nodes
# uniform in ln(1+z) over [0, 3]. The mock data sets are model values at a fiducial cosmology plus
# correlated Gaussian noise drawn here; the model values themselves come from the caller's solver.

C_KMS = 299792.458                  # speed of light, km/s
PROFILE_FIDUCIAL = dict(lam=0.8, om=0.31, H0=68.0, orad=9e-5, omega_b=0.02218, M_abs=-19.25)


@dataclass
class ProfileData:
    z_nodes: np.ndarray       # [64] solver output redshifts (z = 0 first)
    z_bao: np.ndarray         # [7] BAO bin redshifts
    bao_z: np.ndarray         # [13] redshift of each BAO data point
    bao_kind: np.ndarray      # [13] 0 = D_V/r_d, 1 = D_M/r_d, 2 = D_H/r_d
    bao_frac: np.ndarray      # [13] fractional 1-sigma errors
    bao_rho: float            # correlation of D_M/r_d and D_H/r_d in one bin
    z_sn: np.ndarray          # [n_sn] supernova redshifts
    sn_cov: np.ndarray        # [n_sn, n_sn] magnitude covariance (mag^2)
    lam_grid: np.ndarray      # [n_lam] profile grid of the slope lambda
    fiducial: dict


def profile_data(seed=5000, n_sn=1701, n_lam=100):
    rng = np.random.default_rng(seed)
    z_nodes = quintessence_redshifts(dense=True)
    z_bao = quintessence_redshifts()
    bao_z = np.concatenate([[z_bao[0]], np.repeat(z_bao[1:], 2)])
    bao_kind = np.concatenate([[0], np.tile([1, 2], len(z_bao) - 1)]).astype(np.int32)
    bao_frac = np.where(bao_kind == 0, 0.010, np.where(bao_kind == 1, 0.015, 0.025))
    # supernova redshifts: most at low z, a tail to z = 2.26 (Pantheon+-like shape)
    z_sn = np.concatenate([np.exp(rng.uniform(np.log(0.012), np.log(0.1), n_sn * 35 // 100)),
                           rng.uniform(0.1, 0.8, n_sn * 55 // 100)])
    z_sn = np.sort(np.concatenate([z_sn, rng.uniform(0.8, 2.26, n_sn - len(z_sn))]))
    sig = 0.10 + 0.06 * rng.random(n_sn) + 0.02 * z_sn
    modes = np.stack([0.02 * np.cos(np.pi * k * np.log1p(z_sn) / np.log1p(2.26) + rng.uniform(0, 2 * np.pi))
                      for k in range(1, 7)], axis=1)
    sn_cov = np.diag(sig ** 2) + modes @ modes.T
    lam_grid = np.linspace(0.0, 1.5, n_lam)
    return ProfileData(z_nodes, z_bao, bao_z, bao_kind, bao_frac, -0.45, z_sn, sn_cov, lam_grid,
                       dict(PROFILE_FIDUCIAL))


def bao_covariance(data, truth_bao):
    """Covariance of the 13 BAO points: fractional errors of the fiducial values, D_M-D_H correlated."""
    s = data.bao_frac * np.abs(truth_bao)
    C = np.diag(s ** 2)
    for i in range(1, len(s), 2):
        C[i, i + 1] = C[i + 1, i] = data.bao_rho * s[i] * s[i + 1]
    return C


def profile_mocks(truth, cov, n_mocks, seed=5001):
    """n_mocks draws of truth + C^{1/2} eps (C^{1/2} the lower Cholesky factor, eps standard normal)."""
    rng = np.random.default_rng(seed)
    L = np.linalg.cholesky(cov)
    return truth[None, :] + rng.standard_normal((n_mocks, len(truth))) @ L.T


def profile_truth_lcdm(data, om=0.31, H0=68.0, rd=147.0, n_gl=200):
    """Noise-free observables of a flat LambdaCDM universe (closed-form E(z), D_M by Gauss-Legendre
    quadrature), with a fixed sound horizon: the centre of the benchmark's mock data sets. Only the
    data are made this way; the fits use the quintessence model."""
    orad = data.fiducial["orad"]
    E = lambda z: np.sqrt(om * (1 + z) ** 3 + orad * (1 + z) ** 4 + 1.0 - om - orad)
    x, w = np.polynomial.legendre.leggauss(n_gl)

    def DM(z):
        return 0.5 * z * np.sum(w / E(0.5 * z * (x + 1.0)))

    zb = data.bao_z
    dm, dh = np.array([DM(z) for z in zb]), 1.0 / E(zb)
    dv = (zb * dm * dm * dh) ** (1.0 / 3.0)
    X = np.where(data.bao_kind == 0, dv, np.where(data.bao_kind == 1, dm, dh))
    bao = C_KMS / H0 * X / rd
    dms = np.array([DM(z) for z in data.z_sn])
    sn = 5.0 * np.log10((1 + data.z_sn) * dms * C_KMS / H0) + 25.0 + data.fiducial["M_abs"]
    return bao, sn
