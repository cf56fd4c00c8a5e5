"""Pins of the CPU oracle against what the paper and the mathematics fix (CPU only).

* isochrone closed forms: radial period T_r = 2 pi / (-2E)^(3/2) and azimuth advance per radial
  period pi (1 + L / sqrt(L^2 + 4)) (Binney & Tremaine, the textbook the paper cites in Sec. 3);
  apocentre radius at T_r / 2 from the radial energy equation;
* measured convergence orders of every tableau and of the dense output on that closed form;
* Poisson's equation for every potential component against the densities that generate them;
* conserved quantities: energy and angular momentum of the orbit systems (Sec. 3); unit lengths,
  effective spin and total angular momentum of the precession equations (Sec. 5), and their
  radiation reaction from the 2PN energy balance (spin-orbit and spin-spin terms included); Lambda-CDM
  distances by Gauss-Legendre quadrature at lambda = 0, and the decrease of rho_phi (Eq. de-rho)
  and w >= -1 (Eq. de-w) for lambda > 0 (Sec. 4, Appendix C);
* the exactness statement of Sec. 2.3 / Eq. stage-sens: forward sensitivities on a fixed step
  sequence equal the derivative of the discrete solution (central differences of the replay);
* the converged-reference check of Appendix A / Appendix D (10x looser tolerance within eps_req/10);
* the starting step against SciPy's implementation of the same published algorithm;
* the failure conventions (status codes, NaN outputs).
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_28458_gb300 import metrics as M
from paper_2609_28458_gb300 import workloads as W


def _iso_elements(y0):
    x, v = y0[:, :3], y0[:, 3:]
    r0 = np.linalg.norm(x, axis=1)
    E = 0.5 * (v ** 2).sum(1) - 1.0 / (1.0 + np.sqrt(1.0 + r0 ** 2))
    Lv = np.cross(x, v)
    L = np.linalg.norm(Lv, axis=1)
    Tr = 2 * np.pi / (-2 * E) ** 1.5
    dpsi = np.pi * (1 + L / np.sqrt(L ** 2 + 4))
    return r0, E, Lv, L, Tr, dpsi


def _azimuth(x0, x1, Lv):
    nh = Lv / np.linalg.norm(Lv, axis=1)[:, None]
    return np.arctan2((nh * np.cross(x0, x1)).sum(1), (x0 * x1).sum(1))


def _wrap(a):
    return np.abs(np.mod(a + np.pi, 2 * np.pi) - np.pi)


# ---------------------------------------------------------------------------------------------
def test_isochrone_radial_period_and_azimuth_converged():
    e = W.isochrone(n=32, seed=7)
    r0, E, Lv, L, Tr, dpsi = _iso_elements(e.y0)
    res = O.solve("isochrone", e.y0, None, 0.0, Tr, Tr[:, None], 1e-13, 1e-13, method="vern7")
    assert np.all(res["status"] == 0)
    y = res["y"][:, 0]
    r1 = np.linalg.norm(y[:, :3], axis=1)
    assert np.max(np.abs(r1 - r0) / r0) < 1e-11
    ang = _azimuth(e.y0[:, :3], y[:, :3], Lv)
    assert np.max(_wrap(ang - dpsi)) < 1e-10


@pytest.mark.parametrize("method", ["tsit5", "dopri5"])
def test_isochrone_same_algorithm_at_workload_tolerance(method):
    e = W.isochrone(n=32, seed=8)
    r0, E, Lv, L, Tr, dpsi = _iso_elements(e.y0)
    res = O.solve("isochrone", e.y0, None, 0.0, Tr, Tr[:, None], 1e-10, 1e-12, method=method)
    r1 = np.linalg.norm(res["y"][:, 0, :3], axis=1)
    assert np.max(np.abs(r1 - r0) / r0) < 3e-9


def _pericentre_orbit():
    # start at pericentre: x = (r_p, 0, 0), v = (0, v_t, 0) with v_t above the circular speed
    rp = 1.0
    s = np.sqrt(1 + rp * rp)
    vc = np.sqrt(rp * rp / ((1 + s) ** 2 * s))
    y0 = np.array([[rp, 0.0, 0.0, 0.0, 1.3 * vc, 0.0]])
    r0, E, Lv, L, Tr, dpsi = _iso_elements(y0)
    # apocentre: other root of E = L^2/(2 r^2) + Phi(r)
    g = lambda r: 0.5 * L[0] ** 2 / r ** 2 - 1.0 / (1.0 + np.sqrt(1.0 + r * r)) - E[0]
    lo, hi = 1.01 * rp, 100.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0:
            lo = mid
        else:
            hi = mid
    return y0, Tr[0], 0.5 * (lo + hi)


def _uniform_tape(T, n):
    return np.full((1, n), T / n), np.array([n], np.int32)


@pytest.mark.parametrize("method,nu,ns", [("tsit5", 5, (40, 80, 160)), ("dopri5", 5, (40, 80, 160)),
                                          ("vern7", 7, (20, 40, 80))])
def test_convergence_order_on_closed_form(method, nu, ns):
    """Fixed steps over one radial period: |r(T_r) - r0| must shrink as h^nu."""
    y0, Tr, _ = _pericentre_orbit()
    errs = []
    for n in ns:
        tape, nt = _uniform_tape(Tr, n)
        y = O.replay("isochrone", y0, None, 0.0, Tr, np.array([Tr]), tape, nt, method=method)
        errs.append(abs(np.linalg.norm(y[0, 0, :3]) - 1.0))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - nu) < 0.6 for s in slopes), (errs, slopes)


@pytest.mark.parametrize("method", ["tsit5", "dopri5"])
def test_dense_output_convergence_on_closed_form(method):
    """Output at T_r/2 (apocentre) falls strictly inside a step for odd step counts; the dense
    solution must converge to the apocentre radius at order >= 4.5 (Eq. dense)."""
    y0, Tr, rapo = _pericentre_orbit()
    errs = []
    for n in (41, 81, 161):
        tape, nt = _uniform_tape(Tr, n)
        y = O.replay("isochrone", y0, None, 0.0, Tr, np.array([0.5 * Tr]), tape, nt, method=method)
        errs.append(abs(np.linalg.norm(y[0, 0, :3]) - rapo))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > 4.5, (errs, slopes)


def test_vern7_shortened_step_output_converges():
    y0, Tr, rapo = _pericentre_orbit()
    res = O.solve("isochrone", y0, None, 0.0, Tr, np.array([0.5 * Tr, Tr]), 1e-12, 1e-12, method="vern7")
    assert abs(np.linalg.norm(res["y"][0, 0, :3]) - rapo) < 1e-10


@pytest.mark.parametrize("method,nu", [("tsit5", 5), ("vern7", 7)])
def test_step_count_scales_with_tolerance(method, nu):
    """With error-per-step control by an embedded pair of orders (nu, nu-1) the step length scales
    as tol^(1/nu): the accepted-step count over four decades of rtol must grow as 10^(4/nu)."""
    e = W.isochrone(n=16, seed=9)
    counts = []
    for rtol in (1e-6, 1e-10):
        res = O.solve("isochrone", e.y0, None, 0.0, 100.0, np.array([100.0]), rtol, rtol, method=method)
        counts.append(res["n_accept"].mean())
    slope = np.log10(counts[1] / counts[0]) / 4.0
    assert abs(slope - 1.0 / nu) < 0.04, (counts, slope)


# ---------------------------------------------------------------------------------------------
def _energy(system, y, params):
    return 0.5 * (y[..., 3:] ** 2).sum(-1) + M.potential(system, y[:, :3], params)


@pytest.mark.parametrize("system,gen", [("isochrone", lambda: W.isochrone(n=16, seed=3)),
                                        ("mw", lambda: W.mw(n=16, seed=3, t1=1000.0)),
                                        ("loghalo", lambda: W.loghalo(n=16, seed=3))])
def test_orbit_invariants(system, gen):
    e = gen()
    res = O.solve(system, e.y0, e.params, e.t0, e.t1, e.saveat, 1e-12, 1e-12)
    assert np.all(res["status"] == 0)
    y1 = res["y"][:, -1]
    E0 = _energy(system, e.y0, e.params)
    E1 = _energy(system, y1, e.params)
    assert np.max(np.abs(E1 - E0) / np.abs(E0)) < 1e-9
    Lz0 = e.y0[:, 0] * e.y0[:, 4] - e.y0[:, 1] * e.y0[:, 3]
    Lz1 = y1[:, 0] * y1[:, 4] - y1[:, 1] * y1[:, 3]
    Lscale = np.linalg.norm(np.cross(e.y0[:, :3], e.y0[:, 3:]), axis=1)
    assert np.max(np.abs(Lz1 - Lz0) / Lscale) < 1e-9
    # energy drift must be of the size the tolerance implies, not zero: the solve did integrate
    assert np.max(np.linalg.norm(y1[:, :3] - e.y0[:, :3], axis=1)) > 1e-3
    if system == "isochrone":  # spherical: the full angular momentum vector
        L1 = np.cross(y1[:, :3], y1[:, 3:])
        L0 = np.cross(e.y0[:, :3], e.y0[:, 3:])
        assert np.max(np.linalg.norm(L1 - L0, axis=1) / Lscale) < 1e-9


def test_mw_spherical_halo_conserves_full_angular_momentum_without_disc():
    e = W.mw(n=8, seed=4, t1=500.0)
    p = e.params.copy()
    p[:, 0] = 0.0  # no disc
    p[:, 3] = 1.0  # spherical halo
    res = O.solve("mw", e.y0, p, e.t0, e.t1, e.saveat, 1e-12, 1e-12)
    y1 = res["y"][:, -1]
    L0 = np.cross(e.y0[:, :3], e.y0[:, 3:])
    L1 = np.cross(y1[:, :3], y1[:, 3:])
    assert np.max(np.linalg.norm(L1 - L0, axis=1) / np.linalg.norm(L0, axis=1)) < 1e-9


def test_orbit_rhs_is_minus_gradient_of_potential():
    """The acceleration equals minus the central-difference gradient of Phi (Eq. loghalo)."""
    rng = np.random.default_rng(0)
    for system, p in (("isochrone", np.zeros(4)), ("mw", np.array([6.8, 0.5, 54.0, 0.9])),
                      ("loghalo", np.array([1.0, 0.2, 0.7]))):
        for _ in range(5):
            x = rng.uniform(-5, 5, 3)
            f = O.rhs(system, 0.0, np.concatenate([x, [0.1, 0.2, 0.3]]), p)
            assert np.allclose(f[:3], [0.1, 0.2, 0.3], rtol=0, atol=0)
            g = np.zeros(3)
            for i in range(3):
                dx = np.zeros(3)
                dx[i] = 1e-5
                g[i] = (O.potential(system, x + dx, p) - O.potential(system, x - dx, p)) / 2e-5
            assert np.allclose(f[3:], -g, rtol=1e-7, atol=1e-12)


# ---------------------------------------------------------------------------------------------
def _prec_quantities(y, p):
    q, chi1, chi2 = p[..., 0], p[..., 1], p[..., 2]
    m1, m2 = 1 / (1 + q), q / (1 + q)
    S1, S2 = chi1 * m1 ** 2, chi2 * m2 ** 2
    L, s1, s2 = y[..., 0:3], y[..., 3:6], y[..., 6:9]
    xi = ((1 + q) * S1)[..., None] * s1 + ((1 + 1 / q) * S2)[..., None] * s2
    return L, s1, s2, (xi * L).sum(-1), S1, S2, m1 * m2


def _laplacian(system, x, p, h=1e-3):
    c = O.potential(system, x, p)
    acc = 0.0
    for i in range(3):
        dx = np.zeros(3)
        dx[i] = h
        acc += O.potential(system, x + dx, p) - 2 * c + O.potential(system, x - dx, p)
    return acc / h ** 2


def test_potentials_satisfy_poisson_with_textbook_densities():
    """Poisson's equation, Laplacian(Phi) = 4 pi G rho, for each component of the Milky-Way potential
    (Sec. 3) and for the logarithmic halo (Eq. loghalo), with the densities that generate them
    written from Binney & Tremaine (2008): Miyamoto-Nagai rho = b^2 M [a R^2 + (a + 3 zeta)(a +
    zeta)^2] / (4 pi [R^2 + (a + zeta)^2]^(5/2) zeta^3), zeta^2 = z^2 + b^2; Hernquist rho = M c /
    (2 pi r (r + c)^3); NFW rho = M_h / (4 pi r (r_s + r)^2); logarithmic halo 4 pi G rho = (v_c^2 /
    q^2) [(2 q^2 + 1) R_c^2 + R^2 + (2 - 1/q^2) z^2] / (R_c^2 + R^2 + z^2/q^2)^2. G in kpc^3 /
    (1e10 Msun Myr^2) from the IAU solar mass parameter; Laplacian by central differences."""
    G = 1e10 * 1.3271244e20 * 3.15576e13 ** 2 / 3.0856775814913673e19 ** 3
    a, b, c, rs = 3.0, 0.28, 1.0, 15.6
    rng = np.random.default_rng(8)
    for _ in range(20):
        R, phi, z = rng.uniform(1.0, 20.0), rng.uniform(0, 2 * np.pi), rng.uniform(-3.0, 3.0)
        x = np.array([R * np.cos(phi), R * np.sin(phi), z])
        r = np.linalg.norm(x)
        zeta = np.sqrt(z * z + b * b)
        M = 6.8
        rho_d = b * b * M * (a * R * R + (a + 3 * zeta) * (a + zeta) ** 2) / (
            4 * np.pi * (R * R + (a + zeta) ** 2) ** 2.5 * zeta ** 3)
        rho_b = 0.5 * c / (2 * np.pi * r * (r + c) ** 3)
        rho_h = 54.0 / (4 * np.pi * r * (rs + r) ** 2)
        for pv, rho in (([M, 0, 0, 1.0], rho_d), ([0, 0.5, 0, 1.0], rho_b), ([0, 0, 54.0, 1.0], rho_h)):
            lap = _laplacian("mw", x, np.array(pv, dtype=float))
            assert abs(lap / (4 * np.pi * G * rho) - 1) < 1e-5, (pv, lap, 4 * np.pi * G * rho)
        vc, Rc, q = 1.0, 0.2, rng.uniform(0.6, 1.0)
        Q = Rc * Rc + R * R + z * z / q ** 2
        lap_log = vc * vc / q ** 2 * ((2 * q * q + 1) * Rc * Rc + R * R + (2 - 1 / q ** 2) * z * z) / Q ** 2
        lap = _laplacian("loghalo", x, np.array([vc, Rc, q]))
        assert abs(lap / lap_log - 1) < 1e-5, (lap, lap_log)


def test_quintessence_field_equation_preserves_the_friedmann_constraint():
    """Along the flow the constraint E^2 (1 - u^2/6) = Om e^-3N + Or e^-4N + a0 e^-lam phi (Eq. de-model)
    must stay consistent with dlnE/dN = -(3 Om e^-3N + 4 Or e^-4N)/(2 E^2) - u^2/2: the total
    N-derivative of E^2 through phi' = u and the oracle's u' (the scalar-field equation of Eq.
    de-rhs) equals 2 E^2 dlnE/dN (the Bianchi identity). A wrong factor in u' breaks it."""
    rng = np.random.default_rng(12)
    for _ in range(50):
        N = rng.uniform(-3.9, 0.0)
        phi, u = rng.uniform(0, 0.6), rng.uniform(-0.8, 0.8)
        a0, lam, om, orad = rng.uniform(0.6, 0.75), rng.uniform(0, 1.5), rng.uniform(0.28, 0.34), 9e-5
        f = O.rhs("quintessence", N, np.array([phi, u, 0.0]), np.array([a0, lam, om, orad]))
        A, B, V = om * np.exp(-3 * N), orad * np.exp(-4 * N), a0 * np.exp(-lam * phi)
        D = 1 - u * u / 6
        E2 = (A + B + V) / D
        dE2 = (-3 * A - 4 * B) / D + f[0] * (-lam * V / D) + f[1] * E2 * (u / 3) / D
        dlnE = -(3 * A + 4 * B) / (2 * E2) - u * u / 2
        assert abs(f[0] - u) < 1e-15
        assert abs(dE2 - 2 * E2 * dlnE) < 1e-12 * (abs(2 * E2 * dlnE) + E2), (dE2, 2 * E2 * dlnE)
        assert abs(f[2] - np.exp(-N) / np.sqrt(E2)) < 1e-14 * abs(f[2])


def test_precession_rhs_identities():
    """At random states: |Lhat|, |S_jhat| fixed (Eq. prec-spins, prec-L), effective spin fixed, and
    the total angular momentum J = (eta/v) Lhat + S1 + S2 changes only through L: dJ/dv = -eta/v^2 Lhat
    (Sec. 5: Eq. prec-L keeps L + S1 + S2 fixed on the precession time-scale)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        v = rng.uniform(0.05, 0.4)
        p = np.array([rng.uniform(0.1, 1.0), rng.uniform(0, 1), rng.uniform(0, 1)])
        vecs = [u / np.linalg.norm(u) for u in rng.normal(size=(3, 3))]
        y = np.concatenate(vecs)
        f = O.rhs("precession", v, y, p)
        L, s1, s2, xi, S1, S2, eta = _prec_quantities(y, p)
        fL, f1, f2 = f[0:3], f[3:6], f[6:9]
        scale = np.abs(f).max()
        assert abs(L @ fL) < 1e-13 * scale and abs(s1 @ f1) < 1e-13 * scale and abs(s2 @ f2) < 1e-13 * scale
        q = p[0]
        dxi = (1 + q) * S1 * (f1 @ L + s1 @ fL) + (1 + 1 / q) * S2 * (f2 @ L + s2 @ fL)
        assert abs(dxi) < 1e-13 * scale
        dJ = (eta / v) * fL + S1 * f1 + S2 * f2  # dJ/dv + eta/v^2 Lhat
        assert np.max(np.abs(dJ)) < 1e-13 * scale * max(S1 + S2 + eta / v, 1.0)


def _series_div(num, den, order):
    """Coefficients c_0..c_order of num(x) / den(x) for power series with den[0] = 1."""
    c = []
    for n in range(order + 1):
        c.append((num[n] if n < len(num) else 0.0) - sum(den[k] * c[n - k] for k in range(1, min(n, len(den) - 1) + 1)))
    return c


def test_precession_radiation_reaction_matches_energy_balance():
    """Pin of the radiation-reaction coefficients b_2, b_3, b_4 (Sec. 5, Eq. prec-rr), derived here
    independently as dv/dt = -F(v) / (dE/dv) by series division of the 2PN binding energy and
    gravitational-wave flux, with l_j = Lhat.S_jhat, s_12 = S_1hat.S_2hat, m_1 = 1/(1+q), m_2 = q m_1:
      E = -(eta v^2/2) [1 - (3/4 + eta/12) v^2 + sum_j (8/3 m_j^2 + 2 eta) chi_j l_j v^3
          - (27/8 - 19/8 eta + eta^2/24) v^4 + eta chi_1 chi_2 (s_12 - 3 l_1 l_2) v^4],
      F = 32/5 eta^2 v^10 [1 - (1247/336 + 35/12 eta) v^2 + (4 pi - sum_j (11/4 m_j^2 + 5/4 eta)
          chi_j l_j) v^3 + (-44711/9072 + 9271/504 eta + 65/18 eta^2) v^4
          + eta/48 chi_1 chi_2 (-103 s_12 + 289 l_1 l_2) v^4]
    (point masses: Blanchet, Living Rev. Relativ. 17, 2 (2014); spin-orbit and spin-spin terms:
    Kidder, Phys. Rev. D 52, 821 (1995)). The oracle's dv/dt is read off the precession of S1hat:
    dS1hat/dt = Omega_1 x S1hat with Omega_1 = v^6/2 [(4 + 3q)(eta/v) Lhat + S_2 S2hat
    - 3 (S_2 l_2 + q S_1 l_1) Lhat], S_j = chi_j m_j^2 (Eq. prec-omega), so dv/dt = |Omega_1 x S1hat| /
    |dS1hat/dv|. A wrong
    coefficient in any b_k, or a dropped spin term, shows up far above 1e-12."""
    rng = np.random.default_rng(4)
    for _ in range(60):
        q = rng.uniform(0.1, 1.0)
        chi1, chi2 = (0.0, 0.0) if _ < 10 else tuple(rng.uniform(0, 1, 2))
        v = rng.uniform(0.05, 0.35)
        m1 = 1 / (1 + q)
        m2 = q * m1
        eta = m1 * m2
        Lh, s1, s2 = [u / np.linalg.norm(u) for u in rng.normal(size=(3, 3))]
        l1, l2, s12 = Lh @ s1, Lh @ s2, s1 @ s2
        so_e = (8 / 3 * m1 ** 2 + 2 * eta) * chi1 * l1 + (8 / 3 * m2 ** 2 + 2 * eta) * chi2 * l2
        so_f = (11 / 4 * m1 ** 2 + 5 / 4 * eta) * chi1 * l1 + (11 / 4 * m2 ** 2 + 5 / 4 * eta) * chi2 * l2
        e2 = -(0.75 + eta / 12)
        e4 = -(27 / 8 - 19 / 8 * eta + eta ** 2 / 24) + eta * chi1 * chi2 * (s12 - 3 * l1 * l2)
        dE = [1.0, 0.0, 2 * e2, 2.5 * so_e, 3 * e4]          # (dE/dv) / (-eta v)
        flux = [1.0, 0.0, -(1247 / 336 + 35 / 12 * eta), 4 * np.pi - so_f,
                -44711 / 9072 + 9271 / 504 * eta + 65 / 18 * eta ** 2 + eta / 48 * chi1 * chi2 * (-103 * s12 + 289 * l1 * l2)]
        c = _series_div(flux, dE, 4)
        dvdt_2pn = 32 / 5 * eta * v ** 9 * sum(c[k] * v ** k for k in range(5))
        f = O.rhs("precession", v, np.concatenate([Lh, s1, s2]), np.array([q, chi1, chi2]))
        S1, S2 = chi1 * m1 ** 2, chi2 * m2 ** 2
        omega1 = v ** 6 / 2 * ((4 + 3 * q) * (eta / v) * Lh + S2 * s2 - 3 * (S2 * l2 + q * S1 * l1) * Lh)
        dvdt_oracle = np.linalg.norm(np.cross(omega1, s1)) / np.linalg.norm(f[3:6])
        assert abs(dvdt_oracle / dvdt_2pn - 1) < 1e-12, (q, chi1, chi2, v, dvdt_oracle, dvdt_2pn)


@pytest.mark.parametrize("method,order", [("tsit5", 5), ("dopri5", 5), ("vern7", 7)])
def test_starting_step_matches_library_routine(method, order):
    """The oracle's starting step (Hairer, Norsett & Wanner I, Sec. II.4; p = the method's order, our
    reading) equals SciPy's implementation of the same published algorithm, called with the oracle's
    right-hand side, on members of every workload."""
    common = pytest.importorskip("scipy.integrate._ivp.common")
    gens = [("isochrone", W.isochrone(n=6, seed=71)), ("mw", W.mw(n=6, seed=72)),
            ("precession", W.precession(n=6, seed=73, paper_interval=True)),
            ("quintessence", W.quintessence(n=6, seed=74, rtol=1e-6)), ("loghalo", W.loghalo(n=6, seed=75))]
    for system, e in gens:
        for i in range(e.n):
            p = e.params[i] if e.params.shape[1] else None
            t0, t1 = float(np.ravel(e.t0)[i]), float(np.ravel(e.t1)[i])
            rtol, atol = 1e-7, 1e-9

            def fun(t, y):
                return O.rhs(system, t, y, p)

            f0 = fun(t0, e.y0[i])
            try:
                ref = common.select_initial_step(fun, t0, e.y0[i], t1, np.inf, f0, 1.0, order, rtol, atol)
            except TypeError:  # older SciPy signature without t_bound and max_step
                ref = min(common.select_initial_step(fun, t0, e.y0[i], f0, 1.0, order, rtol, atol), t1 - t0)
            h = O.initial_step(system, method, t0, t1, e.y0[i], p, rtol, atol)
            assert abs(h - ref) <= 1e-12 * ref, (system, i, h, ref)


def test_precession_solve_invariants():
    e = W.precession(n=16, seed=5, paper_interval=True)
    res = O.solve("precession", e.y0, e.params, e.t0, e.t1, e.saveat, 1e-11, 1e-11, method="vern7")
    assert np.all(res["status"] == 0)
    y1 = res["y"][:, -1]
    for j in range(3):
        assert np.max(np.abs(np.linalg.norm(y1[:, 3 * j:3 * j + 3], axis=1) - 1.0)) < 1e-8
    xi0 = _prec_quantities(e.y0, e.params)[3]
    xi1 = _prec_quantities(y1, e.params)[3]
    assert np.max(np.abs(xi1 - xi0)) < 1e-8
    # and the spins did precess
    assert np.max(np.linalg.norm(y1[:, 3:6] - e.y0[:, 3:6], axis=1)) > 1e-2


def test_precession_empty_interval_above_87_msun():
    e = W.precession(n=64, seed=6)
    res = O.solve("precession", e.y0, e.params, e.t0, e.t1, e.saveat, 1e-9, 1e-9, method="vern7")
    empty = e.extra["M"] > 0.3 ** 3 / (np.pi * W.T_SUN_S * 20.0)
    assert np.array_equal(res["status"] == O.ST_EMPTY_INTERVAL, empty)
    assert np.array_equal(res["y"][empty, 0], e.y0[empty])
    assert np.all(res["n_accept"][empty] == 0)


# ---------------------------------------------------------------------------------------------
def _gauss_legendre_DM(z, om, orad, a0, n=200):
    x, w = np.polynomial.legendre.leggauss(n)
    zz = 0.5 * z * (x + 1)
    E = np.sqrt(om * (1 + zz) ** 3 + orad * (1 + zz) ** 4 + a0)
    return 0.5 * z * np.sum(w / E)


def test_quintessence_lambda_zero_is_lcdm():
    e = W.quintessence(n=8, seed=1)
    p = e.params.copy()
    p[:, 1] = 0.0
    res = O.solve("quintessence", e.y0, p, e.t0, e.t1, e.saveat, 1e-11, 1e-13)
    y = res["y"]
    assert np.all(y[:, :, 0] == 0.0) and np.all(y[:, :, 1] == 0.0)  # field never moves
    DM, DH = M.distances(y, p, e.saveat)
    z = np.expm1(-e.saveat[:-1])
    for n in range(8):
        a0, lam, om, orad = p[n]
        ref = np.array([_gauss_legendre_DM(zz, om, orad, a0) for zz in z])
        assert np.max(np.abs(DM[n] - ref)) < 1e-9
        Eref = np.sqrt(om * (1 + z) ** 3 + orad * (1 + z) ** 4 + a0)
        assert np.max(np.abs(DH[n] - 1 / Eref)) < 1e-13


def test_quintessence_rho_phi_decreases_and_w_above_minus_one():
    e = W.quintessence(n=16, seed=2, dense=True)
    p = e.params.copy()
    p[:, 1] = np.linspace(0.2, 1.5, 16)
    res = O.solve("quintessence", e.y0, p, e.t0, e.t1, e.saveat, 1e-10, 1e-13)
    y = res["y"]
    E = M.quintessence_E(e.saveat[None, :], y, p)
    kin = E ** 2 * y[:, :, 1] ** 2 / 6
    pot = p[:, 0:1] * np.exp(-p[:, 1:2] * y[:, :, 0])
    rho = kin + pot
    assert np.all(np.diff(rho, axis=1) <= 1e-14)
    w = (kin - pot) / (kin + pot)
    assert np.all(w >= -1.0) and np.all(w[:, -1] > -1.0)
    assert np.all(y[:, -1, 1] > 0)  # the field has started to roll


# ---------------------------------------------------------------------------------------------
def _fd_loss(system, e, w, tape, nt, method, dy0=None, dp=None):
    y0 = e.y0 + (dy0 if dy0 is not None else 0)
    pp = e.params + (dp if dp is not None else 0)
    y = O.replay(system, y0, pp, e.t0, e.t1, e.saveat, tape, nt, method=method)
    return np.sum(w * y, axis=(1, 2))


@pytest.mark.parametrize("system,gen,method", [
    ("mw", lambda: W.mw(n=4, seed=11, t1=300.0), "tsit5"),
    ("precession", lambda: W.precession(n=4, seed=12, paper_interval=True), "vern7"),
    ("quintessence", lambda: W.quintessence(n=4, seed=13), "dopri5"),
    ("loghalo", lambda: W.loghalo(n=4, seed=14), "tsit5"),
])
def test_sensitivities_are_exact_derivative_of_discrete_solution(system, gen, method):
    """Sec. 2.3 / Eq. stage-sens: on a fixed step sequence the forward sensitivities equal the
    derivative of the numerical solution; checked against central differences of the replay."""
    e = gen()
    rec = O.solve(system, e.y0, e.params, e.t0, e.t1, e.saveat, 1e-7, 1e-7, method=method, record=True)
    rng = np.random.default_rng(0)
    w = rng.normal(size=rec["y"].shape)
    g = O.grad(system, e.y0, e.params, e.t0, e.t1, e.saveat, w, method=method, tape=rec["tape"],
               ntape=rec["ntape"])
    # the replay reproduces the adaptive solution bit for bit
    yr = O.replay(system, e.y0, e.params, e.t0, e.t1, e.saveat, rec["tape"], rec["ntape"], method=method)
    assert np.array_equal(yr, rec["y"])
    assert np.array_equal(g["y"], rec["y"])
    d, np_ = O.dims(system)
    for i in range(d):
        eps = 1e-6 * max(1.0, np.abs(e.y0[:, i]).max())
        dy = np.zeros_like(e.y0)
        dy[:, i] = eps
        fd = (_fd_loss(system, e, w, rec["tape"], rec["ntape"], method, dy0=dy) -
              _fd_loss(system, e, w, rec["tape"], rec["ntape"], method, dy0=-dy)) / (2 * eps)
        assert np.allclose(g["dLdy0"][:, i], fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max() + 1e-12), (i, g["dLdy0"][:, i], fd)
    for k in range(np_):
        eps = 1e-6 * max(1.0, np.abs(e.params[:, k]).max())
        dp = np.zeros_like(e.params)
        dp[:, k] = eps
        fd = (_fd_loss(system, e, w, rec["tape"], rec["ntape"], method, dp=dp) -
              _fd_loss(system, e, w, rec["tape"], rec["ntape"], method, dp=-dp)) / (2 * eps)
        assert np.allclose(g["dLdparams"][:, k], fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max() + 1e-12), (k, g["dLdparams"][:, k], fd)


def test_sensitivities_agree_with_differences_of_adaptive_solve():
    """The derivative of the discrete solution approximates that of the exact flow to about the
    tolerance level: central differences of the full adaptive solve at tight tolerance."""
    e = W.mw(n=3, seed=15, t1=300.0)
    w = np.random.default_rng(1).normal(size=(3, 1, 6))
    g = O.grad("mw", e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=1e-11, atol=1e-11)
    for k in range(4):
        eps = 1e-4 * abs(e.params[0, k])
        dp = np.zeros_like(e.params)
        dp[:, k] = eps
        lp = np.sum(w * O.solve("mw", e.y0, e.params + dp, e.t0, e.t1, e.saveat, 1e-12, 1e-12)["y"], axis=(1, 2))
        lm = np.sum(w * O.solve("mw", e.y0, e.params - dp, e.t0, e.t1, e.saveat, 1e-12, 1e-12)["y"], axis=(1, 2))
        fd = (lp - lm) / (2 * eps)
        assert np.allclose(g["dLdparams"][:, k], fd, rtol=1e-4, atol=1e-6 * np.abs(fd).max())


def test_jvp_matches_central_difference_of_rhs():
    rng = np.random.default_rng(2)
    cases = [("isochrone", 6, 0), ("mw", 6, 4), ("precession", 9, 3), ("quintessence", 3, 4), ("loghalo", 6, 3)]
    base_p = {"mw": [6.8, 0.5, 54.0, 0.9], "precession": [0.5, 0.7, 0.3], "quintessence": [0.7, 0.8, 0.3, 9e-5],
              "loghalo": [1.0, 0.2, 0.7], "isochrone": [0.0]}
    for system, d, np_ in cases:
        t = {"precession": 0.2, "quintessence": -1.0}.get(system, 0.0)
        y = rng.uniform(-1, 1, d) + (np.array([3, 4, 1, 0, 0, 0]) if d == 6 else 0)
        if system == "precession":
            y = np.concatenate([u / np.linalg.norm(u) for u in rng.normal(size=(3, 3))])
        if system == "quintessence":
            y = np.array([0.3, 0.5, 1.0])
        p = np.array(base_p[system], dtype=float)
        vy, vp = rng.normal(size=d), rng.normal(size=max(np_, 1))
        j = O.jvp(system, t, y, p, vy, vp if np_ else None)
        eps = 1e-6
        fp = O.rhs(system, t, y + eps * vy, p + (eps * vp if np_ else 0))
        fm = O.rhs(system, t, y - eps * vy, p - (eps * vp if np_ else 0))
        fd = (fp - fm) / (2 * eps)
        assert np.allclose(j, fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max()), system


# ---------------------------------------------------------------------------------------------
def test_converged_reference_self_check():
    """Appendix A / D: a second reference solve 10x looser must agree within eps_req/10."""
    e = W.mw(n=16, seed=16, t1=1000.0)
    a = O.solve("mw", e.y0, e.params, e.t0, e.t1, e.saveat, 1e-13, 1e-13, method="vern7")["y"][:, -1]
    b = O.solve("mw", e.y0, e.params, e.t0, e.t1, e.saveat, 1e-12, 1e-12, method="vern7")["y"][:, -1]
    rE, vE = M.orbit_scales("mw", e.y0, e.params)
    assert np.max(M.orbit_error(b, a, rE, vE)) < 1e-4 / 10


# ---------------------------------------------------------------------------------------------
def test_status_codes_and_nan_outputs():
    e = W.isochrone(n=6, seed=17)
    y0 = e.y0.copy()
    y0[1, 2] = np.nan
    t1 = e.t1.copy()
    t1[2] = 0.0  # empty interval
    sv = np.stack([e.saveat] * 6)
    sv[3, 10] = 150.0  # outside [t0, t1]
    sv[4, 6] = 45.0  # not non-decreasing: that point alone is rejected
    res = O.solve("isochrone", y0, None, e.t0, t1, sv, 1e-8, 1e-8)
    st = res["status"]
    assert st[0] == 0
    assert st[1] == O.ST_NONFINITE and np.all(np.isnan(res["y"][1]))
    assert st[2] == O.ST_EMPTY_INTERVAL and np.array_equal(res["y"][2], np.repeat(y0[2:3], 11, 0))
    assert st[3] & O.ST_SAVEAT_OUTSIDE
    assert np.all(np.isnan(res["y"][3, 10])) and np.all(np.isfinite(res["y"][3, :10]))
    assert st[4] == O.ST_SAVEAT_OUTSIDE and np.all(np.isnan(res["y"][4, 6]))
    assert np.all(np.isfinite(np.delete(res["y"][4], 6, axis=0)))
    res = O.solve("isochrone", e.y0, None, e.t0, e.t1, e.saveat, 1e-8, 1e-8, max_steps=20)
    assert np.all(res["status"] == O.ST_MAX_STEPS) and np.all(np.isnan(res["y"]))
    assert np.all(res["n_accept"] + res["n_reject"] == 20)
    # outputs at t0 are the initial state exactly
    res = O.solve("isochrone", e.y0, None, e.t0, e.t1, e.saveat, 1e-8, 1e-8)
    assert np.array_equal(res["y"][:, 0], e.y0)
