"""The synthetic inputs follow their stated recipe (CPU): seeded, with the sizes, ranges and
distributions of the paper's workloads (Secs. 3-5) as the benchmark uses them."""
import numpy as np

from paper_2609_28458_gb300 import workloads as W


def _unit(v):
    return np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-12)


def test_seeded_and_reproducible():
    for gen in (W.isochrone, W.mw, W.precession, W.quintessence, W.loghalo):
        a, b = gen(n=64, seed=7), gen(n=64, seed=7)
        assert np.array_equal(a.y0, b.y0) and np.array_equal(a.params, b.params)
        c = gen(n=64, seed=8)
        assert not np.array_equal(a.y0, c.y0) or not np.array_equal(a.params, c.params)


def test_isochrone_recipe():
    e = W.isochrone(n=4096, seed=0)
    assert e.y0.shape == (4096, 6) and e.params.shape == (4096, 0)
    r = np.linalg.norm(e.y0[:, :3], axis=1)
    assert r.min() >= 0.5 and r.max() <= 5.0
    s = np.sqrt(1 + r * r)
    vc = np.sqrt(r * r / ((1 + s) ** 2 * s))
    ratio = np.linalg.norm(e.y0[:, 3:], axis=1) / vc
    assert ratio.min() >= 0.3 - 1e-12 and ratio.max() <= 0.9 + 1e-12
    energy = 0.5 * (e.y0[:, 3:] ** 2).sum(1) - 1 / (1 + s)
    assert np.all(energy < 0)                           # every orbit bound
    assert np.allclose(e.saveat, np.linspace(0, 100, 11)) and e.rtol == 1e-10 and e.atol == 1e-12


def test_milky_way_recipe():
    e = W.mw(n=50000, seed=1000)
    x, v = e.y0[:, :3], e.y0[:, 3:]
    R = np.hypot(x[:, 0], x[:, 1])
    assert R.min() >= 4.0 and R.max() <= 20.0 and np.abs(x[:, 2]).max() <= 2.0
    q = e.params[:, 3]
    assert q.min() >= 0.8 and q.max() <= 1.2 and np.allclose(e.params[:, :3], [6.8, 0.5, 54.0])
    phihat = np.stack([-x[:, 1] / R, x[:, 0] / R, np.zeros_like(R)], axis=1)
    dv = v - W.mw_vcirc(R)[:, None] * phihat
    sig = 20.0 * W.KMS_IN_KPC_MYR                      # 20 km/s per component
    assert abs(dv.std() / sig - 1) < 0.02 and abs(dv.mean()) < 0.02 * sig
    assert np.all(e.t0 == 0.0) and np.all(e.t1 == 3000.0) and np.array_equal(e.saveat, [3000.0])


def test_precession_recipe():
    e = W.precession(n=20000, seed=2000)
    q, chi1, chi2 = e.params.T
    assert q.min() >= 0.1 and q.max() <= 1.0 and chi1.min() >= 0 and chi2.max() <= 1.0
    assert _unit(e.y0[:, 0:3]) and _unit(e.y0[:, 3:6]) and _unit(e.y0[:, 6:9])
    M = e.extra["M"]
    assert M.min() >= 10.0 and M.max() <= 100.0
    # v0 from the 20 Hz gravitational-wave frequency: empty intervals exactly above M = 87.2 Msun
    empty = e.t0 >= e.t1
    assert np.all(M[empty] > 87.0) and np.all(M[~empty] < 87.5)
    assert abs(empty.mean() - (100 - 87.2) / 90) < 0.01
    cos1 = e.y0[:, 3:6] @ np.array([0.0, 0.0, 1.0])
    assert abs(cos1.mean()) < 0.02                       # isotropic tilts: cos uniform on [-1, 1]


def test_quintessence_recipe():
    e = W.quintessence(n=20000, seed=3000, rtol=1e-5)
    a0, lam, om, orad = e.params.T
    assert lam.min() >= 0 and lam.max() <= 1.5 and om.min() >= 0.28 and om.max() <= 0.34
    assert np.allclose(orad, 9e-5) and np.allclose(a0, 1 - om - orad)
    assert np.allclose(e.t0, -np.log(51.0)) and np.all(e.t1 == 0.0)
    assert len(e.saveat) == 8 and e.saveat[-1] == 0.0 and np.all(np.diff(e.saveat) > 0)
    assert e.atol == 1e-3 * e.rtol
    dense = W.quintessence(n=4, dense=True)
    assert len(dense.saveat) == 64 and dense.saveat[-1] == 0.0
