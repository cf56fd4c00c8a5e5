"""GPU gradients: the discrete adjoint (gs_vjp) against the oracle.

* VJP of every right-hand side: the dot-product test <w, J v> = <J^T w, v>, with J v from the
  oracle's dual numbers and J^T w from the library's hand-derived reverse code (FP64: 1e-12
  relative; FP32: 2e-5).
* gs_vjp in FP64 against the oracle's forward sensitivities (Sec. 2.3, Eq. stage-sens, chained with
  Eq. chain): on trajectories whose step sequence equals the oracle's, the adjoint is the exact
  derivative of the same numerical solution, so the two agree to rounding (1e-8 relative).
* FP32-stage gradients against the FP64 oracle: within the paper's gradient budget (1e-3, the
  orbit-gradient requirement of Sec. 3) in relative norm.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ensure_built, gpu_solve, gpu_vjp
from paper_2609_28458_gb300 import _abi, api
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STATES = {
    "isochrone": lambda rng: (0.0, np.concatenate([rng.uniform(-3, 3, 3), rng.uniform(-0.5, 0.5, 3)]), np.zeros(0)),
    "mw": lambda rng: (0.0, np.concatenate([rng.uniform(-15, 15, 2), rng.uniform(-2, 2, 1), rng.uniform(-0.3, 0.3, 3)]),
                       np.array([6.8, 0.5, 54.0, rng.uniform(0.8, 1.2)])),
    "loghalo": lambda rng: (0.0, np.concatenate([rng.uniform(-2, 2, 3), rng.uniform(-1, 1, 3)]),
                            np.array([1.0, 0.2, rng.uniform(0.6, 0.9)])),
    "precession": lambda rng: (rng.uniform(0.1, 0.3),
                               np.concatenate([u / np.linalg.norm(u) for u in rng.normal(size=(3, 3))]),
                               np.array([rng.uniform(0.1, 1), rng.uniform(0, 1), rng.uniform(0, 1)])),
    "quintessence": lambda rng: (rng.uniform(-3.9, 0.0), np.array([rng.uniform(0, 0.5), rng.uniform(0, 0.8), rng.uniform(0, 3)]),
                                 np.array([0.69, rng.uniform(0, 1.5), rng.uniform(0.28, 0.34), 9e-5])),
}


@pytest.mark.parametrize("system", list(STATES))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("fp32df", 2e-5)])
def test_vjp_dot_product(system, precision, tol):
    ensure_built()
    rng = np.random.default_rng(5)
    M = 64
    d, p = O.dims(system)
    ts, ys, ps, ws, vys, vps = [], [], [], [], [], []
    for _ in range(M):
        t, y, pp = STATES[system](rng)
        ts.append(t); ys.append(y); ps.append(pp)
        ws.append(rng.normal(size=d)); vys.append(rng.normal(size=d)); vps.append(rng.normal(size=max(p, 1)))
    ts, ys, ps, ws, vys, vps = map(np.array, (ts, ys, ps, ws, vys, vps))
    dev = torch.device("cuda")
    f, gy, gp = api.rhs(system, torch.as_tensor(ts, device=dev), torch.as_tensor(ys, device=dev),
                        ps if p else None, ws, precision=precision)
    f, gy = f.cpu().numpy(), gy.cpu().numpy()
    gp = gp.cpu().numpy() if p else np.zeros((M, 0))
    for m in range(M):
        fo = O.rhs(system, ts[m], ys[m], ps[m] if p else None)
        assert np.allclose(f[m], fo, rtol=tol * 10, atol=tol * 10 * np.abs(fo).max())
        jv = O.jvp(system, ts[m], ys[m], ps[m] if p else None, vys[m], vps[m] if p else None)
        lhs = ws[m] @ jv
        rhs = gy[m] @ vys[m] + (gp[m] @ vps[m][:p] if p else 0.0)
        scale = np.abs(ws[m]).max() * (np.abs(jv).max() + 1e-300) * d
        assert abs(lhs - rhs) <= tol * scale, (m, lhs, rhs)


GRAD_CASES = [
    ("mw", lambda: W.mw(n=64, seed=41, t1=1000.0, rtol=1e-9), "tsit5"),
    ("mw", lambda: W.mw(n=32, seed=42, t1=600.0, rtol=1e-9), "vern7"),
    ("isochrone", lambda: W.isochrone(n=64, seed=43), "tsit5"),  # 11 outputs: dense-output cotangents
    ("isochrone", lambda: W.isochrone(n=32, seed=44), "vern7"),  # shortened-step outputs
    ("quintessence", lambda: W.quintessence(n=64, seed=45, rtol=1e-9), "dopri5"),
    ("quintessence", lambda: W.quintessence(n=64, seed=46, rtol=1e-9, dense=True), "tsit5"),
    ("precession", lambda: W.precession(n=32, seed=47, paper_interval=True, rtol=1e-9), "vern7"),
    ("loghalo", lambda: W.loghalo(n=64, seed=48, rtol=1e-9), "tsit5"),
]


@pytest.mark.parametrize("system,gen,method", GRAD_CASES)
def test_adjoint_fp64_equals_forward_sensitivities(system, gen, method):
    e = gen()
    rng = np.random.default_rng(1)
    d, p = O.dims(system)
    w = rng.normal(size=(e.n, e.saveat.shape[-1], d))
    ref = O.grad(system, e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=e.rtol, atol=e.atol, method=method)
    g = gpu_vjp(e, w, method=method)
    assert np.array_equal(g["status"], ref["status"])
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"])
    assert same.mean() >= 0.9
    gy = np.concatenate([g["dLdy0"], g["dLdparams"]], axis=1)
    ry = np.concatenate([ref["dLdy0"], ref["dLdparams"]], axis=1)
    err = np.linalg.norm(gy - ry, axis=1) / np.linalg.norm(ry, axis=1)
    assert err[same].max() <= 1e-8, (err[same].max(), np.argmax(np.where(same, err, 0)))
    # the re-run forward solve of gs_vjp is the forward solve
    s = gpu_solve(e, method=method)
    assert np.array_equal(s["y"], g["y"])


def _gerr(g, ref):
    gy = np.concatenate([g["dLdy0"], g["dLdparams"]], axis=1)
    ry = np.concatenate([ref["dLdy0"], ref["dLdparams"]], axis=1)
    return np.linalg.norm(gy - ry, axis=1) / np.linalg.norm(ry, axis=1)


@pytest.mark.parametrize("kernel,prec", [("plain", "fp32"), ("persistent", "fp32"), ("persistent", "fp32df")])
def test_adjoint_fp32_meets_gradient_budget(kernel, prec):
    """FP32-stage adjoint on 3 Gyr orbits at a tolerance meeting the gradient budget (1e-3, Sec. 3)
    against the oracle's converged forward-sensitivity gradient."""
    e = W.mw(n=256, seed=49, rtol=3.16e-9)
    w = np.random.default_rng(2).normal(size=(e.n, 1, 6))
    ref = O.grad("mw", e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=1e-11, atol=1e-11, method="vern7")
    a = gpu_vjp(e, w, precision=prec, kernel=kernel)
    assert np.all(a["status"] == 0)
    assert np.percentile(_gerr(a, ref), 99) <= 1e-3, np.percentile(_gerr(a, ref), 99)


@pytest.mark.parametrize("method", ["tsit5", "dopri5"])
@pytest.mark.parametrize("prec", ["fp32", "fp32df"])
def test_saved_stage_factors_match_recomputation(method, prec):
    """The persistent FP32 reverse pass keeps each stage's Jacobian factors (Milky-Way system) in
    shared memory from the stage recomputation; the plain reverse pass re-evaluates them inside every
    VJP. On the same tape and cotangents the two gradients agree to FP32 rounding."""
    ensure_built()
    dev = torch.device("cuda")
    e = W.mw(n=3000, seed=77, t1=750.0)
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    ws = api.Workspace(dev)
    kw = dict(method=method, precision=prec)
    s = api.solve("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, kernel="persistent", record_tape=True, workspace=ws, **kw)
    w = torch.as_tensor(np.random.default_rng(4).normal(size=(e.n, 1, 6)), device=dev)
    gp = api.vjp("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, w, kernel="persistent", reuse_tape=s, workspace=ws, **kw)
    gq = api.vjp("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, w, kernel="plain", reuse_tape=s, workspace=ws, **kw)
    assert int((s["status"] != 0).sum()) == 0
    a = torch.cat([gp["dLdy0"], gp["dLdparams"]], dim=1).cpu().numpy()
    b = torch.cat([gq["dLdy0"], gq["dLdparams"]], dim=1).cpu().numpy()
    rel = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(np.isfinite(rel)) and np.percentile(rel, 99) < 1e-4 and rel.max() < 1e-3, (rel.max(), np.median(rel))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32df"])
@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_recording_does_not_change_the_solve(prec, kernel):
    """A solve gives bit-identical states and step counts whether or not it records the tape, so a
    tape sized from the accepted-step counts of an earlier plain solve always fits."""
    ensure_built()
    dev = torch.device("cuda")
    e = W.mw(n=20000, seed=11, t1=750.0)
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    kw = dict(precision=prec, kernel=kernel)
    s0 = api.solve("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, **kw)
    nb = api.tape_bytes("mw", e.n, n_accept=s0["n_accept"], precision=prec)
    s1 = api.solve("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, record_tape=True, workspace=api.Workspace(dev),
                   tape_nbytes=nb, **kw)
    assert int((s1["status"] != 0).sum()) == 0
    assert torch.equal(s0["n_accept"], s1["n_accept"]) and torch.equal(s0["n_reject"], s1["n_reject"])
    assert torch.equal(s0["y"], s1["y"])


def test_adjoint_converges_to_oracle_gradient():
    """Discretisation: the FP64 adjoint at a tight tolerance against the oracle's converged
    forward-sensitivity gradient (Verner 7, rtol 1e-11)."""
    e = W.mw(n=128, seed=55, t1=1000.0, rtol=1e-10)
    w = np.random.default_rng(6).normal(size=(e.n, 1, 6))
    ref = O.grad("mw", e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=1e-11, atol=1e-11, method="vern7")
    g = gpu_vjp(e, w, precision="fp64", kernel="persistent")
    assert np.percentile(_gerr(g, ref), 99) <= 1e-4, np.percentile(_gerr(g, ref), 99)


def test_adjoint_agrees_with_central_differences_of_gpu_solve():
    e = W.mw(n=16, seed=50, t1=800.0, rtol=1e-10)
    rng = np.random.default_rng(3)
    w = rng.normal(size=(e.n, 1, 6))
    g = gpu_vjp(e, w)
    for k in range(4):
        eps = 1e-5 * abs(e.params[0, k])
        ep, em = e.subset(np.arange(e.n)), e.subset(np.arange(e.n))
        ep.params[:, k] += eps
        em.params[:, k] -= eps
        fd = (np.sum(w * gpu_solve(ep, rtol=1e-12, atol=1e-12)["y"], axis=(1, 2)) -
              np.sum(w * gpu_solve(em, rtol=1e-12, atol=1e-12)["y"], axis=(1, 2))) / (2 * eps)
        assert np.allclose(g["dLdparams"][:, k], fd, rtol=1e-3, atol=1e-4 * np.abs(fd).max())


def test_adjoint_status_conventions():
    e = W.precession(n=64, seed=51)
    w = np.ones((e.n, 1, 9))
    g = gpu_vjp(e, w, method="vern7")
    empty = (g["status"] & O.ST_EMPTY_INTERVAL) != 0
    assert empty.any()
    assert np.all(g["dLdy0"][empty] == 1.0) and np.all(g["dLdparams"][empty] == 0.0)
    e2 = W.mw(n=4, seed=52, t1=500.0)
    e2.y0[1, 0] = np.nan
    g = gpu_vjp(e2, np.ones((4, 1, 6)), max_steps=100000)
    assert np.all(np.isnan(g["dLdy0"][1])) and np.all(np.isfinite(g["dLdy0"][[0, 2, 3]]))
    # a workspace too small for the tape: overflow flagged, gradients NaN, nothing else disturbed
    fixed = api.tape_bytes("mw", 4, n_accept=torch.zeros(4, dtype=torch.int32)) - (16 + 32 * 80)  # no chunk
    g = gpu_vjp(e2, np.ones((4, 1, 6)), tape_nbytes=fixed + 4 * (16 + 32 * 80))
    over = (g["status"] & _abi.ST_TAPE_OVERFLOW) != 0
    assert over.any() and np.all(np.isnan(g["dLdy0"][over])) and np.all(np.isfinite(g["y"][~np.isnan(e2.y0).any(1)]))


def test_reuse_tape_matches_rerun():
    ensure_built()
    e = W.mw(n=512, seed=53, t1=2000.0)
    dev = torch.device("cuda")
    ws = api.Workspace(dev)
    y0 = torch.as_tensor(e.y0, device=dev)
    w = torch.as_tensor(np.random.default_rng(4).normal(size=(e.n, 1, 6)), device=dev)
    for prec in ("fp64", "fp32", "fp32df"):
        s = api.solve("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, precision=prec, record_tape=True,
                      workspace=ws, steps_hint=2000)
        a = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, precision=prec, reuse_tape=s,
                    workspace=ws)
        b = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(a["dLdy0"], b["dLdy0"]) and torch.equal(a["dLdparams"], b["dLdparams"])
        assert torch.equal(s["y"], b["y"])


def test_tape_capacity_limits_recorded_steps():
    """opt.tape_capacity: trajectories with more accepted steps than the capacity get
    GS_ST_TAPE_OVERFLOW and NaN gradients; the others are unchanged (same step sequence, same tape)."""
    ensure_built()
    e = W.mw(n=256, seed=57, t1=1000.0, rtol=1e-8)
    e.t1 = np.random.default_rng(5).uniform(50.0, 1000.0, e.n)
    e.saveat = np.stack([e.t1], axis=1)
    dev = torch.device("cuda")
    y0 = torch.as_tensor(e.y0, device=dev)
    w = torch.as_tensor(np.random.default_rng(6).normal(size=(e.n, 1, 6)), device=dev)
    for prec in ("fp64", "fp32df"):
        full = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, precision=prec)
        nacc = full["n_accept"].cpu().numpy()
        cap = int(np.median(nacc))
        lim = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, precision=prec, tape_capacity=cap)
        torch.cuda.synchronize()
        st = lim["status"].cpu().numpy()
        over = (st & _abi.ST_TAPE_OVERFLOW) != 0
        assert np.array_equal(over, nacc > cap) and over.any() and (~over).any()
        g, gf = lim["dLdy0"].cpu().numpy(), full["dLdy0"].cpu().numpy()
        assert np.all(np.isnan(g[over])) and np.array_equal(g[~over], gf[~over])
        assert np.array_equal(lim["dLdparams"].cpu().numpy()[~over], full["dLdparams"].cpu().numpy()[~over])
        # the forward solution itself is not affected by the tape
        assert torch.equal(lim["y"], full["y"])


def test_autograd_function():
    ensure_built()
    e = W.mw(n=128, seed=54, t1=1000.0)
    dev = torch.device("cuda")
    y0 = torch.as_tensor(e.y0, device=dev).requires_grad_(True)
    pr = torch.as_tensor(e.params, device=dev).requires_grad_(True)
    y, st = api.solve_autograd("mw", y0, pr, e.t0, e.t1, e.saveat, e.rtol, e.atol)
    loss = 0.5 * (y ** 2).sum()
    loss.backward()
    g = gpu_vjp(e, y.detach().cpu().numpy(), kernel="persistent")
    assert np.array_equal(y0.grad.cpu().numpy(), g["dLdy0"])
    assert np.array_equal(pr.grad.cpu().numpy(), g["dLdparams"])
