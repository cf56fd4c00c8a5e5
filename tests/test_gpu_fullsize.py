"""Parity at the full workload sizes, in the launch configuration bench.py times, on outputs the oracle
computes one by one: a seeded sample of trajectories is solved (and differentiated) by the oracle at a
converged tolerance, and the GPU ensemble's values for those members must meet the paper's budgets
(Eq. accept: at most 1 in 48 sampled members above the budget, none above 10x). Every member of
the full ensemble must succeed and be finite.

* configuration 2: 2^20 Milky-Way orbits, the headline step (forward recording the tape and the
  persistent reverse at rtol 1e-8) in the FP32-stage mode and in the FP32-pair mode: final states
  (Eq. st-fwderr, 1e-4) and the gradient of the endpoint loss with respect to (y0, theta) (relative,
  1e-3);
* configuration 3 on the paper's interval (r = 100 M -> 10 M): 10^6 FP64 Verner 7 gradients with
  checkpoint stride 16, whose tape stays under 20 GB (a sixth of stride 1's);
* configuration 3: 10^6 precession solves, FP64 Verner 7 at 3.16e-9: final spin directions
  (Eq. prec-err, 2e-7 rad) and the adjoint of the summed tilt cosines with respect to (q, chi1, chi2);
* configuration 4: 10^4 quintessence cosmologies, FP32-pair Tsit5 at 1e-6: distances (1e-4 c/H0)
  and the adjoint of a chi^2 against mock distances.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ensure_built
from paper_2609_28458_gb300 import api
from paper_2609_28458_gb300 import metrics as M
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SAMPLE = 48


def _sample(n, seed):
    return np.sort(np.random.default_rng(seed).choice(n, SAMPLE, replace=False))


def _budget_ok(err, budget):
    err = np.asarray(err)
    return np.all(np.isfinite(err)) and np.sum(err > budget) <= 1 and np.all(err <= 10 * budget)


@pytest.mark.parametrize("prec", ["fp32", "fp32df"])
def test_config2_mw_full_size_headline_step(prec):
    ensure_built()
    e = W.mw(n=1 << 20, seed=1000)
    dev = torch.device("cuda")
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    rtol = 1e-8
    ptgt = pr.clone()
    ptgt[:, :3] *= 1.01
    y_tgt = api.solve("mw", y0, ptgt, t0, t1, sv, rtol, rtol, precision="fp64")["y"]
    probe = api.solve("mw", y0, pr, t0, t1, sv, rtol, rtol, precision=prec)
    nb = api.tape_bytes("mw", e.n, n_accept=probe["n_accept"], precision=prec)
    ws = api.Workspace(dev)
    s = api.solve("mw", y0, pr, t0, t1, sv, rtol, rtol, precision=prec, kernel="persistent", record_tape=True,
                  workspace=ws, tape_nbytes=nb)
    w = s["y"] - y_tgt
    g = api.vjp("mw", y0, pr, t0, t1, sv, rtol, rtol, w, precision=prec, kernel="persistent", reuse_tape=s,
                workspace=ws)
    torch.cuda.synchronize()
    assert int((s["status"] != 0).sum()) == 0
    assert bool(torch.isfinite(g["dLdy0"]).all()) and bool(torch.isfinite(g["dLdparams"]).all())
    idx = _sample(e.n, 7)
    sub = e.subset(idx)
    ref = O.solve("mw", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, 1e-12, 1e-12, method="vern7")
    rE, vE = M.orbit_scales("mw", sub.y0, sub.params)
    err = M.orbit_error(s["y"][idx, -1].cpu().numpy(), ref["y"][:, -1], rE, vE)
    assert _budget_ok(err, 1e-4), np.sort(err)[-3:]
    wn = w[idx].cpu().numpy()
    gref = O.grad("mw", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, wn, rtol=1e-11, atol=1e-11, method="vern7")
    gy = np.concatenate([g["dLdy0"][idx].cpu().numpy(), g["dLdparams"][idx].cpu().numpy()], axis=1)
    ry = np.concatenate([gref["dLdy0"], gref["dLdparams"]], axis=1)
    rel = np.linalg.norm(gy - ry, axis=1) / np.linalg.norm(ry, axis=1)
    assert _budget_ok(rel, 1e-3), np.sort(rel)[-3:]


def test_config3_precession_full_size():
    ensure_built()
    e = W.precession(n=1_000_000, seed=2000)
    dev = torch.device("cuda")
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    rtol = 3.16e-9
    ws = api.Workspace(dev)
    probe = api.solve("precession", y0, pr, t0, t1, sv, rtol, rtol, method="vern7", precision="fp64")
    nb = api.tape_bytes("precession", e.n, n_accept=probe["n_accept"], precision="fp64")
    s = api.solve("precession", y0, pr, t0, t1, sv, rtol, rtol, method="vern7", precision="fp64", kernel="persistent",
                  record_tape=True, workspace=ws, tape_nbytes=nb)
    y = s["y"][:, -1]
    w = torch.cat([y[:, 3:6] + y[:, 6:9], y[:, 0:3], y[:, 0:3]], dim=1).unsqueeze(1)
    g = api.vjp("precession", y0, pr, t0, t1, sv, rtol, rtol, w, method="vern7", precision="fp64", kernel="persistent",
                reuse_tape=s, workspace=ws)
    torch.cuda.synchronize()
    st = s["status"].cpu().numpy()
    assert np.all((st & ~8) == 0)          # success or empty interval (v0 >= 0.3 for heavy binaries)
    moving = np.nonzero(st == 0)[0]
    idx = np.sort(np.random.default_rng(8).choice(moving, SAMPLE, replace=False))
    sub = e.subset(idx)
    ref = O.solve("precession", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, 1e-12, 1e-12, method="vern7")
    err = M.precession_error(s["y"][idx, -1].cpu().numpy(), ref["y"][:, -1])
    assert _budget_ok(err, 2e-7), np.sort(err)[-3:]
    gref = O.grad("precession", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, w[idx].cpu().numpy(), rtol=1e-12,
                  atol=1e-12, method="vern7")
    gp, rp = g["dLdparams"][idx].cpu().numpy(), gref["dLdparams"]
    rel = np.linalg.norm(gp - rp, axis=1) / np.linalg.norm(rp, axis=1)
    assert _budget_ok(rel, 1e-5), np.sort(rel)[-3:]


def test_config3_paper_interval_checkpointed_gradient():
    ensure_built()
    e = W.precession(n=1_000_000, seed=2001, paper_interval=True)
    dev = torch.device("cuda")
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    rtol, S = 3.16e-9, 16
    kw = dict(method="vern7", precision="fp64", kernel="persistent", ckpt_stride=S)
    probe = api.solve("precession", y0, pr, t0, t1, sv, rtol, rtol, **kw)
    nb = api.tape_bytes("precession", e.n, n_accept=probe["n_accept"], precision="fp64", ckpt_stride=S)
    nb1 = api.tape_bytes("precession", e.n, n_accept=probe["n_accept"], precision="fp64", ckpt_stride=1)
    assert nb < 20e9 and nb1 > 5 * nb, (nb, nb1)
    ws = api.Workspace(dev)
    s = api.solve("precession", y0, pr, t0, t1, sv, rtol, rtol, record_tape=True, workspace=ws, tape_nbytes=nb, **kw)
    y = s["y"][:, -1]
    w = torch.cat([y[:, 3:6] + y[:, 6:9], y[:, 0:3], y[:, 0:3]], dim=1).unsqueeze(1)
    g = api.vjp("precession", y0, pr, t0, t1, sv, rtol, rtol, w, reuse_tape=s, workspace=ws, **kw)
    torch.cuda.synchronize()
    assert int((s["status"] != 0).sum()) == 0 and bool(torch.isfinite(g["dLdparams"]).all())
    idx = _sample(e.n, 11)
    sub = e.subset(idx)
    ref = O.solve("precession", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, 1e-12, 1e-12, method="vern7")
    err = M.precession_error(s["y"][idx, -1].cpu().numpy(), ref["y"][:, -1])
    assert _budget_ok(err, 2e-7), np.sort(err)[-3:]
    gref = O.grad("precession", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, w[idx].cpu().numpy(), rtol=1e-12,
                  atol=1e-12, method="vern7")
    gp, rp = g["dLdparams"][idx].cpu().numpy(), gref["dLdparams"]
    rel = np.linalg.norm(gp - rp, axis=1) / np.linalg.norm(rp, axis=1)
    assert _budget_ok(rel, 1e-5), np.sort(rel)[-3:]


def test_config4_quintessence_full_size():
    ensure_built()
    e = W.quintessence(n=10_000, seed=3000, rtol=1e-6)
    dev = torch.device("cuda")
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    s = api.solve("quintessence", y0, pr, e.t0, e.t1, e.saveat, 1e-6, 1e-9, precision="fp32df", kernel="persistent")
    # chi^2 of the distances against seeded mock values: dL/dy at every output
    rng = np.random.default_rng(9)
    mock = s["y"].cpu().numpy() * (1 + 0.01 * rng.standard_normal(s["y"].shape))
    w = torch.as_tensor(2 * (s["y"].cpu().numpy() - mock) / (0.01 ** 2 + 1e-30), device=dev)
    g = api.vjp("quintessence", y0, pr, e.t0, e.t1, e.saveat, 1e-6, 1e-9, w, precision="fp32df", kernel="persistent")
    torch.cuda.synchronize()
    assert int((s["status"] != 0).sum()) == 0
    idx = _sample(e.n, 10)
    sub = e.subset(idx)
    ref = O.solve("quintessence", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, 1e-12, 1e-15, method="vern7")
    err = M.distance_error(s["y"][idx].cpu().numpy(), ref["y"], sub.params, sub.saveat)
    assert _budget_ok(err, 1e-4), np.sort(err)[-3:]
    gref = O.grad("quintessence", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, w[idx].cpu().numpy(), rtol=1e-12,
                  atol=1e-15, method="vern7")
    gp, rp = g["dLdparams"][idx].cpu().numpy(), gref["dLdparams"]
    rel = np.linalg.norm(gp - rp, axis=1) / np.linalg.norm(rp, axis=1)
    assert _budget_ok(rel, 1e-3), np.sort(rel)[-3:]
