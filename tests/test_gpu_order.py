"""Longest-first ordering of the forward launches (gs_options.order) changes which lane runs which
trajectory and when, never a trajectory's arithmetic: outputs and step counts are bit-for-bit those of
the stored order, for the estimate and for a cost hint, in the persistent and the plain kernels and
through gs_vjp (whose reverse pass is always ordered by the recorded step counts)."""
import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from paper_2609_28458_gb300 import api
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _args(e, dev):
    T = lambda x: torch.as_tensor(x, device=dev)
    return (T(e.y0), T(e.params) if e.params.size else None, T(e.t0), T(e.t1), T(e.saveat))


@pytest.mark.parametrize("system,gen,method,prec", [
    ("mw", lambda: W.mw(n=40000, seed=61, t1=1000.0), "tsit5", "fp32df"),
    ("precession", lambda: W.precession(n=40000, seed=62), "vern7", "fp64"),
    ("isochrone", lambda: W.isochrone(n=4096, seed=63), "dopri5", "fp64"),
])
@pytest.mark.parametrize("kernel", ["persistent", "plain"])
def test_order_does_not_change_results(system, gen, method, prec, kernel):
    ensure_built()
    e = gen()
    dev = torch.device("cuda")
    y0, pr, t0, t1, sv = _args(e, dev)
    rtol = e.rtol if system != "mw" else 1e-8
    kw = dict(method=method, precision=prec, kernel=kernel)
    base = api.solve(system, y0, pr, t0, t1, sv, rtol, rtol, order="natural", **kw)
    base = {k: v.clone() for k, v in base.items()}
    hint = (base["n_accept"] + base["n_reject"]).clone()
    for order, extra in (("estimate", {}), ("hint", {"cost_hint": hint}), ("auto", {})):
        r = api.solve(system, y0, pr, t0, t1, sv, rtol, rtol, order=order, **extra, **kw)
        torch.cuda.synchronize()
        for k in ("y", "status", "n_accept", "n_reject"):
            assert torch.equal(torch.nan_to_num(r[k]), torch.nan_to_num(base[k])), (order, k)


def test_vjp_results_do_not_depend_on_order():
    ensure_built()
    e = W.mw(n=40000, seed=64, t1=800.0)
    dev = torch.device("cuda")
    y0, pr, t0, t1, sv = _args(e, dev)
    w = torch.as_tensor(np.random.default_rng(1).normal(size=(e.n, 1, 6)), device=dev)
    a = api.vjp("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, w, precision="fp32df", order="natural")
    b = api.vjp("mw", y0, pr, t0, t1, sv, 1e-8, 1e-8, w, precision="fp32df", order="estimate")
    torch.cuda.synchronize()
    for k in ("dLdy0", "dLdparams", "y", "n_accept"):
        assert torch.equal(a[k], b[k]), k


def test_fewer_lanes_per_warp_give_identical_results():
    """gs_options.warp_lanes: the persistent kernels hand trajectories to that many lanes of each warp
    only (the rest retire at once). The per-trajectory arithmetic is the same, so solutions, step
    counts and gradients are bit for bit those of full warps, for forward, adjoint and sensitivities."""
    ensure_built()
    dev = torch.device("cuda")
    e = W.isochrone(n=1000, seed=71)
    y0 = torch.as_tensor(e.y0, device=dev)
    w = torch.as_tensor(np.random.default_rng(2).normal(size=(e.n, e.saveat.shape[-1], 6)), device=dev)
    ref_s = api.solve("isochrone", y0, None, e.t0, e.t1, e.saveat, e.rtol, e.atol, kernel="persistent")
    ref_g = api.vjp("isochrone", y0, None, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, kernel="persistent")
    for lanes in (16, 8, 1):
        s = api.solve("isochrone", y0, None, e.t0, e.t1, e.saveat, e.rtol, e.atol, kernel="persistent",
                      warp_lanes=lanes)
        g = api.vjp("isochrone", y0, None, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, kernel="persistent",
                    warp_lanes=lanes)
        torch.cuda.synchronize()
        for k in ("y", "status", "n_accept", "n_reject"):
            assert torch.equal(s[k], ref_s[k]), (lanes, k)
        assert torch.equal(g["dLdy0"], ref_g["dLdy0"]), lanes
    m = W.mw(n=600, seed=72, t1=500.0)
    dp = torch.zeros((m.n, 4, 1), dtype=torch.float64, device=dev)
    dp[:, 3, 0] = 1.0
    a = api.jvp("mw", torch.as_tensor(m.y0, device=dev), m.params, m.t0, m.t1, m.saveat, m.rtol, m.atol, dparams=dp)
    b = api.jvp("mw", torch.as_tensor(m.y0, device=dev), m.params, m.t0, m.t1, m.saveat, m.rtol, m.atol, dparams=dp,
                warp_lanes=8)
    torch.cuda.synchronize()
    assert torch.equal(a["S"], b["S"]) and torch.equal(a["y"], b["y"])
