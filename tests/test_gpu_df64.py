"""Precision mode GS_DF64 (state, stages and error estimate in double-FP32 arithmetic, ~48 bits) against
the oracle, at the tolerances the FP64-only workloads use:

* the isochrone workload at rtol 1e-10 meets the parity gate of the FP64 path (1e-9 relative per
  trajectory and output against the oracle's same-algorithm solve);
* precession (Verner 7, rtol 3.16e-9) meets the 2e-7 rad budget against a converged oracle solve,
  and agrees with the FP64 GPU solve far inside it;
* the df64 adjoint equals the oracle's forward-sensitivity gradient on the members whose step
  sequence matches the oracle's (1e-8 relative), as the FP64 adjoint does;
* systems whose right-hand sides need exp or log (MW, quintessence) and gs_jvp reject the mode.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ensure_built, gpu_solve, gpu_vjp, rel_err
from paper_2609_28458_gb300 import _abi, api
from paper_2609_28458_gb300 import metrics as M
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def oracle_solve(e, **kw):
    return O.solve(e.system, e.y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, method=e.method, **kw)


@pytest.mark.parametrize("kernel", ["plain", "persistent"])
def test_isochrone_df64_parity_gate(kernel):
    ensure_built()
    e = W.isochrone(n=4096, seed=0)
    ref = oracle_solve(e)
    g = gpu_solve(e, precision="df64", kernel=kernel)
    assert np.all(g["status"] == 0)
    err = rel_err(g["y"], ref["y"])
    assert err.max() <= 1e-9, err.max()
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"])
    assert same.mean() >= 0.95


def test_precession_df64_meets_angle_budget():
    ensure_built()
    e = W.precession(n=4096, seed=2001)
    g = gpu_solve(e, precision="df64", kernel="persistent")
    g64 = gpu_solve(e, precision="fp64", kernel="persistent")
    ok = g["status"] == 0
    assert np.array_equal(g["status"], g64["status"])
    idx = np.nonzero(ok)[0][:256]
    sub = e.subset(idx)
    ref = O.solve("precession", sub.y0, sub.params, sub.t0, sub.t1, sub.saveat, 1e-12, 1e-12, method="vern7")
    err = M.precession_error(g["y"][idx, -1], ref["y"][:, -1])
    assert M.accepted(err, 2e-7), M.p99(err)
    diff = M.precession_error(g["y"][ok, -1], g64["y"][ok, -1])
    assert np.percentile(diff, 99) < 2e-8


@pytest.mark.parametrize("system,gen,method", [
    ("isochrone", lambda: W.isochrone(n=128, seed=91), "tsit5"),
    ("precession", lambda: W.precession(n=128, seed=92, method="vern7", paper_interval=True), "vern7"),
    ("loghalo", lambda: W.loghalo(n=128, seed=93, rtol=1e-10), "dopri5"),
])
def test_df64_adjoint_equals_oracle_sensitivities(system, gen, method):
    ensure_built()
    e = gen()
    e.method = method
    rtol = 1e-10 if system != "precession" else 3.16e-9
    rng = np.random.default_rng(5)
    w = rng.normal(size=(e.n, e.saveat.shape[-1], e.y0.shape[1]))
    g = gpu_vjp(e, w, precision="df64", kernel="persistent", rtol=rtol, atol=rtol)
    ref = O.grad(system, e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=rtol, atol=rtol, method=method)
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"]) & (g["status"] == 0)
    assert same.mean() >= 0.9
    gy = np.concatenate([g["dLdy0"], g["dLdparams"]], axis=1)[same]
    ry = np.concatenate([ref["dLdy0"], ref["dLdparams"]], axis=1)[same]
    rel = np.linalg.norm(gy - ry, axis=1) / np.linalg.norm(ry, axis=1)
    assert rel.max() <= 1e-8, rel.max()


def test_df64_rejected_where_not_available():
    ensure_built()
    dev = torch.device("cuda")
    e = W.mw(n=16, seed=3)
    with pytest.raises(_abi.GsError):
        api.solve("mw", torch.as_tensor(e.y0, device=dev), e.params, e.t0, e.t1, e.saveat, 1e-8, 1e-8,
                  precision="df64")
    q = W.quintessence(n=16, seed=4)
    with pytest.raises(_abi.GsError):
        api.solve("quintessence", torch.as_tensor(q.y0, device=dev), q.params, q.t0, q.t1, q.saveat, 1e-6, 1e-9,
                  precision="df64")
    i = W.isochrone(n=16, seed=5)
    with pytest.raises(_abi.GsError):
        api.jvp("isochrone", torch.as_tensor(i.y0, device=dev), None, i.t0, i.t1, i.saveat, 1e-8, 1e-8,
                dy0=np.ones((16, 6, 1)), precision="df64")
