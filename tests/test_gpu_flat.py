"""gs_solve_flat (Sec. 4.1, Eqs. de-flat and de-ift) against the oracle's flatness shooting.

* FP64: the Newton iterates, the solution, da0/dOm and dy/dOm along the flat models agree with the
  oracle run at the same tolerance (same algorithm; Newton started from the paper's 1 - Om - Or).
* FP32-pair mode at the dark-energy tolerance: the distances D_M, D_H of the flat models meet the
  1e-4 c/H0 budget of Sec. 4.2 against a converged FP64 oracle solve, and a0 agrees to 10 rtol.
* Special cases: lambda = 0 needs no Newton step and gives a0 = 1 - Om - Or; one allowed step
  leaves moving fields unconverged; a last output that is not today is flagged.
"""
import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from oracle import flat as OF
from paper_2609_28458_gb300 import _abi, api
from paper_2609_28458_gb300 import metrics as M
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ens(n, seed, rtol, dense=False):
    e = W.quintessence(n=n, seed=seed, rtol=rtol, dense=dense)
    e.params[:, 0] = 1.0 - e.params[:, 2] - e.params[:, 3]   # the paper's Newton start
    return e


def _gpu(e, precision, rtol, atol, **kw):
    dev = torch.device("cuda")
    r = api.solve_flat(torch.as_tensor(e.y0, device=dev), e.params, e.t0, e.t1, e.saveat, rtol, atol,
                       method=e.method, precision=precision, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def _dist(y, params, saveat):
    dm, dh = M.distances(y, params, saveat)
    return dm, dh


def test_flat_fp64_matches_oracle():
    ensure_built()
    e = _ens(96, 71, 1e-10)
    e.params[:8, 1] = 0.0   # a few cosmological constants
    rtol, atol, gtol = 1e-10, 1e-13, 1e-11
    g = _gpu(e, "fp64", rtol, atol, gtol=gtol, max_newton=10)
    o = OF.solve_flat(e.y0, e.params, e.t0, e.t1, e.saveat, rtol, atol, method="tsit5", max_newton=10, gtol=gtol)
    assert np.all(g["status"] == 0) and np.all(o["converged"])
    assert np.all(g["n_newton"] <= 6)
    assert np.mean(g["n_newton"] == o["n_newton"]) >= 0.9
    assert np.max(np.abs(g["a0"] - o["a0"])) <= 1e-9
    assert np.max(np.abs(g["g"])) <= gtol
    assert np.max(np.abs(g["y"] - o["y"])) <= 1e-8
    assert np.max(np.abs(g["da0dOm"] - o["da0dOm"]) / np.abs(o["da0dOm"])) <= 1e-7
    assert np.max(np.abs(g["dydOm"] - o["dydOm"])) <= 1e-7 * np.max(np.abs(o["dydOm"]))
    # lambda = 0: the start is the root
    assert np.all(g["n_newton"][:8] == 1)
    assert np.allclose(g["a0"][:8], 1.0 - e.params[:8, 2] - e.params[:8, 3], rtol=0, atol=1e-15)
    assert np.allclose(g["da0dOm"][:8], -1.0, rtol=0, atol=1e-10)


@pytest.mark.parametrize("method", ["tsit5", "dopri5"])
def test_flat_fp32df_distances_meet_budget(method):
    ensure_built()
    e = _ens(2048, 72, 1e-6)
    e.method = method
    # FP32 stages make g(a0) rough at the 1e-7 level, so the residual is asked down to rtol only
    g = _gpu(e, "fp32df", 1e-6, 1e-9, gtol=1e-6)
    ref = OF.solve_flat(e.y0, e.params, e.t0, e.t1, e.saveat, 1e-12, 1e-15, method="vern7", gtol=1e-13)
    assert np.all(g["status"] == 0), np.unique(g["status"], return_counts=True)
    assert np.all(ref["converged"])
    # the root of the integrated g carries the integration error (rtol 1e-6) into a0
    assert np.max(np.abs(g["a0"] - ref["a0"])) <= 1e-5
    pg = e.params.copy(); pg[:, 0] = g["a0"]
    pr = e.params.copy(); pr[:, 0] = ref["a0"]
    dm, dh = _dist(g["y"], pg, e.saveat)
    dmr, dhr = _dist(ref["y"], pr, e.saveat)
    err = np.maximum(np.abs(dm - dmr).max(1), np.abs(dh - dhr).max(1))
    assert M.accepted(err, 1e-4), M.p99(err)
    # the derivative along flat models, to the same relative level
    assert np.max(np.abs(g["dydOm"] - ref["dydOm"])) <= 1e-3 * np.max(np.abs(ref["dydOm"]))


def test_flat_newton_limits_and_flags():
    ensure_built()
    e = _ens(64, 73, 1e-8)
    e.params[:16, 1] = 0.0
    g = _gpu(e, "fp64", 1e-8, 1e-11, gtol=1e-10, max_newton=1)
    moving = e.params[:, 1] > 0.3
    assert np.all(g["n_newton"] == 1)
    assert np.all((g["status"][:16] & _abi.ST_NO_CONVERGENCE) == 0)
    assert np.all((g["status"][moving] & _abi.ST_NO_CONVERGENCE) != 0)
    assert np.all(np.isfinite(g["y"]))
    # the last output must be today: otherwise flagged, derivatives NaN
    e2 = _ens(8, 74, 1e-8)
    e2.saveat = e2.saveat[:-1]
    g2 = _gpu(e2, "fp64", 1e-8, 1e-11)
    assert np.all((g2["status"] & _abi.ST_NO_CONVERGENCE) != 0)
    assert np.all(np.isnan(g2["dydOm"])) and np.all(g2["n_newton"] == 1)


def test_flat_rejects_bad_arguments():
    ensure_built()
    e = _ens(4, 75, 1e-6)
    with pytest.raises(_abi.GsError):
        _gpu(e, "fp32", 1e-6, 1e-9)            # gs_jvp runs in FP64 or the FP32-pair mode
    with pytest.raises(_abi.GsError):
        _gpu(e, "fp64", 1e-6, 1e-9, gtol=0.0)
    with pytest.raises(_abi.GsError):
        _gpu(e, "fp64", 1e-6, 1e-9, max_newton=0)
