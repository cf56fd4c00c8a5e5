"""Forward sensitivities on the GPU (gs_jvp; Sec. 2.3, Eq. sens; Appendix A, Eq. stage-sens).

* Duality with the adjoint and with the oracle: for a cotangent w and a direction v = (dy0, dtheta),
  sum_k w_k . S(t_k) v = <dL/dy0, dy0> + <dL/dtheta, dtheta>. The oracle's dual-number sensitivities
  and gs_vjp give the right side; on trajectories whose step sequence is the same, the two sides
  agree to rounding (1e-8 relative).
* The value part of gs_jvp is the solve (same steps as gs_solve).
* FP32-pair mode against FP64 at the orbit-gradient budget (1e-3).
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ensure_built
from paper_2609_28458_gb300 import api
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("mw", lambda: W.mw(n=128, seed=101, t1=800.0, rtol=1e-9), "tsit5", 10),   # 4 + 4 + 2 directions
    ("mw", lambda: W.mw(n=64, seed=102, t1=500.0, rtol=1e-9), "vern7", 3),     # one direction per launch
    ("isochrone", lambda: W.isochrone(n=128, seed=103), "dopri5", 3),        # 11 dense outputs
    ("quintessence", lambda: W.quintessence(n=256, seed=104, rtol=1e-9, dense=True), "tsit5", 4),
    ("precession", lambda: W.precession(n=64, seed=105, paper_interval=True, rtol=1e-9), "tsit5", 5),
    ("loghalo", lambda: W.loghalo(n=128, seed=106, rtol=1e-9), "tsit5", 2),
]


def _directions(e, m, rng):
    d, p = e.y0.shape[1], e.params.shape[1]
    dy0 = rng.normal(size=(e.n, d, m))
    dp = rng.normal(size=(e.n, p, m)) * (np.abs(e.params)[:, :, None] + 1e-3) if p else None
    return dy0, dp


@pytest.mark.parametrize("system,gen,method,m", CASES)
def test_jvp_duality_with_oracle_and_adjoint(system, gen, method, m):
    ensure_built()
    e = gen()
    rng = np.random.default_rng(11)
    d, p = O.dims(system)
    K = e.saveat.shape[-1]
    dy0, dp = _directions(e, m, rng)
    dev = torch.device("cuda")
    j = api.jvp(system, torch.as_tensor(e.y0, device=dev), e.params if p else None, e.t0, e.t1, e.saveat, e.rtol,
                e.atol, dy0=dy0, dparams=dp, method=method)
    torch.cuda.synchronize()
    y, S = j["y"].cpu().numpy(), j["S"].cpu().numpy()
    w = rng.normal(size=(e.n, K, d))
    lhs = np.einsum("nkd,nkdm->nm", w, S)
    ref = O.grad(system, e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=e.rtol, atol=e.atol, method=method)
    rhs = np.einsum("nd,ndm->nm", ref["dLdy0"], dy0) + (np.einsum("np,npm->nm", ref["dLdparams"], dp) if p else 0)
    same = (j["n_accept"].cpu().numpy() == ref["n_accept"]) & (j["n_reject"].cpu().numpy() == ref["n_reject"])
    assert np.array_equal(j["status"].cpu().numpy(), ref["status"])
    assert same.mean() >= 0.9
    scale = np.abs(rhs).max(axis=1) + 1e-300
    rel = np.abs(lhs - rhs).max(axis=1) / scale
    assert rel[same].max() <= 1e-8, rel[same].max()
    # value part = the solve
    s = api.solve(system, torch.as_tensor(e.y0, device=dev), e.params if p else None, e.t0, e.t1, e.saveat, e.rtol,
                  e.atol, method=method, kernel="persistent")
    ys = s["y"].cpu().numpy()
    same2 = (s["n_accept"].cpu().numpy() == j["n_accept"].cpu().numpy())
    err = np.max(np.abs(y - ys).reshape(e.n, -1), axis=1) / (np.abs(ys).reshape(e.n, -1).max(axis=1) + 1e-300)
    assert err[same2].max() <= 1e-10
    # and the adjoint gives the same contraction
    g = api.vjp(system, torch.as_tensor(e.y0, device=dev), e.params if p else None, e.t0, e.t1, e.saveat, e.rtol,
                e.atol, torch.as_tensor(w, device=dev), method=method, kernel="persistent")
    gy0, gp = g["dLdy0"].cpu().numpy(), g["dLdparams"].cpu().numpy()
    rhs2 = np.einsum("nd,ndm->nm", gy0, dy0) + (np.einsum("np,npm->nm", gp, dp) if p else 0)
    same3 = same2 & (g["n_accept"].cpu().numpy() == j["n_accept"].cpu().numpy())
    rel2 = np.abs(lhs - rhs2).max(axis=1) / (np.abs(rhs2).max(axis=1) + 1e-300)
    assert rel2[same3].max() <= 1e-8, rel2[same3].max()


def test_jvp_fp32df_meets_sensitivity_budget():
    """dy(t1)/dtheta of 3 Gyr MW orbits with the FP32-pair mode at rtol 1e-8, against FP64 at 1e-11,
    in the scaled Frobenius measure of Eq. st-graderr (budget 1e-3)."""
    from paper_2609_28458_gb300 import metrics as M

    ensure_built()
    e = W.mw(n=2048, seed=107, rtol=1e-8)
    dev = torch.device("cuda")
    dp = np.zeros((e.n, 4, 4))
    for q in range(4):
        dp[:, q, q] = 1.0
    a = api.jvp("mw", torch.as_tensor(e.y0, device=dev), e.params, e.t0, e.t1, e.saveat, 1e-8, 1e-8, dparams=dp,
                precision="fp32df")
    b = api.jvp("mw", torch.as_tensor(e.y0, device=dev), e.params, e.t0, e.t1, e.saveat, 1e-11, 1e-11, dparams=dp,
                precision="fp64")
    Sa, Sb = a["S"][:, -1].cpu().numpy(), b["S"][:, -1].cpu().numpy()
    rE, vE = M.orbit_scales("mw", e.y0, e.params)
    err = M.sensitivity_error(Sa, Sb, rE, vE, e.params)
    assert M.accepted(err, 1e-3), M.p99(err)


def test_jvp_empty_interval_and_t0_outputs_carry_the_seed():
    ensure_built()
    e = W.precession(n=64, seed=108)
    dev = torch.device("cuda")
    dy0 = np.random.default_rng(2).normal(size=(e.n, 9, 2))
    j = api.jvp("precession", torch.as_tensor(e.y0, device=dev), e.params, e.t0, e.t1, e.saveat, 1e-8, 1e-8, dy0=dy0,
                method="vern7")
    st = j["status"].cpu().numpy()
    empty = (st & O.ST_EMPTY_INTERVAL) != 0
    assert empty.any()
    assert np.array_equal(j["S"].cpu().numpy()[empty, 0], dy0[empty])
