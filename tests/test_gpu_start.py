"""Prepared starts of the persistent forward (k_start): with a workspace that holds the start rows
(gs_workspace_bytes), every trajectory of the launch is started by a one-thread-per-trajectory pass
and the persistent kernel loads its row; with a workspace of only the 256-byte counter header it
starts trajectories in place. Both run the same start-up (Traj::init) and the same attempts, in
different kernels, so:
- trajectories that start-up already finishes (empty interval, non-finite input, outputs outside
  [t0, t1]) get the same status, counts and outputs bit for bit;
- FP64: step counts agree for nearly every member (the compiler may fuse multiply-adds differently
  in different kernels) and outputs to rounding;
- FP32 modes: step counts agree on average and outputs within the orbit budget (borderline accept
  tests may flip with a different fusion of the FP32 error estimate).
The ensemble is below the size at which the automatic longest-first order starts (32,768), so both
launches take trajectories in stored order."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import ensure_built, rel_err
from paper_2609_28458_gb300 import _abi
from paper_2609_28458_gb300 import metrics as M
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _solve(e, precision, ws_bytes):
    """gs_solve through the C ABI with a workspace of ws_bytes (None: gs_workspace_bytes)."""
    ensure_built()
    dev = torch.device("cuda")
    d, p = _abi.dims(e.system)
    N, K = e.n, e.saveat.shape[-1]
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    y0, pr, t0, t1, sv = T(e.y0), T(e.params) if p else None, T(e.t0), T(e.t1), T(e.saveat)
    opt = _abi.options(e.method, precision, "persistent", per_traj_saveat=int(e.saveat.ndim == 2))
    L = _abi.lib()
    full = L.gs_workspace_bytes(_abi.SYSTEMS[e.system], N, K, ctypes.byref(opt), 0, 0.0)
    nb = full if ws_bytes is None else ws_bytes
    ws = torch.zeros(max(nb, 256) // 8 + 32, dtype=torch.float64, device=dev)
    y = torch.full((N, K, d), 7.0, dtype=torch.float64, device=dev)
    st, na, nr = (torch.full((N,), -5, dtype=torch.int32, device=dev) for _ in range(3))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.gs_solve(_abi.SYSTEMS[e.system], N, _p(y0), _p(pr), _p(t0), _p(t1), e.rtol, e.atol, K, _p(sv),
                    ctypes.byref(opt), _p(y), _p(st), _p(na), _p(nr), _p(ws), nb, stream)
    _abi.check(rc)
    torch.cuda.synchronize()
    return dict(y=y.cpu().numpy(), status=st.cpu().numpy(), n_accept=na.cpu().numpy(), n_reject=nr.cpu().numpy()), full


def _with_finished_members(e):
    """Some members that start-up finishes: an empty interval, a non-finite state, a reversed one."""
    e.t0 = np.broadcast_to(np.asarray(e.t0, dtype=np.float64), (e.n,)).copy()
    e.t1 = np.broadcast_to(np.asarray(e.t1, dtype=np.float64), (e.n,)).copy()
    e.y0 = np.array(e.y0, dtype=np.float64).copy()
    e.t1[3] = e.t0[3]
    e.y0[5, 2] = np.nan
    e.t1[7] = -1.0
    return e


@pytest.mark.parametrize("system,gen,precision", [
    ("mw", lambda: W.mw(n=3000, seed=301, t1=800.0), "fp64"),
    ("mw", lambda: W.mw(n=3000, seed=302, t1=800.0), "fp32"),
    ("mw", lambda: W.mw(n=3000, seed=303, t1=800.0), "fp32df"),
    ("isochrone", lambda: W.isochrone(n=2000, seed=304), "fp64"),
    ("precession", lambda: W.precession(n=1000, seed=305), "fp64"),
])
def test_prepared_starts_match_starts_in_place(system, gen, precision):
    e = _with_finished_members(gen())
    a, full = _solve(e, precision, None)
    b, _ = _solve(e, precision, 256)
    assert full > 256 * 1024  # the start rows are part of the workspace
    assert np.array_equal(a["status"], b["status"])
    done = (a["status"] & (_abi.ST_FAILED | _abi.ST_EMPTY_INTERVAL)) != 0
    assert done[[3, 5, 7]].all()
    for k in ("status", "n_accept", "n_reject"):
        assert np.array_equal(a[k][done], b[k][done]), k
    assert np.array_equal(a["y"][done], b["y"][done], equal_nan=True)
    live = ~done
    same = (a["n_accept"] == b["n_accept"]) & (a["n_reject"] == b["n_reject"]) & live
    if precision == "fp64":
        assert same.sum() >= 0.95 * live.sum()
        assert rel_err(a["y"][same], b["y"][same]).max() <= 1e-10
    else:
        assert abs(a["n_accept"][live].mean() / b["n_accept"][live].mean() - 1) < 0.02
        rE, vE = M.orbit_scales("mw", e.y0[live], e.params[live])
        err = M.orbit_error(a["y"][live][:, -1], b["y"][live][:, -1], rE, vE)
        assert M.p99(err) <= 1e-4, M.p99(err)
