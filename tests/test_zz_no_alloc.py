"""gs_vjp_noalloc, the gradient entry point for callers that cannot allocate device memory (code in a
framework whose memory pool forbids foreign allocations, plug-ins whose host owns every device
allocation). Its scratch is a fixed array inside the library; the test calls it through the C ABI and
checks its outputs against gs_vjp with a caller workspace, on two calls in a row (the array keeps the
previous call's contents, which the call must not depend on). Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from paper_2609_28458_gb300 import _abi, api
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _noalloc(e, w, method, precision):
    dev = torch.device("cuda")
    d, p = _abi.dims(e.system)
    N, K = e.n, e.saveat.shape[-1]
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    y0, pr, t0, t1, sv, wt = T(e.y0), T(e.params) if p else None, T(e.t0), T(e.t1), T(e.saveat), T(w)
    out = dict(dLdy0=torch.empty((N, d), dtype=torch.float64, device=dev),
               dLdparams=torch.empty((N, p), dtype=torch.float64, device=dev),
               y=torch.empty((N, K, d), dtype=torch.float64, device=dev),
               status=torch.empty(N, dtype=torch.int32, device=dev),
               n_accept=torch.empty(N, dtype=torch.int32, device=dev),
               n_reject=torch.empty(N, dtype=torch.int32, device=dev))
    opt = _abi.options(method, precision, "persistent", per_traj_saveat=int(e.saveat.ndim == 2))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _abi.lib().gs_vjp_noalloc(_abi.SYSTEMS[e.system], N, _p(y0), _p(pr), _p(t0), _p(t1), e.rtol, e.atol, K, _p(sv),
                                   ctypes.byref(opt), _p(wt), _p(out["dLdy0"]), _p(out["dLdparams"]), _p(out["y"]),
                                   _p(out["status"]), _p(out["n_accept"]), _p(out["n_reject"]), stream)
    _abi.check(rc)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _with_workspace(e, w, method, precision):
    dev = torch.device("cuda")
    r = api.vjp(e.system, torch.as_tensor(e.y0, device=dev), e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol,
                torch.as_tensor(w, device=dev), method=method, precision=precision, kernel="persistent")
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


CASES = [
    ("mw", lambda: W.mw(n=256, seed=61, t1=1000.0, rtol=1e-8), "tsit5", "fp64"),
    ("mw", lambda: W.mw(n=512, seed=62, t1=3000.0, rtol=1e-8), "tsit5", "fp32df"),
    ("quintessence", lambda: W.quintessence(n=1024, seed=63, rtol=1e-6), "dopri5", "fp32"),
]


@pytest.mark.parametrize("system,gen,method,precision", CASES)
def test_noalloc_matches_workspace_vjp_on_two_calls(system, gen, method, precision):
    ensure_built()
    e = gen()
    d, _ = _abi.dims(system)
    w = np.random.default_rng(8).normal(size=(e.n, e.saveat.shape[-1], d))
    ref = _with_workspace(e, w, method, precision)
    assert np.all((ref["status"] & _abi.ST_FAILED) == 0)
    for _ in range(2):
        got = _noalloc(e, w, method, precision)
        assert np.array_equal(got["status"], ref["status"])
        assert np.array_equal(got["n_accept"], ref["n_accept"]) and np.array_equal(got["n_reject"], ref["n_reject"])
        assert _rel(got["y"], ref["y"]) <= 1e-12
        assert _rel(got["dLdy0"], ref["dLdy0"]) <= 1e-12
        assert _rel(got["dLdparams"], ref["dLdparams"]) <= 1e-12


def test_noalloc_rejects_ensembles_beyond_its_scratch():
    ensure_built()
    opt = _abi.options()
    fake = ctypes.c_void_p(256)
    n = _abi.NOALLOC_SCRATCH_BYTES // 8 + 1  # per-trajectory bookkeeping alone exceeds the array
    rc = _abi.lib().gs_vjp_noalloc(1, n, fake, fake, fake, fake, 1e-6, 1e-6, 1, fake, ctypes.byref(opt), fake, fake,
                                   fake, fake, fake, fake, fake, None)
    assert rc == _abi.GS_ERR_WORKSPACE
    assert "built-in scratch" in _abi.lib().gs_last_error().decode()


def test_noalloc_limit_is_exactly_gs_vjps():
    """The largest ensemble the built-in scratch accepts is the one whose part before the tape pool
    plus one tape chunk fits it, as gs_vjp would require of a workspace of that size: the call just
    inside the limit runs (every trajectory has an empty interval, so no tape is needed), the next size
    is refused before any launch."""
    ensure_built()
    L = _abi.lib()
    opt = _abi.options(kernel="persistent")
    chunk = L.gs_tape_chunk_bytes(1, ctypes.byref(opt))

    def need(n):
        return L.gs_workspace_bytes(1, n, 1, ctypes.byref(opt), 1, 0.0) + chunk

    lo, hi = 1, _abi.NOALLOC_SCRATCH_BYTES
    while hi - lo > 1:  # largest n with need(n) <= the scratch
        mid = (lo + hi) // 2
        if need(mid) <= _abi.NOALLOC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid
    n_in, n_out = lo, hi
    dev = torch.device("cuda")
    f64 = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=dev)
    i32 = lambda n: torch.zeros(n, dtype=torch.int32, device=dev)
    y0, pr, t0, t1, sv, w = f64(n_out, 6), f64(n_out, 4), f64(n_out), f64(n_out), f64(1), f64(n_out, 1, 6)
    pr[:, :3] = 1.0
    pr[:, 3] = 1.0
    gy, gp, y = f64(n_out, 6), f64(n_out, 4), f64(n_out, 1, 6)
    st, na, nr = i32(n_out), i32(n_out), i32(n_out)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(n):
        return L.gs_vjp_noalloc(1, n, _p(y0), _p(pr), _p(t0), _p(t1), 1e-6, 1e-6, 1, _p(sv), ctypes.byref(opt), _p(w),
                                _p(gy), _p(gp), _p(y), _p(st), _p(na), _p(nr), stream)

    assert call(n_out) == _abi.GS_ERR_WORKSPACE
    assert call(n_in) == _abi.GS_OK
    torch.cuda.synchronize()
    assert bool((st[:n_in] == _abi.ST_EMPTY_INTERVAL).all())
