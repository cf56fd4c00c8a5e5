"""CPU oracle for the ensemble Runge-Kutta path (TEST INFRASTRUCTURE).

A plain, slow FP64 restatement of the paper's method (Sec. 2.1-2.3, Appendix A: Eqs. ivp, rk,
errnorm, controller, dense, sens, stage-sens, chain), written in C++ in ``oracle.cpp`` and
called here through ctypes on NumPy arrays. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the product path never does, and it
shares no code with the GPU library.

Every function here is argument marshalling; the arithmetic is in the C++ source, which cites
the passage each step follows.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SYSTEMS = {"isochrone": 0, "mw": 1, "precession": 2, "quintessence": 3, "loghalo": 4,
           "linear": 5}  # linear: the test equation y' = lambda y (tests of the controller only)
METHODS = {"tsit5": 0, "dopri5": 1, "vern7": 2}
ST_MAX_STEPS, ST_H_UNDERFLOW, ST_NONFINITE, ST_EMPTY_INTERVAL, ST_SAVEAT_OUTSIDE = 1, 2, 4, 8, 16

_lib = None


class _Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("max_steps", ctypes.c_int), ("safety", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("h0", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _sys(s):
    return SYSTEMS[s] if isinstance(s, str) else int(s)


def _meth(m):
    return METHODS[m] if isinstance(m, str) else int(m)


def opts(method="tsit5", max_steps=1_000_000, safety=0.9, alpha_min=0.2, alpha_max=5.0, beta1=0.0,
         beta2=0.0, h0=0.0):
    """Controller options; beta1 = 0 selects 1/nu (Eq. controller)."""
    return _Opts(_meth(method), int(max_steps), safety, alpha_min, alpha_max, beta1, beta2, h0)


def dims(system):
    d, p = ctypes.c_int(), ctypes.c_int()
    lib().orc_dims(_sys(system), ctypes.byref(d), ctypes.byref(p))
    return d.value, p.value


def max_threads():
    return lib().orc_max_threads()


def tableau(method):
    s, o, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    A = np.zeros(100); b = np.zeros(10); bh = np.zeros(10); c = np.zeros(10)
    lib().orc_tableau(_meth(method), ctypes.byref(s), ctypes.byref(o), ctypes.byref(f), _p(A), _p(b),
                      _p(bh), _p(c))
    n = s.value
    return dict(s=n, order=o.value, fsal=bool(f.value), A=A[: n * n].reshape(n, n).copy(), b=b[:n].copy(),
                bh=bh[:n].copy(), c=c[:n].copy())


def dense_weights(method, sigma):
    w = np.zeros(10)
    rc = lib().orc_dense_weights(_meth(method), ctypes.c_double(sigma), _p(w))
    if rc != 0:
        raise ValueError("no dense-output polynomial for this method")
    return w[: tableau(method)["s"]]


def rhs(system, t, y, p=None):
    d, np_ = dims(system)
    y = np.ascontiguousarray(y, dtype=np.float64)
    p = np.ascontiguousarray(p if p is not None else np.zeros(max(np_, 1)), dtype=np.float64)
    f = np.zeros(d)
    lib().orc_rhs(_sys(system), ctypes.c_double(t), _p(y), _p(p), _p(f))
    return f


def initial_step(system, method, t0, t1, y0, p=None, rtol=1e-6, atol=1e-6):
    """The starting step a solve of `method` takes from (t0, y0) towards t1 (HNW I, Sec. II.4)."""
    d, np_ = dims(system)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    p = np.ascontiguousarray(p if p is not None else np.zeros(max(np_, 1)), dtype=np.float64)
    f = lib().orc_initial_step
    f.restype = ctypes.c_double
    return f(_sys(system), _meth(method), ctypes.c_double(t0), ctypes.c_double(t1), _p(y0), _p(p),
             ctypes.c_double(rtol), ctypes.c_double(atol))


def jvp(system, t, y, p, vy, vp=None):
    d, np_ = dims(system)
    y = np.ascontiguousarray(y, dtype=np.float64)
    p = np.ascontiguousarray(p if p is not None else np.zeros(max(np_, 1)), dtype=np.float64)
    vy = np.ascontiguousarray(vy, dtype=np.float64)
    vp = np.ascontiguousarray(vp if vp is not None else np.zeros(max(np_, 1)), dtype=np.float64)
    out = np.zeros(d)
    lib().orc_jvp(_sys(system), ctypes.c_double(t), _p(y), _p(p), _p(vy), _p(vp), _p(out))
    return out


def potential(system, x, p=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p if p is not None else np.zeros(4), dtype=np.float64)
    phi = ctypes.c_double()
    lib().orc_potential(_sys(system), _p(x), _p(p), ctypes.byref(phi))
    return phi.value


def _prep(system, y0, params, t0, t1, saveat):
    d, np_ = dims(system)
    y0 = np.ascontiguousarray(y0, dtype=np.float64).reshape(-1, d)
    N = y0.shape[0]
    params = (np.ascontiguousarray(params, dtype=np.float64).reshape(N, np_) if np_ else np.zeros((N, 1)))
    t0 = np.ascontiguousarray(np.broadcast_to(np.asarray(t0, dtype=np.float64), (N,)))
    t1 = np.ascontiguousarray(np.broadcast_to(np.asarray(t1, dtype=np.float64), (N,)))
    saveat = np.ascontiguousarray(saveat, dtype=np.float64)
    per_traj = 1 if saveat.ndim == 2 else 0
    K = saveat.shape[-1]
    return d, np_, N, y0, params, t0, t1, saveat, per_traj, K


def solve(system, y0, params, t0, t1, saveat, rtol, atol, method="tsit5", record=False, tape_cap=1 << 16,
          nthreads=0, **kw):
    """Adaptive solve (same-algorithm mode). Returns dict with y [N,K,d], status, n_accept, n_reject
    and, if record, the accepted step sizes tape [N, tape_cap] with counts ntape [N]."""
    d, np_, N, y0, params, t0, t1, saveat, per_traj, K = _prep(system, y0, params, t0, t1, saveat)
    o = opts(method, **kw)
    y = np.empty((N, K, d))
    st = np.zeros(N, np.int32); na = np.zeros(N, np.int32); nr = np.zeros(N, np.int32)
    tape = np.zeros((N, tape_cap)) if record else None
    nt = np.zeros(N, np.int32) if record else None
    lib().orc_solve(_sys(system), ctypes.byref(o), ctypes.c_long(N), _p(y0), _p(params), _p(t0), _p(t1),
                    ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_int(K), _p(saveat),
                    ctypes.c_int(per_traj), _p(y), _p(st), _p(na), _p(nr), _p(tape), ctypes.c_int(tape_cap),
                    _p(nt), ctypes.c_int(nthreads))
    out = dict(y=y, status=st, n_accept=na, n_reject=nr)
    if record:
        out["tape"] = tape
        out["ntape"] = nt
    return out


def replay(system, y0, params, t0, t1, saveat, tape, ntape, method="tsit5", nthreads=0):
    """Fixed-step replay of recorded step sizes (no error control)."""
    d, np_, N, y0, params, t0, t1, saveat, per_traj, K = _prep(system, y0, params, t0, t1, saveat)
    o = opts(method)
    tape = np.ascontiguousarray(tape, dtype=np.float64).reshape(N, -1)
    ntape = np.ascontiguousarray(ntape, dtype=np.int32)
    y = np.empty((N, K, d))
    lib().orc_replay(_sys(system), ctypes.byref(o), ctypes.c_long(N), _p(y0), _p(params), _p(t0), _p(t1),
                     ctypes.c_int(K), _p(saveat), ctypes.c_int(per_traj), _p(tape), ctypes.c_int(tape.shape[1]),
                     _p(ntape), _p(y), ctypes.c_int(nthreads))
    return y


def grad(system, y0, params, t0, t1, saveat, w, rtol=0.0, atol=0.0, method="tsit5", tape=None, ntape=None,
         nthreads=0, **kw):
    """Gradient of L = sum_k w[n,k,:] . y_n(t_k) per member by forward sensitivities (Eq. sens,
    Eq. stage-sens, Eq. chain). Along the adaptive step sequence, or along a recorded tape."""
    d, np_, N, y0, params, t0, t1, saveat, per_traj, K = _prep(system, y0, params, t0, t1, saveat)
    o = opts(method, **kw)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(N, K, d)
    y = np.empty((N, K, d)); gy0 = np.empty((N, d)); gp = np.empty((N, max(np_, 1)))
    st = np.zeros(N, np.int32); na = np.zeros(N, np.int32); nr = np.zeros(N, np.int32)
    tcap = 0
    if tape is not None:
        tape = np.ascontiguousarray(tape, dtype=np.float64).reshape(N, -1)
        ntape = np.ascontiguousarray(ntape, dtype=np.int32)
        tcap = tape.shape[1]
    lib().orc_grad(_sys(system), ctypes.byref(o), ctypes.c_long(N), _p(y0), _p(params), _p(t0), _p(t1),
                   ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_int(K), _p(saveat),
                   ctypes.c_int(per_traj), _p(w), _p(y), _p(gy0), _p(gp), _p(st), _p(na), _p(nr), _p(tape),
                   ctypes.c_int(tcap), _p(ntape), ctypes.c_int(nthreads))
    return dict(y=y, dLdy0=gy0, dLdparams=gp[:, :np_], status=st, n_accept=na, n_reject=nr)


def sens(system, y0, params, t0, t1, saveat, rtol, atol, method="tsit5", nthreads=0, **kw):
    """Solution and full forward-sensitivity matrix S [N, K, d, d + p]: derivatives of y(t_k) with
    respect to (y0, theta) along the adaptive step sequence (Eq. sens, Eq. stage-sens)."""
    d, np_, N, y0, params, t0, t1, saveat, per_traj, K = _prep(system, y0, params, t0, t1, saveat)
    o = opts(method, **kw)
    y = np.empty((N, K, d)); S = np.empty((N, K, d, d + np_))
    st = np.zeros(N, np.int32); na = np.zeros(N, np.int32); nr = np.zeros(N, np.int32)
    lib().orc_sens(_sys(system), ctypes.byref(o), ctypes.c_long(N), _p(y0), _p(params), _p(t0), _p(t1),
                   ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_int(K), _p(saveat), ctypes.c_int(per_traj),
                   _p(y), _p(S), _p(st), _p(na), _p(nr), ctypes.c_int(nthreads))
    return dict(y=y, S=S, status=st, n_accept=na, n_reject=nr)
