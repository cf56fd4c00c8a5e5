"""PyTorch-facing calls of the ensemble solver. Argument marshalling only: tensors are checked,
made contiguous FP64 on the GPU, and their device pointers are handed to libgs.so together with
the current CUDA stream. Torch provides device memory and streams; every step of the solve and of
its gradient runs in the library's kernels.
"""
import ctypes

import torch

from . import _abi

_i32 = torch.int32


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else None


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev(x, device, name):
    """FP64 contiguous copy of x on `device`. The first tensor of a call (device None) must already
    live on a CUDA device: it decides where the solve runs. Later arguments are moved there."""
    if not torch.is_tensor(x):
        x = torch.as_tensor(x, dtype=torch.float64)
    if device is None:
        if x.device.type != "cuda":
            raise ValueError("%s must be a CUDA tensor (the solver runs only on the GPU)" % name)
        device = x.device
    return x.to(device=device, dtype=torch.float64).contiguous()


def _vec(x, n, dev, name):
    """A per-trajectory FP64 vector of length n on dev from a scalar, a NumPy array or a tensor."""
    if not torch.is_tensor(x):
        x = torch.as_tensor(x, dtype=torch.float64)
    if x.dim() == 0 or x.numel() == 1:
        return torch.full((n,), float(x.reshape(-1)[0]), dtype=torch.float64, device=dev)
    return _dev(x, dev, name).reshape(n)


def _hint(kw, dev, N):
    """cost_hint as a contiguous int32 device tensor of N entries (returned so the caller keeps it alive
    for the call); the option passes its address."""
    h = kw.get("cost_hint")
    if h is None or isinstance(h, int):
        return None
    h = torch.as_tensor(h).to(device=dev, dtype=_i32).reshape(-1).contiguous()
    if h.numel() != N:
        raise ValueError("cost_hint must have one entry per trajectory")
    kw["cost_hint"] = h
    return h


def _sysid(system):
    return _abi.SYSTEMS[system] if isinstance(system, str) else int(system)


class Workspace:
    """A reusable device workspace (256-byte aligned torch allocation)."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.buf = None

    def get(self, nbytes):
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.buf

    @property
    def nbytes(self):
        return 0 if self.buf is None else self.buf.numel()


_default_ws = {}


def _ws(device, nbytes, ws):
    """Exactly `nbytes` of a (possibly larger, reused) workspace buffer."""
    if ws is None:
        ws = _default_ws.setdefault(str(device), Workspace(device))
    return ws.get(nbytes)[: int(nbytes)]


def tape_bytes(system, n, n_accept=None, steps_hint=None, opt=None, precision="fp64", K=1, ckpt_stride=None):
    """Workspace bytes for a tape: exact from per-trajectory accepted-step counts, else from a hint.
    The chunk size depends on the precision mode and checkpoint stride (of opt, else of `precision`
    and `ckpt_stride`); K (outputs per trajectory) sizes the output attribution of strides above 1."""
    if opt is None:
        opt = _abi.options(precision=precision)
        if ckpt_stride is not None:
            opt.ckpt_stride = int(ckpt_stride)
    L, sid = _abi.lib(), _sysid(system)
    if n_accept is not None:
        fixed = L.gs_workspace_bytes(sid, n, K, ctypes.byref(opt), 1, 0.0)
        chunk = L.gs_tape_chunk_bytes(sid, ctypes.byref(opt))
        chunks = int(((n_accept.to(torch.int64) + 31) // 32).sum().item()) + 1
        return fixed + chunks * chunk
    return L.gs_workspace_bytes(sid, n, K, ctypes.byref(opt), 1, float(steps_hint or 1024))


def solve(system, y0, params, t0, t1, saveat, rtol, atol, method="tsit5", precision="fp64", kernel="auto",
          workspace=None, record_tape=False, tape_nbytes=None, out=None, **kw):
    """Adaptive ensemble solve. Returns dict(y [N,K,d], status, n_accept, n_reject) on the GPU."""
    y0 = _dev(y0, None, "y0")
    dev = y0.device
    d, p = _abi.dims(system)
    N = y0.shape[0]
    y0 = y0.reshape(N, d)
    params = _dev(params, dev, "params").reshape(N, p) if p else None
    t0 = _vec(t0, N, dev, "t0")
    t1 = _vec(t1, N, dev, "t1")
    saveat = _dev(saveat, dev, "saveat")
    per_traj = saveat.dim() == 2
    K = saveat.shape[-1]
    steps_hint = kw.pop("steps_hint", 1024)
    hint = _hint(kw, dev, N)  # noqa: F841 (kept alive through the call)
    opt = _abi.options(method, precision, kernel, per_traj_saveat=int(per_traj), record_tape=int(record_tape), **kw)
    if out is None:
        out = dict(y=torch.empty((N, K, d), dtype=torch.float64, device=dev),
                   status=torch.empty(N, dtype=_i32, device=dev), n_accept=torch.empty(N, dtype=_i32, device=dev),
                   n_reject=torch.empty(N, dtype=_i32, device=dev))
    if record_tape:
        nbytes = tape_nbytes or tape_bytes(system, N, steps_hint=steps_hint, opt=opt, K=K)
    else:
        nbytes = _abi.lib().gs_workspace_bytes(_sysid(system), N, K, ctypes.byref(opt), 0, 0.0)
    wsb = _ws(dev, nbytes, workspace)
    _abi.check(_abi.lib().gs_solve(_sysid(system), N, _ptr(y0), _ptr(params), _ptr(t0), _ptr(t1), float(rtol),
                                   float(atol), K, _ptr(saveat), ctypes.byref(opt), _ptr(out["y"]),
                                   _ptr(out["status"]), _ptr(out["n_accept"]), _ptr(out["n_reject"]), _ptr(wsb),
                                   wsb.numel(), _stream(dev)))
    return out


def vjp(system, y0, params, t0, t1, saveat, rtol, atol, dLdy, method="tsit5", precision="fp64", kernel="auto",
        workspace=None, reuse_tape=None, n_accept_hint=None, tape_nbytes=None, **kw):
    """Discrete-adjoint gradient. Returns dict(dLdy0 [N,d], dLdparams [N,p], y, status, n_accept, n_reject).

    reuse_tape: the result dict of a ``solve(..., record_tape=True, workspace=workspace)`` with the
    same inputs; its tape (in `workspace`) is reversed instead of re-running the forward solve."""
    y0 = _dev(y0, None, "y0")
    dev = y0.device
    d, p = _abi.dims(system)
    N = y0.shape[0]
    y0 = y0.reshape(N, d)
    params = _dev(params, dev, "params").reshape(N, p) if p else None
    t0 = _vec(t0, N, dev, "t0")
    t1 = _vec(t1, N, dev, "t1")
    saveat = _dev(saveat, dev, "saveat")
    per_traj = saveat.dim() == 2
    K = saveat.shape[-1]
    dLdy = _dev(dLdy, dev, "dLdy").reshape(N, K, d)
    steps_hint = kw.pop("steps_hint", 1024)
    hint = _hint(kw, dev, N)  # noqa: F841 (kept alive through the call)
    opt = _abi.options(method, precision, kernel, per_traj_saveat=int(per_traj), reuse_tape=int(reuse_tape is not None),
                       **kw)
    if reuse_tape:
        if workspace is None:
            raise ValueError("reuse_tape needs the workspace the tape was recorded into")
        wsb = workspace.buf
    else:
        if tape_nbytes is None and n_accept_hint is None:
            # size the tape exactly from a forward solve with the same options (one extra solve)
            n_accept_hint = solve(system, y0, params, t0, t1, saveat, rtol, atol, method=method, precision=precision,
                                  kernel=kernel, **kw)["n_accept"]
        nbytes = tape_nbytes or tape_bytes(system, N, n_accept=n_accept_hint, steps_hint=steps_hint, opt=opt, K=K)
        wsb = _ws(dev, nbytes, workspace)
    res = dict(dLdy0=torch.empty((N, d), dtype=torch.float64, device=dev),
               dLdparams=torch.empty((N, max(p, 0)), dtype=torch.float64, device=dev))
    if reuse_tape is not None:
        res.update(y=reuse_tape["y"], status=reuse_tape["status"], n_accept=reuse_tape["n_accept"],
                   n_reject=reuse_tape["n_reject"])
    else:
        res.update(y=torch.empty((N, K, d), dtype=torch.float64, device=dev),
                   status=torch.empty(N, dtype=_i32, device=dev), n_accept=torch.empty(N, dtype=_i32, device=dev),
                   n_reject=torch.empty(N, dtype=_i32, device=dev))
    _abi.check(_abi.lib().gs_vjp(_sysid(system), N, _ptr(y0), _ptr(params), _ptr(t0), _ptr(t1), float(rtol), float(atol),
                                 K, _ptr(saveat), ctypes.byref(opt), _ptr(dLdy), _ptr(res["dLdy0"]),
                                 _ptr(res["dLdparams"]), _ptr(res["y"]), _ptr(res["status"]), _ptr(res["n_accept"]),
                                 _ptr(res["n_reject"]), _ptr(wsb), wsb.numel(), _stream(dev)))
    return res


def jvp(system, y0, params, t0, t1, saveat, rtol, atol, dy0=None, dparams=None, method="tsit5", precision="fp64",
        workspace=None, **kw):
    """Forward sensitivities along m directions (Sec. 2.3): returns dict(y [N,K,d], S [N,K,d,m], status,
    n_accept, n_reject). dy0 [N,d,m] and dparams [N,p,m] give the directions (None = 0)."""
    y0 = _dev(y0, None, "y0")
    dev = y0.device
    d, p = _abi.dims(system)
    N = y0.shape[0]
    y0 = y0.reshape(N, d)
    params = _dev(params, dev, "params").reshape(N, p) if p else None
    t0 = _vec(t0, N, dev, "t0")
    t1 = _vec(t1, N, dev, "t1")
    saveat = _dev(saveat, dev, "saveat")
    per_traj = saveat.dim() == 2
    K = saveat.shape[-1]
    dy0 = _dev(dy0, dev, "dy0") if dy0 is not None else None
    dparams = _dev(dparams, dev, "dparams") if dparams is not None else None
    m = dy0.shape[-1] if dy0 is not None else dparams.shape[-1]
    if dy0 is not None:
        dy0 = dy0.reshape(N, d, m)
    if dparams is not None:
        dparams = dparams.reshape(N, p, m)
    hint = _hint(kw, dev, N)  # noqa: F841 (kept alive through the call)
    opt = _abi.options(method, precision, "persistent", per_traj_saveat=int(per_traj), **kw)
    nbytes = _abi.lib().gs_workspace_bytes(_sysid(system), N, K, ctypes.byref(opt), 0, 0.0)
    wsb = _ws(dev, nbytes, workspace)
    out = dict(y=torch.empty((N, K, d), dtype=torch.float64, device=dev),
               S=torch.empty((N, K, d, m), dtype=torch.float64, device=dev),
               status=torch.empty(N, dtype=_i32, device=dev), n_accept=torch.empty(N, dtype=_i32, device=dev),
               n_reject=torch.empty(N, dtype=_i32, device=dev))
    _abi.check(_abi.lib().gs_jvp(_sysid(system), N, _ptr(y0), _ptr(params), _ptr(t0), _ptr(t1), float(rtol), float(atol),
                                 K, _ptr(saveat), ctypes.byref(opt), m, _ptr(dy0), _ptr(dparams), _ptr(out["y"]),
                                 _ptr(out["S"]), _ptr(out["status"]), _ptr(out["n_accept"]), _ptr(out["n_reject"]),
                                 _ptr(wsb), wsb.numel(), _stream(dev)))
    return out


def solve_flat(y0, params, t0, t1, saveat, rtol, atol, method="tsit5", precision="fp64", max_newton=8, gtol=None,
               workspace=None, **kw):
    """Quintessence cosmologies with the amplitude a0 solved from flatness (Sec. 4.1, Eqs. de-flat, de-ift).

    params [N,4] = (a0, lambda, Om, Or); its a0 column is the Newton start (not modified: a copy is
    solved). saveat must end at t1 (today). gtol defaults to rtol. Returns dict(a0 [N], params [N,4],
    y [N,K,3], dydOm [N,K,3], da0dOm [N], g [N], status, n_accept, n_reject, n_newton)."""
    y0 = _dev(y0, None, "y0")
    dev = y0.device
    N = y0.shape[0]
    y0 = y0.reshape(N, 3)
    prm = _dev(params, dev, "params").reshape(N, 4).clone()
    t0 = _vec(t0, N, dev, "t0")
    t1 = _vec(t1, N, dev, "t1")
    saveat = _dev(saveat, dev, "saveat")
    per_traj = saveat.dim() == 2
    K = saveat.shape[-1]
    opt = _abi.options(method, precision, "persistent", per_traj_saveat=int(per_traj), **kw)
    out = dict(y=torch.empty((N, K, 3), dtype=torch.float64, device=dev),
               dydOm=torch.empty((N, K, 3), dtype=torch.float64, device=dev),
               da0dOm=torch.empty(N, dtype=torch.float64, device=dev), g=torch.empty(N, dtype=torch.float64, device=dev),
               status=torch.empty(N, dtype=_i32, device=dev), n_accept=torch.empty(N, dtype=_i32, device=dev),
               n_reject=torch.empty(N, dtype=_i32, device=dev), n_newton=torch.empty(N, dtype=_i32, device=dev))
    wsb = _ws(dev, _abi.lib().gs_flat_workspace_bytes(N, K), workspace)
    gtol = float(rtol if gtol is None else gtol)
    _abi.check(_abi.lib().gs_solve_flat(N, _ptr(y0), _ptr(prm), _ptr(t0), _ptr(t1), float(rtol), float(atol), K,
                                        _ptr(saveat), ctypes.byref(opt), int(max_newton), gtol, _ptr(out["y"]),
                                        _ptr(out["dydOm"]), _ptr(out["da0dOm"]), _ptr(out["g"]), _ptr(out["status"]),
                                        _ptr(out["n_accept"]), _ptr(out["n_reject"]), _ptr(out["n_newton"]), _ptr(wsb),
                                        wsb.numel(), _stream(dev)))
    out["params"] = prm
    out["a0"] = prm[:, 0]
    return out


class ProfileData:
    """Prepared data of the profile-likelihood fits (gs_profile_prepare): node redshifts, BAO points
    with their covariance's Cholesky factor, supernova magnitudes likewise, all mock data sets."""

    def __init__(self, z_nodes, bao_z, bao_kind, L_bao, z_sn, L_sn, d_bao, d_sn, device=None):
        dev = torch.device(device or "cuda")
        t = lambda a: _dev(a, dev, "data")
        self.device = dev
        self.z_nodes, self.bao_z, self.L_bao = t(z_nodes), t(bao_z), t(L_bao)
        self.z_sn, self.L_sn = t(z_sn), t(L_sn)
        self.d_bao, self.d_sn = t(d_bao).reshape(-1, len(bao_z)), t(d_sn).reshape(-1, len(z_sn))
        self.bao_kind = torch.as_tensor(bao_kind, dtype=_i32).to(dev).contiguous()
        self.n_nodes, self.n_bao, self.n_sn = len(z_nodes), len(bao_z), len(z_sn)
        self.n_mocks = self.d_sn.shape[0]
        nbytes = _abi.lib().gs_profile_prep_bytes(self.n_nodes, self.n_bao, self.n_sn, self.n_mocks)
        if not nbytes:
            raise ValueError("unsupported profile data sizes")
        self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        _abi.check(_abi.lib().gs_profile_prepare(self.n_nodes, _ptr(self.z_nodes), self.n_bao, _ptr(self.bao_z),
                                                 _ptr(self.bao_kind), _ptr(self.L_bao), self.n_sn, _ptr(self.z_sn),
                                                 _ptr(self.L_sn), self.n_mocks, _ptr(self.d_bao), _ptr(self.d_sn),
                                                 _ptr(self.buf), self.buf.numel(), _stream(dev)))


def profile_fit(data, lam, mock, workspace=None, **opts):
    """Gauss-Newton fits (Eq. de-gn) of (Om, H0) at fixed lambda [n] on mock data sets mock [n] of a
    ProfileData. Returns dict(om, H0, a0, chi2, decrement, converged, status)."""
    dev = data.device
    lam = _dev(lam, dev, "lam").reshape(-1)
    n = lam.shape[0]
    mock = torch.as_tensor(mock, dtype=_i32).to(dev).reshape(-1).contiguous()
    o = _abi.profile_options(**opts)
    out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in ("om", "H0", "a0", "chi2", "decrement")}
    out["converged"] = torch.empty(n, dtype=_i32, device=dev)
    out["status"] = torch.empty(n, dtype=_i32, device=dev)
    wsb = _ws(dev, _abi.lib().gs_profile_workspace_bytes(n, data.n_nodes), workspace)
    _abi.check(_abi.lib().gs_profile_fit(n, _ptr(lam), _ptr(mock), _ptr(data.buf), data.n_nodes, data.n_bao,
                                         data.n_sn, data.n_mocks, ctypes.byref(o), _ptr(out["om"]), _ptr(out["H0"]),
                                         _ptr(out["a0"]), _ptr(out["chi2"]), _ptr(out["decrement"]),
                                         _ptr(out["converged"]), _ptr(out["status"]), _ptr(wsb), wsb.numel(),
                                         _stream(dev)))
    return out


def rhs(system, t, y, params=None, w=None, precision="fp64"):
    """f(t, y, theta) and, if w is given, J_y^T w and J_theta^T w, evaluated by the device code."""
    y = _dev(y, None, "y")
    dev = y.device
    d, p = _abi.dims(system)
    M = y.shape[0]
    t = _vec(t, M, dev, "t")
    params = _dev(params, dev, "params").reshape(M, p) if p else None
    f = torch.empty((M, d), dtype=torch.float64, device=dev)
    gy = gp = None
    if w is not None:
        w = _dev(w, dev, "w").reshape(M, d)
        gy = torch.empty((M, d), dtype=torch.float64, device=dev)
        gp = torch.empty((M, max(p, 1)), dtype=torch.float64, device=dev) if p else None
    _abi.check(_abi.lib().gs_rhs(_sysid(system), _abi.PRECISIONS[precision], M, _ptr(t), _ptr(y), _ptr(params),
                                 _ptr(w) if w is not None else None, _ptr(f), _ptr(gy), _ptr(gp), _stream(dev)))
    return f, gy, gp


def alu_peak(fp64=False, iters=None, blocks_per_sm=4, device=None, reps=3, packed=False):
    """Measured multiply-add throughput of the plain ALUs (TFLOP/s, 2 flops per FMA; best of `reps`
    launches of gs_alu_probe timed with CUDA events on the current stream). packed: FP32 on the
    two-lane FFMA2 instruction."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(8 * sms, dtype=torch.float64, device=dev)
    kind = 1 if fp64 else (2 if packed else 0)
    iters = int(iters or ((1 << 11) if fp64 else (1 << 16)))
    cnt = ctypes.c_int64()
    best = float("inf")
    for _ in range(reps + 1):  # the first launch warms up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _abi.check(_abi.lib().gs_alu_probe(kind, iters, int(blocks_per_sm), _ptr(sink), ctypes.byref(cnt),
                                           _stream(dev)))
        b.record()
        torch.cuda.synchronize(dev)
        best = min(best, a.elapsed_time(b))
    return 2.0 * cnt.value / (best / 1e3) / 1e12


SELFTEST_NAMES = ("narrow_f64", "widen_f32", "le_f64", "eq_f64", "nan_finite", "sign_ops", "le_nonneg_f64",
                  "log2_f64_f32", "max_abs_2m48")


def selftest(n=1 << 22, seed=0, device=None):
    """gs_selftest: the kernels' bit-level FP64 helpers against the instructions they replace, on the
    device. Returns {check name: (mismatches, bit pattern of one mismatching input)}."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    counts = torch.zeros(2 * _abi.SELFTEST_CHECKS, dtype=torch.int64, device=dev)
    _abi.check(_abi.lib().gs_selftest(int(n), int(seed), _ptr(counts), _stream(dev)))
    c = [v & 0xFFFFFFFFFFFFFFFF for v in counts.cpu().tolist()]
    return {name: (c[i], c[_abi.SELFTEST_CHECKS + i]) for i, name in enumerate(SELFTEST_NAMES)}


class GsSolve(torch.autograd.Function):
    """y = solve(y0, params) with the discrete adjoint as backward (torch autograd wiring)."""

    @staticmethod
    def forward(ctx, y0, params, system, t0, t1, saveat, rtol, atol, opts):
        r = solve(system, y0, params, t0, t1, saveat, rtol, atol, **opts)
        ctx.save_for_backward(y0, params if params is not None else torch.empty(0, device=y0.device), t0, t1, saveat,
                              r["n_accept"])
        ctx.cfg = (system, rtol, atol, opts)
        ctx.mark_non_differentiable(r["status"])
        return r["y"], r["status"]

    @staticmethod
    def backward(ctx, gy, gstatus):
        y0, params, t0, t1, saveat, n_acc = ctx.saved_tensors
        system, rtol, atol, opts = ctx.cfg
        _, p = _abi.dims(system)
        o = {k: v for k, v in opts.items() if k not in ("record_tape",)}
        r = vjp(system, y0, params if p else None, t0, t1, saveat, rtol, atol, gy.contiguous(), n_accept_hint=n_acc, **o)
        return r["dLdy0"], (r["dLdparams"] if p else None), None, None, None, None, None, None, None


def solve_autograd(system, y0, params, t0, t1, saveat, rtol, atol, **opts):
    """Differentiable solve: returns (y [N,K,d], status); y.backward() runs gs_vjp."""
    dev = y0.device
    N = y0.shape[0]
    t0 = torch.as_tensor(t0, dtype=torch.float64, device=dev).expand(N).contiguous()
    t1 = torch.as_tensor(t1, dtype=torch.float64, device=dev).expand(N).contiguous()
    saveat = torch.as_tensor(saveat, dtype=torch.float64, device=dev)
    return GsSolve.apply(y0, params, system, t0, t1, saveat, rtol, atol, opts)


class GraphedStep:
    """A forward solve (optionally recording its tape), an optional loss cotangent and the reverse
    sweep, captured once into a CUDA graph and replayed. Inputs and outputs are static device tensors:
    copy new inputs into `inputs[...]` and read `outputs[...]` after `replay()`.

    cotangent(y) -> dL/dy is captured with the solve (it must be made of stream-ordered device ops).
    The library's launches query occupancy and the device only on the host side, and every kernel
    argument lives in the captured tensors, so the graph is valid for as long as this object lives.
    The first call of the library on a device must happen before capture (it is warmed up here)."""

    def __init__(self, system, y0, params, t0, t1, saveat, rtol, atol, cotangent=None, grad=True, tape_slack=1.5,
                 **opts):
        dev = y0.device
        N = y0.shape[0]
        d, p = _abi.dims(system)
        self.inputs = dict(y0=y0.detach().clone(), params=(params.detach().clone() if p else None),
                           t0=_vec(t0, N, dev, "t0").clone(), t1=_vec(t1, N, dev, "t1").clone(),
                           saveat=_dev(saveat, dev, "saveat").clone())
        self.system, self.rtol, self.atol, self.opts, self.grad = system, rtol, atol, dict(opts), grad
        self.cotangent = cotangent
        self.ws = Workspace(dev)
        probe = solve(system, self.inputs["y0"], self.inputs["params"], self.inputs["t0"], self.inputs["t1"],
                      self.inputs["saveat"], rtol, atol, **opts)
        # the tape is sized once, from these inputs, with headroom for later inputs that take more steps;
        # trajectories that still do not fit report GS_ST_TAPE_OVERFLOW
        self.tape_nbytes = (tape_bytes(system, N, n_accept=(probe["n_accept"].double() * tape_slack).ceil().int(),
                                       precision=opts.get("precision", "fp64")) if grad else None)
        self.outputs = None
        self._run()  # warm-up outside capture: library load, workspace allocation, occupancy cache
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            with torch.cuda.graph(self.graph, stream=s):
                self._run()
        torch.cuda.current_stream(dev).wait_stream(s)

    def _run(self):
        i = self.inputs
        s = solve(self.system, i["y0"], i["params"], i["t0"], i["t1"], i["saveat"], self.rtol, self.atol,
                  record_tape=self.grad, workspace=self.ws, tape_nbytes=self.tape_nbytes, out=self.outputs and
                  {k: self.outputs[k] for k in ("y", "status", "n_accept", "n_reject")}, **self.opts)
        out = dict(s)
        if self.grad:
            w = self.cotangent(s["y"]) if self.cotangent is not None else torch.ones_like(s["y"])
            g = vjp(self.system, i["y0"], i["params"], i["t0"], i["t1"], i["saveat"], self.rtol, self.atol, w,
                    workspace=self.ws, reuse_tape=s, **self.opts)
            out.update(dLdy0=g["dLdy0"], dLdparams=g["dLdparams"])
        if self.outputs is None:
            self.outputs = out
        else:
            for k, v in out.items():
                if v.data_ptr() != self.outputs[k].data_ptr():
                    self.outputs[k].copy_(v)

    def replay(self):
        self.graph.replay()
        return self.outputs


class MixedBatch:
    """A serving batch of independent pieces (e.g. profile-likelihood fits, orbit gradients and
    precession solves) issued on one stream each and captured as one CUDA graph, so that they run
    concurrently; each piece's persistent kernels are held to its SM budget (gs_options.sm_limit).

    pieces: dict name -> callable(sm_limit) that enqueues the piece on the current stream and returns
    its output tensors. Every piece must use its own workspaces (concurrent pieces must not share
    scratch) and launch only stream-ordered work (graph-safe flatness solves for the fits). The
    callables are run once outside capture (library load, workspace allocation), then captured."""

    def __init__(self, pieces, sm_limits=None, device=None):
        dev = torch.device(device or "cuda")
        self.device = dev
        self.sm_limits = dict(sm_limits or {k: 0 for k in pieces})
        for k, f in pieces.items():
            f(self.sm_limits[k])
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        s0 = torch.cuda.Stream(dev)
        side = {k: torch.cuda.Stream(dev) for k in pieces}
        s0.wait_stream(torch.cuda.current_stream(dev))
        self.outputs = {}
        with torch.cuda.stream(s0):
            with torch.cuda.graph(self.graph, stream=s0):
                for k, f in pieces.items():
                    side[k].wait_stream(s0)
                    with torch.cuda.stream(side[k]):
                        self.outputs[k] = f(self.sm_limits[k])
                for st in side.values():
                    s0.wait_stream(st)
        torch.cuda.current_stream(dev).wait_stream(s0)

    def replay(self):
        """Run the whole batch (asynchronously on the current stream's device) and return the outputs."""
        self.graph.replay()
        return self.outputs
