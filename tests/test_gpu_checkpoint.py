"""Checkpoint stride S > 1 of the step tape (gs_options.ckpt_stride): the forward records the full
integrator state every S accepted steps and the reverse pass re-runs each segment of S steps from
its checkpoint before reversing it (the discrete counterpart of the checkpointing trade-off of
Appendix A, Eq. disc-modes).

The replay repeats the forward's own stage arithmetic (explicit fused multiply-adds, so the compiler
cannot round it differently in the two kernels) on the recorded step lengths, so it reproduces every
step's start state bit for bit. That is checked directly by the option ckpt_verify: the reverse pass
replays each full segment's last step as well and compares the state it reaches with the next
segment's checkpoint, bit for bit; every comparison must match.

The gradients then differ from the stride-1 gradient only by the rounding of the reverse arithmetic
itself, which the compiler may contract differently in the stride-1 and the checkpointed reverse
kernels: at most 1e-12 relative per trajectory in FP64 (about 1e-14 measured) and 1e-5 in the FP32
modes (their VJP chain rounds at 6e-8 per operation over ~10^3 steps). The stride-1 gradient is itself
checked against the oracle's forward sensitivities in tests/test_gpu_gradients.py; one case here
repeats that check for S = 16.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ensure_built, gpu_vjp
from paper_2609_28458_gb300 import _abi, api
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("mw", lambda: W.mw(n=512, seed=81, t1=1500.0, rtol=1e-9), "tsit5", "fp64"),
    ("mw", lambda: W.mw(n=256, seed=82, t1=800.0, rtol=1e-9), "vern7", "fp64"),
    ("isochrone", lambda: W.isochrone(n=256, seed=83), "dopri5", "fp64"),  # 11 outputs, t0 and t1 among them
    ("isochrone", lambda: W.isochrone(n=128, seed=84), "vern7", "fp64"),  # shortened-step outputs
    ("precession", lambda: W.precession(n=256, seed=85, paper_interval=True, rtol=1e-9), "vern7", "fp64"),
    ("precession", lambda: W.precession(n=512, seed=86), "tsit5", "fp64"),  # 20 Hz start: empty intervals
    ("quintessence", lambda: W.quintessence(n=256, seed=87, rtol=1e-8, dense=True), "tsit5", "fp64"),
    ("loghalo", lambda: W.loghalo(n=256, seed=88, rtol=1e-8), "dopri5", "fp64"),
    ("mw", lambda: W.mw(n=2048, seed=89, rtol=1e-8), "tsit5", "fp32df"),
    ("mw", lambda: W.mw(n=1024, seed=90, t1=1500.0, rtol=1e-8), "tsit5", "fp32"),
    ("quintessence", lambda: W.quintessence(n=512, seed=91, rtol=1e-6), "dopri5", "fp32df"),
    ("isochrone", lambda: W.isochrone(n=256, seed=92), "tsit5", "fp32df"),
]


def _same(a, b):
    return np.array_equal(a, b, equal_nan=True)


GRAD_TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32df": 1e-5}


def _grad(g):
    return np.concatenate([g["dLdy0"], g["dLdparams"]], axis=1)


@pytest.mark.parametrize("system,gen,method,prec", CASES)
def test_stride_replay_is_exact_and_gradient_matches_stride_one(system, gen, method, prec):
    e = gen()
    d, _ = O.dims(system)
    w = np.random.default_rng(3).normal(size=(e.n, e.saveat.shape[-1], d))
    ref = gpu_vjp(e, w, method=method, precision=prec, kernel="persistent", ckpt_stride=1)
    assert np.all((ref["status"] & _abi.ST_FAILED) == 0)
    gr = _grad(ref)
    ok = np.all(np.isfinite(gr), axis=1)
    for S in (2, 4, 16, 32):
        ws = api.Workspace(torch.device("cuda"))
        g = gpu_vjp(e, w, method=method, precision=prec, kernel="persistent", ckpt_stride=S, ckpt_verify=1,
                    workspace=ws)
        compared, differed = ws.buf[16:24].cpu().numpy().view(np.uint32)
        assert differed == 0 and (compared > 0 or S == 32), (S, compared, differed)
        for k in ("status", "n_accept", "n_reject", "y"):
            assert _same(g[k], ref[k]), (S, k)
        gg = _grad(g)
        assert np.array_equal(np.isnan(gg), np.isnan(gr))
        rel = np.linalg.norm(gg[ok] - gr[ok], axis=1) / np.maximum(np.linalg.norm(gr[ok], axis=1), 1e-300)
        assert rel.max() <= GRAD_TOL[prec], (S, rel.max())


def test_stride_sixteen_matches_oracle_sensitivities():
    """S = 16 against the oracle's forward-sensitivity gradient on equal step sequences (1e-8)."""
    e = W.mw(n=128, seed=93, t1=1000.0, rtol=1e-9)
    w = np.random.default_rng(4).normal(size=(e.n, 1, 6))
    ref = O.grad("mw", e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=e.rtol, atol=e.atol, method="tsit5")
    g = gpu_vjp(e, w, kernel="persistent", ckpt_stride=16)
    same = (g["n_accept"] == ref["n_accept"]) & (g["n_reject"] == ref["n_reject"])
    assert same.mean() >= 0.9
    gy = np.concatenate([g["dLdy0"], g["dLdparams"]], axis=1)
    ry = np.concatenate([ref["dLdy0"], ref["dLdparams"]], axis=1)
    err = np.linalg.norm(gy - ry, axis=1) / np.linalg.norm(ry, axis=1)
    assert err[same].max() <= 1e-8, err[same].max()


def test_stride_with_unused_outputs_and_per_trajectory_times():
    """Outputs outside [t0, t1] (NaN, no cotangent), outputs at t0 (y0 itself), per-trajectory output
    times and end times, and step counts that are not multiples of S: all as stride 1."""
    e = W.isochrone(n=300, seed=94)
    rng = np.random.default_rng(5)
    t1 = rng.uniform(5.0, 100.0, e.n)
    sv = np.stack([np.full(e.n, -1.0), np.zeros(e.n), 0.3 * t1, 0.71 * t1, t1, t1 + 3.0], axis=1)
    e.t1, e.saveat = t1, sv
    w = rng.normal(size=(e.n, sv.shape[1], 6))
    ref = gpu_vjp(e, w, method="tsit5", kernel="persistent")
    assert np.all((ref["status"] & O.ST_SAVEAT_OUTSIDE) != 0) and np.all((ref["status"] & _abi.ST_FAILED) == 0)
    assert len(np.unique(ref["n_accept"] % 8)) > 4
    for S in (4, 8):
        g = gpu_vjp(e, w, method="tsit5", kernel="persistent", ckpt_stride=S)
        for k in ("status", "y"):
            assert _same(g[k], ref[k]), (S, k)
        rel = np.linalg.norm(g["dLdy0"] - ref["dLdy0"], axis=1) / np.linalg.norm(ref["dLdy0"], axis=1)
        assert rel.max() <= GRAD_TOL["fp64"], (S, rel.max())


def test_stride_reuse_tape_and_overflow():
    """A tape recorded by gs_solve with a stride is reversed by gs_vjp(reuse_tape) as the re-run
    would; a workspace too small for every trajectory's tape flags those trajectories
    (GS_ST_TAPE_OVERFLOW, NaN gradients) and leaves the others bit for bit as with room to spare."""
    ensure_built()
    e = W.mw(n=1024, seed=95, t1=2000.0)
    dev = torch.device("cuda")
    y0 = torch.as_tensor(e.y0, device=dev)
    w = torch.as_tensor(np.random.default_rng(6).normal(size=(e.n, 1, 6)), device=dev)
    for prec in ("fp64", "fp32df"):
        kw = dict(precision=prec, kernel="persistent", ckpt_stride=16)
        ws = api.Workspace(dev)
        s = api.solve("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, record_tape=True, workspace=ws,
                      steps_hint=4000, **kw)
        a = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, reuse_tape=s, workspace=ws, **kw)
        b = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, **kw)
        torch.cuda.synchronize()
        assert torch.equal(a["dLdy0"], b["dLdy0"]) and torch.equal(a["dLdparams"], b["dLdparams"])
        nacc = b["n_accept"]
        full = api.tape_bytes("mw", e.n, n_accept=nacc, precision=prec, ckpt_stride=16)
        chunk = _abi.lib().gs_tape_chunk_bytes(1, _abi.ctypes.byref(_abi.options(precision=prec, ckpt_stride=16)))
        c = api.vjp("mw", y0, e.params, e.t0, e.t1, e.saveat, e.rtol, e.atol, w, tape_nbytes=full - 3 * e.n // 4 * chunk,
                    **kw)
        torch.cuda.synchronize()
        over = ((c["status"] & _abi.ST_TAPE_OVERFLOW) != 0).cpu().numpy()
        assert over.any() and (~over).any()
        g, gb = c["dLdy0"].cpu().numpy(), b["dLdy0"].cpu().numpy()
        assert np.all(np.isnan(g[over])) and np.array_equal(g[~over], gb[~over])
        assert torch.equal(c["y"], b["y"])
