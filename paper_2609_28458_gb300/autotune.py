"""Launch-configuration autotuner for the ensemble kernels.

For a (system, method, precision, forward or gradient) key it times the candidate configurations on a
sample of the caller's ensemble and keeps the fastest, cached in a JSON file so later processes reuse
the choice. Candidates: kernel (plain one-thread-per-trajectory, or persistent work queue) x block
size (64, 96, 128 threads); for ensembles smaller than the GPU's resident lanes, the lanes per warp
that take trajectories in the persistent kernels (gs_options.warp_lanes: 32, 16, 8; fewer spread a
small ensemble over more warps and schedulers); and, for gradient runs, the checkpoint stride of the
step tape (gs_options.ckpt_stride: 1, 4, 8, 16, 32; strides above 1 run in the persistent kernels).
A stride is a candidate only if the tape it needs for the whole ensemble fits the memory budget:
stride 1 never recomputes a step but stores every step's state; a stride S stores a checkpoint every
S steps and the reverse pass replays each segment (about S times less tape for one more forward step
per reversed step). The per-trajectory arithmetic does not depend on the configuration, so every
candidate returns the same solution; only time and memory differ.

The cache key includes the GPU name so a cache copied to other hardware is not reused.
"""
import json
import os
import time
from collections import namedtuple

import numpy as np
import torch

from . import api

KERNELS = [(k, b) for k in ("persistent", "plain") for b in (128, 96, 64)]
STRIDES = (1, 4, 8, 16, 32)
LANES = (32, 16, 8)
SMALL_ENSEMBLE = 1 << 16  # below this, fewer lanes per warp are candidates too
CANDIDATES = KERNELS  # the forward's (kernel, block) pairs
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gs_gb300_autotune.json")

Choice = namedtuple("Choice", ["kernel", "block_size", "warp_lanes", "ckpt_stride"])


def _key(system, method, precision, fwd_grad):
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return "%s|%s|%s|%s|%s" % (name, system, method, precision, "fwdgrad" if fwd_grad else "fwd")


def load_cache(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(timings):
    """The fastest candidate of {candidate: ms}."""
    return min(timings.items(), key=lambda kv: kv[1])[0]


def candidates(fwd_grad, stride_fits=None, small=False):
    """(kernel, block, lanes, stride) candidates: lanes below 32 only for small ensembles and the
    persistent kernels; strides only for gradient runs, above 1 only in the persistent kernels, and
    only those whose tape fits (stride_fits(S), default: all)."""
    base = [(k, b, l) for k, b in KERNELS for l in (LANES if small else (32,)) if l == 32 or k == "persistent"]
    if not fwd_grad:
        return [(k, b, l, 1) for k, b, l in base]
    fits = stride_fits or (lambda s: True)
    out = [(k, b, l, s) for s in STRIDES for k, b, l in base if (s == 1 or k == "persistent") and fits(s)]
    if not out:
        raise MemoryError("no checkpoint stride up to %d fits the tape into the memory budget" % STRIDES[-1])
    return out


def pick_stride(system, n, n_accept, precision, budget_bytes, kernel="persistent", K=1, strides=STRIDES):
    """The memory rule alone (no timing): stride 1, the fastest reverse pass, when its tape for the
    accepted-step counts n_accept [n] fits budget_bytes; else the smallest stride whose tape fits.
    The plain kernel records every step. Raises MemoryError when none fits."""
    for s in strides:
        if s > 1 and kernel == "plain":
            break
        if api.tape_bytes(system, n, n_accept=n_accept, precision=precision, K=K, ckpt_stride=s) <= budget_bytes:
            return s
    raise MemoryError("the %s tape of %d trajectories fits no checkpoint stride within %.1f GB" %
                      (system, n, budget_bytes / 1e9))


def tune(system, y0, params, t0, t1, saveat, rtol, atol, method="tsit5", precision="fp64", fwd_grad=False,
         sample=65536, reps=2, cache_path=DEFAULT_CACHE, force=False, timer=None, budget_bytes=None,
         stride_fits=None, n=None):
    """Best Choice(kernel, block_size, warp_lanes, ckpt_stride) for this key; times candidates on up
    to `sample` trajectories (n, the ensemble size, defaults to y0's). For gradient runs the strides
    considered are those whose tape for the whole ensemble (the sample's accepted-step counts scaled
    to it) fits budget_bytes (default: half the free device memory). `timer(kernel, block, lanes,
    stride)` and `stride_fits(stride)` may replace the GPU timing (milliseconds) and the memory test."""
    key = _key(system, method, precision, fwd_grad)
    cache = load_cache(cache_path)
    if not force and key in cache:
        c = cache[key]
        return Choice(c["kernel"], int(c["block_size"]), int(c.get("warp_lanes", 32)), int(c.get("ckpt_stride", 1)))
    if n is None:
        n = y0.shape[0] if y0 is not None else SMALL_ENSEMBLE
    if timer is None:
        idx = torch.as_tensor(np.sort(np.random.default_rng(0).choice(n, min(n, sample), replace=False)),
                              device=y0.device)
        sub = lambda x: (x[idx] if torch.is_tensor(x) and x.dim() and x.shape[0] == n else x)
        Y0, P, T0, T1, SV = sub(y0), (sub(params) if params is not None else None), sub(t0), sub(t1), sub(saveat)
        K = SV.shape[-1]
        ws = api.Workspace(y0.device)
        nbytes = {}
        if fwd_grad:
            probe = api.solve(system, Y0, P, T0, T1, SV, rtol, atol, method=method, precision=precision)
            scale = n / Y0.shape[0]
            if budget_bytes is None:
                budget_bytes = torch.cuda.mem_get_info(y0.device)[0] // 2
            for s in STRIDES:
                nbytes[s] = api.tape_bytes(system, Y0.shape[0], n_accept=probe["n_accept"], precision=precision, K=K,
                                           ckpt_stride=s)
            if stride_fits is None:
                stride_fits = lambda s: nbytes[s] * scale <= budget_bytes

        def timer(kernel, block, lanes, stride):
            def run():
                kw = dict(method=method, precision=precision, kernel=kernel, block_size=block, warp_lanes=lanes)
                if fwd_grad:
                    s = api.solve(system, Y0, P, T0, T1, SV, rtol, atol, record_tape=True, workspace=ws,
                                  tape_nbytes=nbytes[stride], ckpt_stride=stride, **kw)
                    api.vjp(system, Y0, P, T0, T1, SV, rtol, atol, torch.ones_like(s["y"]), reuse_tape=s,
                            workspace=ws, ckpt_stride=stride, **kw)
                else:
                    api.solve(system, Y0, P, T0, T1, SV, rtol, atol, **kw)

            run()
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                run()
                b.record()
                torch.cuda.synchronize()
                best = min(best, a.elapsed_time(b))
            return best

    t = time.time()
    timings = {c: timer(*c) for c in candidates(fwd_grad, stride_fits, small=n < SMALL_ENSEMBLE)}
    kernel, block, lanes, stride = pick(timings)
    cache[key] = {"kernel": kernel, "block_size": block, "warp_lanes": lanes, "ckpt_stride": stride,
                  "ms": {"%s/%d/L%d/S%d" % c: v for c, v in timings.items()}, "tuned_at": t}
    save_cache(cache, cache_path)
    return Choice(kernel, block, lanes, stride)


def share_sms(pieces, sm_count=None, reps=2):
    """SM budgets for the pieces of a MixedBatch: each piece is timed alone on the whole GPU and gets
    SMs in proportion to its time, so that the concurrent pieces finish together. Returns
    (dict name -> sm_limit, dict name -> ms alone)."""
    dev = torch.device("cuda")
    if sm_count is None:
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alone = {}
    for k, f in pieces.items():
        f(0)
        torch.cuda.synchronize(dev)
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f(0)
            b.record()
            torch.cuda.synchronize(dev)
            best = min(best, a.elapsed_time(b))
        alone[k] = best
    total = sum(alone.values())
    shares = {k: max(1, int(round(sm_count * t / total))) for k, t in alone.items()}
    return shares, alone
