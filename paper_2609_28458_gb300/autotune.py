"""Launch-configuration autotuner for the ensemble kernels.

For a (system, method, precision) key it times the candidate launch configurations on a sample of
the caller's ensemble and keeps the fastest, cached in a JSON file so later processes reuse the
choice. Candidates: kernel (plain one-thread-per-trajectory, or persistent work queue) x block size
(64, 96, 128 threads). The per-trajectory arithmetic does not depend on the launch configuration, so
every candidate returns the same results; only the time differs.

The cache key includes the GPU name so a cache copied to other hardware is not reused.
"""
import json
import os
import time

import numpy as np
import torch

from . import api

CANDIDATES = [(k, b) for k in ("persistent", "plain") for b in (128, 96, 64)]
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gs_gb300_autotune.json")


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
    """The fastest (kernel, block) of {(kernel, block): ms}."""
    return min(timings.items(), key=lambda kv: kv[1])[0]


def tune(system, y0, params, t0, t1, saveat, rtol, atol, method="tsit5", precision="fp64", fwd_grad=False,
         sample=65536, reps=2, cache_path=DEFAULT_CACHE, force=False, timer=None):
    """Best (kernel, block_size) for this key; times candidates on up to `sample` trajectories.
    `timer(kernel, block)` may replace the GPU timing (it returns milliseconds)."""
    key = _key(system, method, precision, fwd_grad)
    cache = load_cache(cache_path)
    if not force and key in cache:
        c = cache[key]
        return c["kernel"], int(c["block_size"])
    if timer is None:
        n = y0.shape[0]
        idx = torch.as_tensor(np.sort(np.random.default_rng(0).choice(n, min(n, sample), replace=False)),
                              device=y0.device)
        sub = lambda x: (x[idx] if torch.is_tensor(x) and x.dim() and x.shape[0] == n else x)
        Y0, P, T0, T1, SV = sub(y0), (sub(params) if params is not None else None), sub(t0), sub(t1), sub(saveat)
        ws = api.Workspace(y0.device)

        def timer(kernel, block):
            def run():
                if fwd_grad:
                    s = api.solve(system, Y0, P, T0, T1, SV, rtol, atol, method=method, precision=precision,
                                  kernel=kernel, block_size=block, record_tape=True, workspace=ws,
                                  tape_nbytes=nbytes)
                    api.vjp(system, Y0, P, T0, T1, SV, rtol, atol, torch.ones_like(s["y"]), method=method,
                            precision=precision, kernel=kernel, block_size=block, reuse_tape=s, workspace=ws)
                else:
                    api.solve(system, Y0, P, T0, T1, SV, rtol, atol, method=method, precision=precision,
                              kernel=kernel, block_size=block)

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

        nbytes = None
        if fwd_grad:
            probe = api.solve(system, Y0, P, T0, T1, SV, rtol, atol, method=method, precision=precision)
            nbytes = api.tape_bytes(system, Y0.shape[0], n_accept=probe["n_accept"], precision=precision)
    t = time.time()
    timings = {c: timer(*c) for c in CANDIDATES}
    kernel, block = pick(timings)
    cache[key] = {"kernel": kernel, "block_size": block, "ms": {"%s/%d" % c: v for c, v in timings.items()},
                  "tuned_at": t}
    save_cache(cache, cache_path)
    return kernel, block


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
