"""CUDA-graph capture of the forward + adjoint sequence: replays are bitwise equal to eager launches
with the same inputs, including after new inputs are copied into the captured tensors."""
import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from paper_2609_28458_gb300 import api
from paper_2609_28458_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _eager(system, e, y0, pr, precision, method, cot):
    s = api.solve(system, y0, pr, e.t0, e.t1, e.saveat, e.rtol, e.atol, precision=precision, method=method)
    g = api.vjp(system, y0, pr, e.t0, e.t1, e.saveat, e.rtol, e.atol, cot(s["y"]), precision=precision,
                method=method)
    return s, g


@pytest.mark.parametrize("system,gen,precision,method", [
    ("isochrone", lambda s: W.isochrone(n=4096, seed=s), "fp64", "tsit5"),
    ("mw", lambda s: W.mw(n=8192, seed=70 + s, t1=1000.0, rtol=1e-8), "fp32df", "tsit5"),
    ("quintessence", lambda s: W.quintessence(n=4096, seed=80 + s, rtol=1e-6), "fp32", "dopri5"),
])
def test_graph_replay_equals_eager(system, gen, precision, method):
    ensure_built()
    dev = torch.device("cuda")
    e = gen(0)
    y0 = torch.as_tensor(e.y0, device=dev)
    pr = torch.as_tensor(e.params, device=dev) if e.params.shape[1] else None
    tgt = torch.as_tensor(np.random.default_rng(1).normal(size=(e.n, e.saveat.shape[-1], e.y0.shape[1])), device=dev)
    cot = lambda y: y - tgt
    gs = api.GraphedStep(system, y0, pr, e.t0, e.t1, e.saveat, e.rtol, e.atol, cotangent=cot, precision=precision,
                         method=method, kernel="persistent")
    for rep in range(2):
        out = gs.replay()
        torch.cuda.synchronize()
        s, g = _eager(system, e, y0, pr, precision, method, cot)
        torch.cuda.synchronize()
        assert torch.equal(out["y"], s["y"]) and torch.equal(out["status"], s["status"])
        assert torch.equal(out["dLdy0"], g["dLdy0"]) and torch.equal(out["dLdparams"], g["dLdparams"])
    # new inputs copied into the captured tensors
    e2 = gen(1)
    y2 = torch.as_tensor(e2.y0, device=dev)
    p2 = torch.as_tensor(e2.params, device=dev) if e2.params.shape[1] else None
    gs.inputs["y0"].copy_(y2)
    if p2 is not None:
        gs.inputs["params"].copy_(p2)
    out = gs.replay()
    torch.cuda.synchronize()
    s, g = _eager(system, e2, y2, p2, precision, method, cot)
    torch.cuda.synchronize()
    ok = (out["status"] & 32) == 0
    assert ok.float().mean() > 0.99
    assert torch.equal(out["y"], s["y"])
    assert torch.equal(out["dLdy0"][ok], g["dLdy0"][ok]) and torch.equal(out["dLdparams"][ok], g["dLdparams"][ok])


def test_autotuned_configuration_gives_identical_results(tmp_path):
    from paper_2609_28458_gb300 import autotune

    ensure_built()
    dev = torch.device("cuda")
    e = W.mw(n=20000, seed=90, t1=1000.0, rtol=1e-8)
    y0, pr = torch.as_tensor(e.y0, device=dev), torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    kernel, block, lanes, _ = autotune.tune("mw", y0, pr, t0, t1, sv, e.rtol, e.atol, precision="fp32df", sample=8192,
                                  cache_path=str(tmp_path / "c.json"))
    assert (kernel, block) in autotune.CANDIDATES and lanes in autotune.LANES
    a = api.solve("mw", y0, pr, t0, t1, sv, e.rtol, e.atol, precision="fp64", kernel=kernel, block_size=block,
                  warp_lanes=lanes)
    b = api.solve("mw", y0, pr, t0, t1, sv, e.rtol, e.atol, precision="fp64", kernel="plain", block_size=128)
    torch.cuda.synchronize()
    same = (a["n_accept"] == b["n_accept"]) & (a["n_reject"] == b["n_reject"])
    assert same.float().mean() > 0.95
