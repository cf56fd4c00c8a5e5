"""Helpers shared by the GPU tests: run the library on a workload and bring results to the host."""
import numpy as np
import torch

from paper_2609_28458_gb300 import api
from paper_2609_28458_gb300 import build as gsbuild

_built = False


def ensure_built():
    global _built
    if not _built:
        gsbuild.build()
        _built = True


def gpu_solve(e, method=None, precision="fp64", kernel="plain", rtol=None, atol=None, **kw):
    ensure_built()
    dev = torch.device("cuda")
    y0 = torch.as_tensor(e.y0, device=dev)
    r = api.solve(e.system, y0, e.params, e.t0, e.t1, e.saveat, e.rtol if rtol is None else rtol,
                  e.atol if atol is None else atol, method=method or e.method, precision=precision, kernel=kernel, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def gpu_vjp(e, w, method=None, precision="fp64", kernel="plain", rtol=None, atol=None, **kw):
    ensure_built()
    dev = torch.device("cuda")
    y0 = torch.as_tensor(e.y0, device=dev)
    r = api.vjp(e.system, y0, e.params, e.t0, e.t1, e.saveat, e.rtol if rtol is None else rtol,
                e.atol if atol is None else atol, torch.as_tensor(w, device=dev), method=method or e.method,
                precision=precision, kernel=kernel, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def rel_err(a, b):
    """Per trajectory: max over outputs of ||a - b||_2 / ||b||_2."""
    num = np.linalg.norm(a - b, axis=-1)
    den = np.linalg.norm(b, axis=-1)
    return np.max(num / np.maximum(den, 1e-300), axis=-1)
