"""Multi-process sharding of an ensemble (CPU, gloo, world size 2): shards cover every member exactly
once, and the shared-parameter gradient summed across ranks equals the unsharded sum (Eq. chain).
Per-member gradients come from the CPU oracle; no GPU is involved."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2609_28458_gb300.sharding import shard_bounds, sum_shared_gradient


def test_shard_bounds_partition():
    for n in (0, 1, 7, 64, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [shard_bounds(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, out):
    import oracle as O
    from paper_2609_28458_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    e = W.mw(n=n, seed=91, t1=300.0, rtol=1e-8)
    a, b = shard_bounds(n, world, rank)
    s = e.subset(np.arange(a, b))
    w = np.random.default_rng(3).normal(size=(n, 1, 6))[a:b]
    g = O.grad("mw", s.y0, s.params, s.t0, s.t1, s.saveat, w, rtol=s.rtol, atol=s.atol, nthreads=1)
    total = sum_shared_gradient(torch.as_tensor(g["dLdparams"]))
    out[rank] = total.numpy().tolist()
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_rank_shared_gradient_equals_unsharded():
    import oracle as O
    from paper_2609_28458_gb300 import workloads as W

    n, world = 24, 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), n, out), nprocs=world, start_method="spawn", join=True)
    e = W.mw(n=n, seed=91, t1=300.0, rtol=1e-8)
    w = np.random.default_rng(3).normal(size=(n, 1, 6))
    g = O.grad("mw", e.y0, e.params, e.t0, e.t1, e.saveat, w, rtol=e.rtol, atol=e.atol, nthreads=1)
    ref = g["dLdparams"].sum(axis=0)
    for r in range(world):
        assert np.allclose(out[r], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
