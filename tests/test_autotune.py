"""Autotuner host logic (CPU): candidate selection, the memory rule for the checkpoint stride and the
JSON cache, with a fake timer and a fake memory test."""
import os

import pytest

from paper_2609_28458_gb300 import autotune


def test_pick_and_cache_roundtrip(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def fake_timer(kernel, block, lanes, stride):
        calls.append((kernel, block, lanes, stride))
        return {"persistent": 10.0, "plain": 20.0}[kernel] + {128: 1.0, 96: 0.5, 64: 2.0}[block]

    # a large ensemble: every lane of a warp takes work
    c = autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, timer=fake_timer, cache_path=path, n=1 << 20)
    assert c == ("persistent", 96, 32, 1)
    assert sorted(calls) == sorted((k, b, 32, 1) for k, b in autotune.KERNELS)
    assert os.path.exists(path)
    calls.clear()
    assert autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, timer=fake_timer, cache_path=path) == c
    assert calls == []  # served from the cache
    c2 = autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, precision="fp32df", cache_path=path,
                       timer=lambda kernel, block, lanes, stride: {"persistent": 5.0, "plain": 1.0}[kernel] + block / 1000)
    assert c2.kernel == "plain"  # a different key is tuned separately
    assert len(autotune.load_cache(path)) == 2


def test_gradient_candidates_respect_the_memory_budget(tmp_path):
    """Gradient runs add the checkpoint stride: stride 1 for both kernels, larger strides for the
    persistent kernels only, and only strides whose tape fits; the fastest fitting one wins."""
    path = str(tmp_path / "cache.json")
    cand = autotune.candidates(True)
    assert {s for _, _, _, s in cand} == set(autotune.STRIDES)
    assert all(k == "persistent" for k, _, _, s in cand if s > 1)
    # only strides >= 8 fit: stride 1 (fastest) is not a candidate
    fits = lambda s: s >= 8
    c = autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, fwd_grad=True, cache_path=path,
                      stride_fits=fits, timer=lambda k, b, l, s: 1.0 * s + (0 if b == 128 else 1), n=1 << 20)
    assert c == ("persistent", 128, 32, 8)
    with pytest.raises(MemoryError):
        autotune.candidates(True, stride_fits=lambda s: False)


def test_small_ensembles_also_try_fewer_lanes_per_warp(tmp_path):
    """A small ensemble (fewer trajectories than the GPU's resident lanes) may leave lanes idle to
    spread over more warps; the candidates then include 16 and 8 lanes, persistent kernels only."""
    small = autotune.candidates(False, small=True)
    assert {l for _, _, l, _ in small} == set(autotune.LANES)
    assert all(k == "persistent" for k, _, l, _ in small if l < 32)
    c = autotune.tune("isochrone", None, None, None, None, None, 1e-10, 1e-12, cache_path=str(tmp_path / "c.json"),
                      n=4096, timer=lambda k, b, l, s: {32: 3.0, 16: 2.0, 8: 2.5}[l] + (0 if k == "persistent" else 9))
    assert c.warp_lanes == 16 and c.kernel == "persistent"
