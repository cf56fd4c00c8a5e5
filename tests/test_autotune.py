"""Autotuner host logic (CPU): candidate selection and the JSON cache, with a fake timer."""
import os

from paper_2609_28458_gb300 import autotune


def test_pick_and_cache_roundtrip(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def fake_timer(kernel, block):
        calls.append((kernel, block))
        return {"persistent": 10.0, "plain": 20.0}[kernel] + {128: 1.0, 96: 0.5, 64: 2.0}[block]

    k, b = autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, timer=fake_timer, cache_path=path)
    assert (k, b) == ("persistent", 96)
    assert sorted(calls) == sorted(autotune.CANDIDATES)
    assert os.path.exists(path)
    calls.clear()
    assert autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, timer=fake_timer, cache_path=path) == (k, b)
    assert calls == []  # served from the cache
    k2, _ = autotune.tune("mw", None, None, None, None, None, 1e-8, 1e-8, precision="fp32df", cache_path=path,
                          timer=lambda kernel, block: {"persistent": 5.0, "plain": 1.0}[kernel] + block / 1000)
    assert k2 == "plain"  # a different key is tuned separately
    assert len(autotune.load_cache(path)) == 2
