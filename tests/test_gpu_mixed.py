"""The mixed serving batch (three ensembles in one CUDA graph, on concurrent streams with SM budgets)
gives exactly the results of the same pieces run one after another: every trajectory's arithmetic is
deterministic, so concurrency, SM budgets and graph replay change nothing. Replays repeat."""
import pytest
import torch

from gpu_util import ensure_built
from paper_2609_28458_gb300 import api, autotune, serving

pytestmark = pytest.mark.gpu


def _same(a, b):
    assert not torch.isnan(a).any() if a.is_floating_point() else True
    return torch.equal(a, b)


def test_mixed_batch_graph_matches_separate_calls():
    ensure_built()
    P = serving.pieces(n_lam=2, n_mock=4, n_mw=4096, n_prec=2048)
    sep = {}
    for k, f in P.items():
        sep[k] = {kk: v.clone() for kk, v in f(0).items()}
    torch.cuda.synchronize()
    assert bool((sep["fits"]["converged"] == 1).all())
    assert int((sep["orbits"]["status"] != 0).sum()) == 0
    shares, alone = autotune.share_sms(P, reps=1)
    assert set(shares) == set(P) and all(v >= 1 for v in shares.values())
    mb = api.MixedBatch(P, sm_limits=shares)
    for _ in range(2):
        out = mb.replay()
        torch.cuda.synchronize()
        for k in P:
            for kk, v in sep[k].items():
                assert _same(out[k][kk], v), (k, kk)
