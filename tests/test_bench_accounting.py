"""The benchmark's algorithmic flop accounting (CPU): the tableau nonzeros it uses equal those of the
oracle's published coefficients, and its per-attempt count for the Milky-Way Tsit5 forward is the
one the headline roofline uses."""
import importlib.util
import os

import numpy as np

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_tableau_nonzeros_match_the_oracle():
    b = _bench()
    for method, (S, fsal, n_a, n_b, n_e) in b.TABLEAU_NNZ.items():
        T = O.tableau(method)
        A, bb, bh = np.array(T["A"]), np.array(T["b"]), np.array(T["bh"])
        assert T["s"] == S and bool(T["fsal"]) == fsal
        assert int((A != 0).sum()) == n_a and int((bb != 0).sum()) == n_b
        assert int((bb - bh != 0).sum()) == n_e


def test_forward_flops_is_the_headline_count():
    b = _bench()
    assert b.forward_flops("mw", "tsit5", 6, 1, 1) == b.F_ATT_FWD
    # non-FSAL pairs add the new-state combination and one right-hand side per accepted step
    S, _, n_a, n_b, n_e = b.TABLEAU_NNZ["vern7"]
    f = b.F_RHS["precession"]
    assert b.forward_flops("precession", "vern7", 9, 10, 7) == 10 * ((S - 1) * f + 18 * (n_a + n_b + n_e) + 40) + 7 * f
