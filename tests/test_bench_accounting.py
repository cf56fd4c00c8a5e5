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


def test_nystrom_counts_match_the_oracle_tableaux():
    """The FP32 modes take second-order systems' stages in Nystrom form: X_j = x + h c'_j v +
    h^2 sum_m (A^2)_jm a_m. A is strictly lower triangular, so (A^2)_jm vanishes for m >= j - 1, and
    the counts the benchmark uses are the nonzeros of A^2 and of (b - bhat) A."""
    b = _bench()
    for method, (n_aa, n_aa_rev, n_ea, n_ba) in b.NYSTROM_NNZ.items():
        T = O.tableau(method)
        A, bb, bh = np.array(T["A"]), np.array(T["b"]), np.array(T["bh"])
        AA = A @ A
        S = T["s"]
        for j in range(S):
            assert np.all(AA[j, max(j - 1, 0):] == 0.0)
        nz = lambda x: int((np.abs(x) > 1e-14).sum())
        assert nz(AA[1:S]) == n_aa
        assert nz(AA[1:6]) == n_aa_rev
        assert nz((bb - bh) @ A) == n_ea and nz(bb @ A) == n_ba
        # the error weights sum to zero (b and bhat both sum to one), so the position error has no v term
        assert abs((bb - bh).sum()) < 1e-15 and abs(bb.sum() - 1.0) < 1e-15
    assert b.forward_flops("mw", "tsit5", 6, 1, 1, "fp32") == b.F_ATT_FWD_NY
    assert b.reverse_flops("mw", "tsit5", 6, 1, "fp32") - b.reverse_flops("mw", "tsit5", 6, 1) == \
        6 * (10 + 10) - 2 * 6 * 21 + 6 * (10 + 6 + 6 + 5) - 2 * 6 * (21 + 6)
    assert b.att_flops("fp64") == (b.F_ATT_FWD, b.F_STEP_REV)
    assert b.att_flops("fp32") == (b.F_ATT_FWD_NY, b.F_STEP_REV_NY)


def test_nystrom_form_is_the_same_stages():
    """For f = (v, a(x)) the general-form stage positions x + h sum_l a_jl V_l, V_l = v + h sum_m
    a_lm a_m, the new position and the position error equal their Nystrom forms, for any values of
    the stage accelerations (the identity the FP32 kernels' Nystrom stages rest on)."""
    rng = np.random.default_rng(5)
    for method in ("tsit5", "dopri5"):
        T = O.tableau(method)
        A, bb, bh = np.array(T["A"]), np.array(T["b"]), np.array(T["bh"])
        S = T["s"]
        x, v, h = rng.normal(size=3), rng.normal(size=3), 0.37
        acc = rng.normal(size=(S, 3))
        V = v[None, :] + h * (A @ acc)
        X_general = x[None, :] + h * (A @ V)
        X_nystrom = x[None, :] + h * A.sum(1)[:, None] * v[None, :] + h * h * ((A @ A) @ acc)
        assert np.allclose(X_general, X_nystrom, rtol=0, atol=1e-13)
        assert np.allclose(x + h * (bb @ V), x + h * v + h * h * ((bb @ A) @ acc), rtol=0, atol=1e-13)
        assert np.allclose(h * ((bb - bh) @ V), h * h * (((bb - bh) @ A) @ acc), rtol=0, atol=1e-13)


def test_nystrom_systems_match_the_kernels():
    """bench.py counts Nystrom-form work for exactly the systems the kernels mark second-order
    (gs_systems.cuh, SECOND_ORDER) and the pairs they take in that form (7-stage FSAL)."""
    import re
    src = open(os.path.join(ROOT, "paper_2609_28458_gb300", "csrc", "gs_systems.cuh")).read()
    marked = set()
    for m in re.finditer(r"struct (\w+) \{(.*?)\n\};", src, re.S):
        if "SECOND_ORDER = true" in m.group(2):
            marked.add(m.group(1))
    names = {"Isochrone": "isochrone", "MilkyWay": "mw", "LogHalo": "loghalo"}
    assert {names[m] for m in marked} == set(_bench().SECOND_ORDER)
    b = _bench()
    for method, (S, fsal, *_rest) in b.TABLEAU_NNZ.items():
        assert (method in b.NYSTROM_NNZ) == (fsal and S == 7)
