"""Pins of the oracle's Butcher tableaux (CPU only).

The paper names the methods (Sec. 2.2: Tsit5, Dopri5, Verner 7) but prints no coefficients, so the
oracle carries those of the primary publications. Here they are checked against what the
mathematics fixes: the Butcher order conditions for every rooted tree up to the claimed order
(85 trees for order 7), the row-sum condition, the failure of the next order (so the claimed
order is exact), and for the dense-output polynomials of Eq. dense b_j(1) = b_j and the order-4
conditions at every sigma.
"""
import numpy as np
import pytest

import butcher
import oracle as O

CASES = [("tsit5", 5, 1e-13), ("dopri5", 5, 1e-15), ("vern7", 7, 1e-14)]


def test_tree_counts():
    # number of rooted trees with n nodes (OEIS A000081)
    assert [len(butcher.trees(n)) for n in range(1, 8)] == [1, 1, 2, 4, 9, 20, 48]


@pytest.mark.parametrize("method,nu,tol", CASES)
def test_row_sums(method, nu, tol):
    T = O.tableau(method)
    assert np.allclose(T["A"].sum(axis=1), T["c"], atol=1e-15 * 200)
    assert np.all(np.triu(T["A"]) == 0.0), "explicit method: A strictly lower triangular"


@pytest.mark.parametrize("method,nu,tol", CASES)
def test_order_conditions_propagated(method, nu, tol):
    T = O.tableau(method)
    res = butcher.residuals(T["A"], T["b"], nu)
    assert len(res) == sum(len(butcher.trees(n)) for n in range(1, nu + 1))
    worst = max(abs(r[2]) for r in res)
    assert worst < tol, worst
    # and the order is not higher than claimed
    nxt = butcher.residuals(T["A"], T["b"], nu + 1)
    assert max(abs(r[2]) for r in nxt if r[0] == nu + 1) > 1e-7


@pytest.mark.parametrize("method,nu,tol", CASES)
def test_order_conditions_embedded(method, nu, tol):
    T = O.tableau(method)
    res = butcher.residuals(T["A"], T["bh"], nu - 1)
    assert max(abs(r[2]) for r in res) < tol
    nxt = butcher.residuals(T["A"], T["bh"], nu)
    assert max(abs(r[2]) for r in nxt if r[0] == nu) > 1e-6


@pytest.mark.parametrize("method", ["tsit5", "dopri5"])
def test_fsal_structure(method):
    T = O.tableau(method)
    assert T["fsal"]
    assert np.allclose(T["A"][-1, :-1], T["b"][:-1], atol=0, rtol=0)
    assert T["b"][-1] == 0.0 and T["c"][-1] == 1.0


@pytest.mark.parametrize("method", ["tsit5", "dopri5"])
def test_dense_output(method):
    T = O.tableau(method)
    assert np.allclose(O.dense_weights(method, 1.0), T["b"], atol=5e-15)
    assert np.allclose(O.dense_weights(method, 0.0), 0.0, atol=0)
    for sig in np.linspace(0.0, 1.0, 21):
        w = O.dense_weights(method, sig)
        res = butcher.residuals(T["A"], w, 4, sigma=sig)
        assert max(abs(r[2]) for r in res) < 5e-14, (sig, res)


def test_vern7_has_no_polynomial():
    with pytest.raises(ValueError):
        O.dense_weights("vern7", 0.5)


@pytest.mark.parametrize("method,nu,tol", CASES)
def test_any_single_mistyped_coefficient_fails_a_condition(method, nu, tol):
    """A plausible transcription error (one entry off in its 7th significant digit) in A, b or bh
    breaks at least one order condition: the pins above cannot be passed by a wrong tableau."""
    T = O.tableau(method)
    for name, order in (("A", nu), ("b", nu), ("bh", nu - 1)):
        arr = T[name]
        for idx in zip(*np.nonzero(arr)):
            bad = {k: v.copy() for k, v in T.items() if isinstance(v, np.ndarray)}
            bad[name][idx] *= 1 + 1e-6
            weights = bad["b"] if name in ("A", "b") else bad["bh"]
            worst = max(abs(r[2]) for r in butcher.residuals(bad["A"], weights, order))
            if name == "A":  # an entry of A also breaks the row-sum condition
                worst = max(worst, np.abs(bad["A"].sum(1) - T["c"]).max())
            assert worst > 1e-12, (name, idx)
