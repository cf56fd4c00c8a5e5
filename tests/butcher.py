"""Rooted trees and Runge-Kutta order conditions (Butcher theory, as in Hairer, Norsett & Wanner I,
Sec. II.2). Test helper: it generates every rooted tree up to a given order and evaluates the
elementary weights of a tableau, so that a tableau of order nu must satisfy
b . Phi(t) = 1/gamma(t) for every tree t with at most nu nodes."""
import itertools
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def trees(n):
    """All rooted trees with n nodes; a tree is a sorted tuple of its child subtrees."""
    if n == 1:
        return [()]
    out = set()
    for parts in _partitions(n - 1):
        pools = [trees(k) for k in parts]
        for combo in itertools.product(*pools):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def _partitions(n, maxpart=None):
    if maxpart is None:
        maxpart = n
    if n == 0:
        yield ()
        return
    for k in range(min(n, maxpart), 0, -1):
        for rest in _partitions(n - k, k):
            yield (k,) + rest


def order(t):
    return 1 + sum(order(c) for c in t)


def gamma(t):
    g = order(t)
    for c in t:
        g *= gamma(c)
    return g


def elementary(t, A):
    """Vector g(t) with g(leaf) = 1 and g([t1..tm]) = prod_k A g(t_k)."""
    s = A.shape[0]
    g = np.ones(s)
    for c in t:
        g = g * (A @ elementary(c, A))
    return g


def residuals(A, b, p, sigma=1.0):
    """Residuals b . g(t) - sigma^|t| / gamma(t) for every tree with at most p nodes."""
    res = []
    for n in range(1, p + 1):
        for t in trees(n):
            res.append((n, t, float(b @ elementary(t, A)) - sigma ** n / gamma(t)))
    return res
