"""Butcher-series expansion of a Runge-Kutta step for the scalar autonomous ODE w' = K w^p.

Test-side mathematics (Hairer, Norsett & Wanner, "Solving Ordinary Differential Equations I",
Sec. II.2): a Runge-Kutta method with stage matrix A and weights w maps w0 to

    w1 = w0 + sum over rooted trees t of  h^|t| / sigma(t) * Phi_w(t) * F(t)(w0),

and the exact flow is the same series with Phi_w(t) replaced by 1/gamma(t).  For F(w) = K w^p each
elementary differential is  h^|t| F(t)(w) = w * u^|t| * P(t)  with  u = h K w^(p-1)  and P(t) the
product over the tree's nodes of the falling factorial p (p-1) ... (p-m+1), m the node's number of
children.  The leading-order chirp (Eq. 1 with every correction off) is this ODE with p = 11/3 and
K = (96/5) eta.

Nothing here uses the oracle's integrator or error norm: only the Butcher tableau, which the
order-condition tests pin on their own.
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial

import numpy as np


def _canon(children) -> tuple:
    return tuple(sorted(children))


def _grow(t: tuple) -> list:
    """Every tree obtained from t by attaching one leaf to one of its nodes."""
    out = [_canon(t + ((),))]
    for i, c in enumerate(t):
        for g in _grow(c):
            out.append(_canon(t[:i] + (g,) + t[i + 1:]))
    return out


@lru_cache(maxsize=None)
def trees(order: int) -> tuple:
    """All rooted trees with `order` nodes, each a sorted tuple of its children's trees."""
    if order == 1:
        return ((),)
    found = set()
    for t in trees(order - 1):
        found.update(_grow(t))
    return tuple(sorted(found))


def size(t: tuple) -> int:
    return 1 + sum(size(c) for c in t)


def gamma(t: tuple) -> int:
    """Density: |t| times the densities of the subtrees."""
    g = size(t)
    for c in t:
        g *= gamma(c)
    return g


def sigma(t: tuple) -> int:
    """Symmetry: product over distinct subtrees of (multiplicity)! sigma(subtree)^multiplicity."""
    s = 1
    for c in set(t):
        m = t.count(c)
        s *= factorial(m) * sigma(c) ** m
    return s


def stage_weights(t: tuple, A: np.ndarray, memo: dict | None = None) -> np.ndarray:
    """Phi_i(t) for every stage i: 1 for a leaf, else the product over subtrees of (A Phi(subtree))_i."""
    memo = {} if memo is None else memo
    if t not in memo:
        v = np.ones(A.shape[0])
        for c in t:
            v = v * (A @ stage_weights(c, A, memo))
        memo[t] = v
    return memo[t]


def falling_product(t: tuple, p: float) -> float:
    """P(t): product over the nodes of p (p-1) ... (p-m+1), m the node's number of children."""
    m = len(t)
    f = 1.0
    for j in range(m):
        f *= p - j
    for c in t:
        f *= falling_product(c, p)
    return f


def exact_coefficients(p: float, kmax: int) -> np.ndarray:
    """a_k with w(t0 + h)/w0 = sum_k a_k u^k from the tree sum with Phi = 1/gamma (a_0 = 1)."""
    a = np.zeros(kmax + 1)
    a[0] = 1.0
    for k in range(1, kmax + 1):
        a[k] = sum(falling_product(t, p) / (sigma(t) * gamma(t)) for t in trees(k))
    return a


def method_coefficients(A: np.ndarray, w: np.ndarray, p: float, kmax: int) -> np.ndarray:
    """c_k with (one step of the method with weights w)/w0 = sum_k c_k u^k (c_0 = 1)."""
    c = np.zeros(kmax + 1)
    c[0] = 1.0
    memo: dict = {}
    for k in range(1, kmax + 1):
        c[k] = sum(float(w @ stage_weights(t, A, memo)) * falling_product(t, p) / sigma(t) for t in trees(k))
    return c


def series(coef: np.ndarray, u: float) -> float:
    return float(sum(ck * u ** k for k, ck in enumerate(coef)))
