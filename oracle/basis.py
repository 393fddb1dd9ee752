"""1D polynomial machinery on the reference interval [0, 1] (Section 2.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The nodal basis of Section 2.2 is the Lagrange basis at the p+1 Gauss-Lobatto
points.  Exact integration uses Gauss-Legendre rules.  Everything here is the
textbook definition written out; numpy's Legendre module supplies roots and
Gauss-Legendre rules as library primitives.
"""
from __future__ import annotations

import functools

import numpy as np
from numpy.polynomial import legendre as L


@functools.lru_cache(maxsize=None)
def gll_nodes(p: int) -> np.ndarray:
    """p+1 Gauss-Lobatto points on [0,1]: the endpoints and the roots of P_p'."""
    if p < 1:
        raise ValueError("p >= 1")
    interior = np.sort(L.Legendre.basis(p).deriv().roots().real) if p > 1 else np.zeros(0)
    x = np.concatenate([[-1.0], interior, [1.0]])
    return 0.5 * (x + 1.0)


@functools.lru_cache(maxsize=None)
def gll_weights(p: int) -> np.ndarray:
    """Gauss-Lobatto weights on [0,1]: w_i = 1 / (p (p+1) P_p(x_i)^2) (x on [-1,1])."""
    x = 2.0 * gll_nodes(p) - 1.0
    pp = L.legval(x, [0] * p + [1])
    return 1.0 / (p * (p + 1) * pp * pp)


@functools.lru_cache(maxsize=None)
def gauss(q: int):
    """q-point Gauss-Legendre rule on [0,1] (exact for degree 2q-1)."""
    x, w = L.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange(nodes: np.ndarray, x) -> np.ndarray:
    """Values l_i(x) of the Lagrange polynomials on `nodes`; shape (len(x), n)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                out[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return out


def lagrange_deriv(nodes: np.ndarray, x) -> np.ndarray:
    """Derivatives l_i'(x) by the product rule; shape (len(x), n)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(x), n))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[k]))
            for j in range(n):
                if j != i and j != k:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            out[:, i] += term
    return out
