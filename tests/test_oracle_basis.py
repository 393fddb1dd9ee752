"""Pins of the oracle's 1D basis (Section 2.2) against closed forms."""
import os

import numpy as np
import pytest

from oracle import basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    out = {}
    for p, x, w in rows:
        out.setdefault(int(p), []).append((float(x), float(w)))
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_closed_forms(p):
    g = _golden()[p]
    np.testing.assert_allclose(basis.gll_nodes(p), [x for x, _ in g], rtol=0, atol=1e-15)
    np.testing.assert_allclose(basis.gll_weights(p), [w for _, w in g], rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 11))
def test_gll_rule_exactness(p):
    # Gauss-Lobatto with p+1 points integrates degree 2p-1 exactly on [0,1]
    x, w = basis.gll_nodes(p), basis.gll_weights(p)
    for deg in range(2 * p):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 1e-14
    assert abs(np.sum(w * x ** (2 * p)) - 1.0 / (2 * p + 1)) > 1e-13


@pytest.mark.parametrize("q", range(1, 12))
def test_gauss_exactness(q):
    x, w = basis.gauss(q)
    for deg in range(2 * q):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 1e-14


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_cardinal_and_derivative(p):
    g = basis.gll_nodes(p)
    np.testing.assert_allclose(basis.lagrange(g, g), np.eye(p + 1), atol=1e-13)
    # derivative against a central difference of the values
    x = np.linspace(0.05, 0.95, 7)
    eps = 1e-6
    fd = (basis.lagrange(g, x + eps) - basis.lagrange(g, x - eps)) / (2 * eps)
    np.testing.assert_allclose(basis.lagrange_deriv(g, x), fd, atol=1e-6 * (p + 1) ** 3)
    # partition of unity: sum of values 1, sum of derivatives 0
    np.testing.assert_allclose(basis.lagrange(g, x).sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(basis.lagrange_deriv(g, x).sum(axis=1), 0.0, atol=1e-10)
