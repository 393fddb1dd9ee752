"""Pins of the oracle's smoothed-aggregation AMG (the LOR solve of Section 3.4,
one V-cycle as in Section 4.1) against hand-worked aggregations and the
error-propagation form of a symmetric multigrid cycle.

The golden cases in tests/golden/amg_aggregation.txt were worked by hand; their
comments give the working."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "amg_aggregation.txt")


def _golden():
    agg, P = {}, {}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "agg":
            agg[f[1]] = [int(v) for v in f[2:]]
        elif f[0] == "P":
            P.setdefault(f[1], []).append((int(f[2]), int(f[3]), Fraction(int(f[4]), int(f[5]))))
    return agg, P


def _chain(strong37: bool) -> sp.csr_matrix:
    A = 4.0 * np.eye(9)
    for i, j in [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (1, 6), (4, 6), (4, 8)]:
        A[i, j] = A[j, i] = -1.0
    A[3, 7] = A[7, 3] = -0.35 if strong37 else -0.3
    return sp.csr_matrix(A)


def _q1_interior(n: int = 5) -> sp.csr_matrix:
    """Q1 stiffness of the n x n interior nodes of an (n+1)^2 grid of unit
    squares: 8/3 on the diagonal, -1/3 to each edge or diagonal neighbour."""
    N = n * n
    A = np.zeros((N, N))
    for j in range(n):
        for i in range(n):
            r = j * n + i
            A[r, r] = 8.0 / 3.0
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    if (di or dj) and 0 <= i + di < n and 0 <= j + dj < n:
                        A[r, (j + dj) * n + i + di] = -1.0 / 3.0
    return sp.csr_matrix(A)


@pytest.mark.parametrize("case", ["chain", "chain_strong37", "q1"])
def test_aggregation_matches_hand_worked(case):
    agg, _ = _golden()
    A = {"chain": _chain(False), "chain_strong37": _chain(True), "q1": _q1_interior()}[case]
    got = amg.aggregate(A, amg.THETA)
    assert got.tolist() == agg[case]


def test_prolongator_matches_hand_worked():
    _, P = _golden()
    levels = amg.setup(_q1_interior(), amg.THETA, coarse_max=4)
    assert len(levels) == 2 and levels[1].n == 4
    Pm = levels[0].P.toarray()
    for row, col, val in P["q1"]:
        assert abs(Pm[row, col] - float(val)) < 1e-15, (row, col, Pm[row, col], val)
    # interior rows of D^-1 A sum to zero, so those rows of P sum to one
    assert abs(Pm[12].sum() - 1.0) < 1e-15


def _error_propagation(levels, lev=0):
    """I - M A of the V-cycle below level `lev`, written as the product of
    its stages' error propagators: S (I - P M_c P^T A) S with the l1-Jacobi
    step S = I - D^-1 A and M_c the cycle on the next level (the exact
    inverse on the coarsest)."""
    L = levels[lev]
    A = L.A.toarray()
    n = L.n
    if L.Ainv is not None:
        return np.eye(n) - L.Ainv @ A
    S = np.eye(n) - A / L.d_l1[:, None]
    P = L.P.toarray()
    Ac = levels[lev + 1].A.toarray()
    Ec = _error_propagation(levels, lev + 1)
    Mc = (np.eye(Ac.shape[0]) - Ec) @ np.linalg.inv(Ac)
    return S @ (np.eye(n) - P @ Mc @ P.T @ A) @ S


def test_vcycle_error_propagation_form():
    # three levels on a 2D Poisson matrix; the V-cycle as the oracle runs it
    # must equal the composition of its smoothing and coarse-correction steps
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(12, 12))
    A = (sp.kron(sp.identity(12), T) + sp.kron(T, sp.identity(12))).tocsr()
    levels = amg.setup(A, amg.THETA, coarse_max=20)
    assert len(levels) >= 3
    n = A.shape[0]
    M = np.stack([amg.vcycle(levels, e) for e in np.eye(n)], axis=1)
    E = _error_propagation(levels)
    np.testing.assert_allclose(np.eye(n) - M @ A.toarray(), E, atol=1e-12)


def test_isolated_rows_become_singletons():
    # a diagonal matrix has no strong links: pass 3 makes every node its own
    # aggregate, which stops the coarsening (no shrinkage)
    A = sp.diags(np.arange(1.0, 7.0)).tocsr()
    assert amg.aggregate(A).tolist() == [0, 1, 2, 3, 4, 5]
    assert len(amg.setup(A, coarse_max=2)) == 1
