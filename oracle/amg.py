"""Deterministic smoothed-aggregation AMG for the LOR conforming matrix.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper approximates the inverse of the LOR matrix by one V-cycle of
BoomerAMG (Section 3.4 and Section 4.1) without giving its parameters.  This
oracle instead fixes one plain algorithm (the same one the CUDA library sets
up), step by step:

setup(A):
  1. if n <= coarse_max (COARSE_MAX unless a test asks for fewer): coarsest
     level, dense inverse.
  2. strength: j != i is strong for i when a_ij^2 > theta^2 a_ii a_jj
     (theta = THETA on squares, THETA3 on cubes).
  3. aggregation in natural order:
     pass 1: i unaggregated, has a strong neighbour, and all its strong
             neighbours unaggregated -> new aggregate {i} + strong neighbours;
     pass 2: i unaggregated -> joins the aggregate (from pass 1) of its
             lowest-numbered strong neighbour that has one;
     pass 3: i still unaggregated -> new aggregate {i} + its unaggregated
             strong neighbours.
  4. tentative prolongator T (one 1 per row, in the column of the aggregate),
     smoothed: P = (I - omega D^-1 A) T, omega = 4 / (3 rho),
     rho = max_i sum_j |a_ij| / a_ii.
  5. A_c = P^T A P; recurse (stop if the level does not shrink below 0.9 n
     or MAX_LEVELS is reached; the last level is solved densely).
V-cycle(b) on a level with l1-Jacobi smoother d_i = sum_j |a_ij|:
  x = b / d                       (pre-smoothing from zero)
  x = x + P Vcycle_c(P^T (b - A x))
  x = x + (b - A x) / d           (post-smoothing)
which is a symmetric operator.
"""
from __future__ import annotations

from typing import List

import numpy as np
import scipy.sparse as sp

THETA = 0.08          # squares: the Q1 9-point stencil's links are strong
THETA3 = 0.02         # cubes: the trilinear 27-point stencil's links are ~1/32 of the diagonal
COARSE_MAX = 1024
MAX_LEVELS = 12


class Level:
    def __init__(self, A: sp.csr_matrix):
        self.A = A.tocsr()
        self.A.sort_indices()
        self.n = A.shape[0]
        self.d_l1 = np.asarray(abs(self.A).sum(axis=1)).ravel()
        self.P = None
        self.Ainv = None


def strength_lists(A: sp.csr_matrix, theta: float = THETA) -> List[np.ndarray]:
    d = A.diagonal()
    out = []
    for i in range(A.shape[0]):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        keep = [(c, v) for c, v in zip(cols, vals)
                if c != i and v * v > theta * theta * d[i] * d[c]]
        out.append(np.asarray(sorted(c for c, _ in keep), dtype=np.int64))
    return out


def aggregate(A: sp.csr_matrix, theta: float = THETA) -> np.ndarray:
    n = A.shape[0]
    S = strength_lists(A, theta)
    agg = np.full(n, -1, dtype=np.int64)
    na = 0
    for i in range(n):
        if agg[i] < 0 and len(S[i]) > 0 and np.all(agg[S[i]] < 0):
            agg[i] = na
            agg[S[i]] = na
            na += 1
    after1 = agg.copy()
    for i in range(n):
        if agg[i] < 0:
            for j in S[i]:
                if after1[j] >= 0:
                    agg[i] = after1[j]
                    break
    for i in range(n):
        if agg[i] < 0:
            agg[i] = na
            for j in S[i]:
                if agg[j] < 0:
                    agg[j] = na
            na += 1
    return agg


def setup(A: sp.csr_matrix, theta: float = THETA, coarse_max: int = COARSE_MAX) -> List[Level]:
    levels = [Level(A)]
    while True:
        L = levels[-1]
        if L.n <= coarse_max or len(levels) >= MAX_LEVELS:
            break
        agg = aggregate(L.A, theta)
        nc = int(agg.max()) + 1
        if nc >= 0.9 * L.n:
            break
        T = sp.csr_matrix((np.ones(L.n), (np.arange(L.n), agg)), shape=(L.n, nc))
        d = L.A.diagonal()
        rho = float(np.max(np.asarray(abs(L.A).sum(axis=1)).ravel() / d))
        omega = 4.0 / (3.0 * rho)
        S = sp.identity(L.n, format="csr") - omega * sp.diags(1.0 / d) @ L.A
        P = (S @ T).tocsr()
        P.sort_indices()
        L.P = P
        Ac = (P.T @ L.A @ P).tocsr()
        levels.append(Level(Ac))
    last = levels[-1]
    last.Ainv = np.linalg.inv(last.A.toarray())
    return levels


def vcycle(levels: List[Level], b: np.ndarray, lev: int = 0) -> np.ndarray:
    L = levels[lev]
    if L.Ainv is not None:
        return L.Ainv @ b
    x = b / L.d_l1
    r = b - L.A @ x
    x = x + L.P @ vcycle(levels, L.P.T @ r, lev + 1)
    x = x + (b - L.A @ x) / L.d_l1
    return x
