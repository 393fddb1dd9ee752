"""Low-order-refined matrices (Section 3.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For element k of degree p the LOR element matrix is the (bi/tri)linear (Q1)
finite element stiffness matrix on the Cartesian sub-mesh whose vertices are
the (p+1)^d Gauss-Lobatto nodes of k.  A-tilde is block diagonal with these
blocks (on the DG numbering); the LOR conforming matrix is P^T A-tilde P.
Each Q1 sub-cell matrix is integrated here with a 2^d Gauss rule from the
Q1 shape functions (exact for the Q1 stiffness).  On mapped elements the
sub-cells are the images of the Gauss-Lobatto cells (geometry.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis
from .dg import DGSpace


def q1_cell_stiffness(a: float, b: float) -> np.ndarray:
    """Stiffness of the 4 bilinear functions on an a x b rectangle, corner
    order (0,0), (1,0), (0,1), (1,1)."""
    x, w = basis.gauss(2)
    K = np.zeros((4, 4))
    for gx, wx in zip(x, w):
        for gy, wy in zip(x, w):
            # shape functions N = Nx(s) Ny(t) with Nx in {1-s, s}
            dNx = np.array([-1.0, 1.0]) / a
            Nx = np.array([1.0 - gx, gx])
            dNy = np.array([-1.0, 1.0]) / b
            Ny = np.array([1.0 - gy, gy])
            gxv = np.array([dNx[i] * Ny[j] for j in range(2) for i in range(2)])
            gyv = np.array([Nx[i] * dNy[j] for j in range(2) for i in range(2)])
            K += wx * wy * a * b * (np.outer(gxv, gxv) + np.outer(gyv, gyv))
    return K


def q1_cell_stiffness3(a: float, b: float, c: float) -> np.ndarray:
    """Stiffness of the 8 trilinear functions on an a x b x c box, corner
    order x fastest: (0,0,0), (1,0,0), (0,1,0), ..., (1,1,1)."""
    x, w = basis.gauss(2)
    K = np.zeros((8, 8))
    for gx, wx in zip(x, w):
        for gy, wy in zip(x, w):
            for gz, wz in zip(x, w):
                N = [np.array([1.0 - g, g]) for g in (gx, gy, gz)]
                dN = [np.array([-1.0, 1.0]) / e for e in (a, b, c)]
                corners = [(i, j, k) for k in range(2) for j in range(2) for i in range(2)]
                G = np.array([[dN[0][i] * N[1][j] * N[2][k], N[0][i] * dN[1][j] * N[2][k],
                               N[0][i] * N[1][j] * dN[2][k]] for (i, j, k) in corners])
                K += wx * wy * wz * a * b * c * (G @ G.T)
    return K


def lor_element(p: int, h: float = 1.0, dim: int = 2) -> np.ndarray:
    g = basis.gll_nodes(p) * h
    n = p + 1
    if dim == 3:
        A = np.zeros((n ** 3, n ** 3))
        for kz in range(p):
            for j in range(p):
                for i in range(p):
                    K = q1_cell_stiffness3(g[i + 1] - g[i], g[j + 1] - g[j], g[kz + 1] - g[kz])
                    idx = [(kz + dz) * n * n + (j + dy) * n + i + dx
                           for dz in range(2) for dy in range(2) for dx in range(2)]
                    A[np.ix_(idx, idx)] += K
        return A
    A = np.zeros((n * n, n * n))
    for j in range(p):
        for i in range(p):
            K = q1_cell_stiffness(g[i + 1] - g[i], g[j + 1] - g[j])
            idx = [j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1]
            A[np.ix_(idx, idx)] += K
    return A


def assemble_lor(space: DGSpace) -> sp.csr_matrix:
    """Block-diagonal A-tilde; element k's block is scaled by its coefficient
    a_k, so that A-tilde discretises the same -div(a grad u) as A."""
    blocks = []
    mapped = hasattr(space, "map")
    if mapped:
        from .geometry import lor_element_mapped
    for k in range(space.topo.n):
        if mapped:
            blocks.append(space.coef[k] * lor_element_mapped(space, k))
        else:
            blocks.append(space.coef[k] * lor_element(int(space.topo.p[k]), space.h(k), space.dim))
    return sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr")


def lor_conforming(space: DGSpace, P: sp.csr_matrix) -> sp.csr_matrix:
    At = assemble_lor(space)
    Ac = (P.T @ At @ P).tocsr()
    Ac.sum_duplicates()
    Ac.sort_indices()
    return Ac
