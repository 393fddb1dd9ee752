"""The additive subspace-correction preconditioner and PCG (Sections 3.1, 3.3,
3.4, 4.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

B r = P M_C P^T r + sum_e R_e^T A_e^{-1} R_e r + sum_{j in J} r_j / A_jj e_j
(Section 3.1: B = sum_i R_i Q_i with exact solves on V_e and on the 1D spaces
V_j; Section 4.1: B = B_B + B_C).  M_C is either the exact inverse of the LOR
conforming matrix or one V-cycle of the AMG in `amg`.  The simplified variant
B~ = J_B + B_C (Section 4.1) uses point Jacobi on every V_B node.

PCG (Section 4.1): x0 = 0, stop when ||r_k||_2 <= rtol ||b||_2.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp

from . import amg as amg_mod
from .dg import DGSpace, assemble, br2_eta
from .lor import lor_conforming
from .space import E_NODE, I_NODE, J_NODE, ConformingSpace
from .topology import Topology


@dataclasses.dataclass
class Problem:
    topo: Topology
    space: DGSpace
    A: sp.csr_matrix
    cs: ConformingSpace


def build_operator(mesh, form: str = "sipg", eta: Optional[float] = None,
                   penalty_form: str = "paper"):
    """(topology, DG space, sparse A) of a 2D or 3D mesh description."""
    if mesh.dim == 3:
        from .topology3 import Topology3
        topo = Topology3(mesh.lo, mesh.size, mesh.p, mesh.extent)
    else:
        topo = Topology(mesh.lo, mesh.size, mesh.p, mesh.extent)
    corners = getattr(mesh, "corners", None)
    mapping = getattr(mesh, "mapping", None)
    if corners is not None or mapping is not None:
        from .geometry import MappedDGSpace
        space = MappedDGSpace(topo, mesh.lattice_h, corners, getattr(mesh, "coeff", None), mapping=mapping)
    else:
        space = DGSpace(topo, mesh.lattice_h, getattr(mesh, "coeff", None))
    if eta is None:
        eta = br2_eta(topo) if form == "br2" else 100.0
    return topo, space, assemble(space, eta, form=form, penalty_form=penalty_form)


def build_problem(mesh, form: str = "sipg", eta: Optional[float] = None,
                  penalty_form: str = "paper", remark_cases: bool = False) -> Problem:
    topo, space, A = build_operator(mesh, form, eta, penalty_form)
    if mesh.dim == 3:
        from .space3 import ConformingSpaceN
        cs = ConformingSpaceN(space)
    else:
        cs = ConformingSpace(space, remark_cases=remark_cases)
    return Problem(topo, space, A, cs)


class Preconditioner:
    def __init__(self, prob: Problem, lor: str = "amg", smoother: str = "full"):
        self.prob = prob
        A = prob.A
        cs = prob.cs
        self.P = cs.P
        self.Ac = lor_conforming(prob.space, cs.P)
        self.lor = lor
        if lor == "exact":
            self.Ac_inv = np.linalg.inv(self.Ac.toarray())
        else:
            self.levels = amg_mod.setup(self.Ac, amg_mod.THETA3 if prob.space.dim == 3 else amg_mod.THETA)
        diag = A.diagonal()
        kind = cs.kind.copy()
        if smoother == "jacobi_only":
            kind[kind == E_NODE] = J_NODE
            self.blocks = []
        else:
            self.blocks = cs.blocks
        self.jmask = kind == J_NODE
        self.dinv = np.where(self.jmask, 1.0 / diag, 0.0)
        self.block_inv = [np.linalg.inv(A[b][:, b].toarray()) for b in self.blocks]

    def lor_solve(self, rc: np.ndarray) -> np.ndarray:
        if self.lor == "exact":
            return self.Ac_inv @ rc
        return amg_mod.vcycle(self.levels, rc)

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = self.P @ self.lor_solve(self.P.T @ r)
        z = z + self.dinv * r
        for b, Binv in zip(self.blocks, self.block_inv):
            z[b] += Binv @ r[b]
        return z

    def matrix(self) -> np.ndarray:
        n = self.prob.A.shape[0]
        return np.stack([self.apply(e) for e in np.eye(n)], axis=1)


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    rel_res: float
    converged: bool
    history: list


def pcg(A, b: np.ndarray, M: Callable[[np.ndarray], np.ndarray], rtol: float,
        maxit: int) -> SolveResult:
    """Preconditioned conjugate gradients from x0 = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [1.0]
    if bnorm == 0.0:
        return SolveResult(x, 0, 0.0, True, hist)
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if rel <= rtol:
            return SolveResult(x, it, rel, True, hist)
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return SolveResult(x, maxit, hist[-1], False, hist)
