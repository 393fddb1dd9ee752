"""Explicit assembly of the 2D DG stiffness matrix (Section 2, Eq. fe-problem;
BR2 form of Section 4.4).

Global numbering: element-major, element k owns (p_k+1)^2 consecutive DOFs;
inside an element the nodal DOF (ix, iy) has local index iy*(p+1) + ix, with
the Gauss-Lobatto nodes of Section 2.2 in each direction.

Quadrature (exact on axis-aligned squares): Gauss-Legendre with p+1 points per
direction for the volume, max(p-, p+)+1 points on every sub-face.

Sign convention: the paper writes Laplace(u) = f; this oracle solves
-Laplace(u) = f so that the matrix is SPD (the two differ by f -> -f).

A[i, j] = a(phi_j, phi_i) with
  a(u, v) = int grad u . grad v
            - int_G {grad u}.[[v]] - int_G {grad v}.[[u]] + stabilisation
SIPG stabilisation: int_G sigma [[u]].[[v]], sigma = eta p_e^2 / h_e with
p_e = max, h_e = min over the two sides ("paper" form), or
sigma = eta (p_e + 1)^2 / h_e ("p1sq" form of the 8x8 p=2 workload).
BR2 stabilisation: sum_e int eta r_e([[u]]) . r_e([[v]]), with the lifting
int r_e(phi).tau = -int_e phi.{tau} solved with each adjacent element's exact
mass matrix; on a boundary sub-face {tau} = tau.
On the boundary (homogeneous Dirichlet): [[u]] = u n, {grad u} = grad u.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import numpy as np
import scipy.sparse as sp

from . import basis
from .topology import Topology


class DGSpace:
    def __init__(self, topo: Topology, lattice_h: float):
        self.topo = topo
        self.lh = float(lattice_h)
        p = topo.p
        self.ndof_elem = (p + 1) ** 2
        self.offset = np.zeros(topo.n + 1, dtype=np.int64)
        self.offset[1:] = np.cumsum(self.ndof_elem)
        self.n = int(self.offset[-1])

    def h(self, k: int) -> float:
        return float(self.topo.size[k]) * self.lh

    def origin(self, k: int) -> np.ndarray:
        return self.topo.lo[k].astype(np.float64) * self.lh

    def node_coords(self, k: int) -> np.ndarray:
        """Physical coordinates of the (p+1)^2 nodes, local order."""
        p = int(self.topo.p[k])
        g = basis.gll_nodes(p)
        X, Y = np.meshgrid(g, g)          # Y varies along rows -> iy outer
        o = self.origin(k)
        h = self.h(k)
        return np.stack([o[0] + h * X.ravel(), o[1] + h * Y.ravel()], axis=1)

    def eval(self, k: int, pts: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        """Basis values (npts, nloc) and physical gradients (npts, nloc, 2)."""
        p = int(self.topo.p[k])
        g = basis.gll_nodes(p)
        h = self.h(k)
        o = self.origin(k)
        xi = (pts[:, 0] - o[0]) / h
        et = (pts[:, 1] - o[1]) / h
        lx, ly = basis.lagrange(g, xi), basis.lagrange(g, et)
        dx, dy = basis.lagrange_deriv(g, xi), basis.lagrange_deriv(g, et)
        # local index iy*(p+1)+ix  ->  outer product ly[:, iy] * lx[:, ix]
        val = (ly[:, :, None] * lx[:, None, :]).reshape(len(pts), -1)
        gx = (ly[:, :, None] * dx[:, None, :]).reshape(len(pts), -1) / h
        gy = (dy[:, :, None] * lx[:, None, :]).reshape(len(pts), -1) / h
        return val, np.stack([gx, gy], axis=2)

    def volume_quadrature(self, k: int, q: int) -> Tuple[np.ndarray, np.ndarray]:
        x, w = basis.gauss(q)
        X, Y = np.meshgrid(x, x)
        W = np.outer(w, w).ravel()
        o = self.origin(k)
        h = self.h(k)
        pts = np.stack([o[0] + h * X.ravel(), o[1] + h * Y.ravel()], axis=1)
        return pts, W * h * h

    def face_quadrature(self, f, q: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Points, weights (with the length) and unit normal of a sub-face."""
        x, w = basis.gauss(q)
        t = (f.t0 + (f.t1 - f.t0) * x) * self.lh
        c = np.full(q, f.c * self.lh)
        pts = np.stack([c, t], axis=1) if f.axis == 0 else np.stack([t, c], axis=1)
        n = np.zeros(2)
        n[f.axis] = f.normal_sign
        return pts, w * (f.t1 - f.t0) * self.lh, n

    def mass(self, k: int) -> np.ndarray:
        p = int(self.topo.p[k])
        pts, W = self.volume_quadrature(k, p + 1)
        v, _ = self.eval(k, pts)
        return v.T @ (W[:, None] * v)

    def dofs(self, k: int) -> np.ndarray:
        return np.arange(self.offset[k], self.offset[k + 1])


def penalty(space: DGSpace, f, eta: float, form: str) -> float:
    t = space.topo
    if f.kp >= 0:
        pe = max(int(t.p[f.km]), int(t.p[f.kp]))
        he = min(space.h(f.km), space.h(f.kp))
    else:
        pe, he = int(t.p[f.km]), space.h(f.km)
    if form == "paper":
        return eta * pe * pe / he
    if form == "p1sq":
        return eta * (pe + 1) ** 2 / he
    raise ValueError(form)


def assemble(space: DGSpace, eta: float, form: str = "sipg",
             penalty_form: str = "paper", broken_only: bool = False) -> sp.csr_matrix:
    """Sparse DG matrix.  form: "sipg" or "br2".  broken_only: the broken
    Laplacian A-hat of Section 3.4 (volume terms only)."""
    topo = space.topo
    rows, cols, vals = [], [], []

    def add(ri, ci, block):
        R, C = np.meshgrid(ri, ci, indexing="ij")
        rows.append(R.ravel())
        cols.append(C.ravel())
        vals.append(block.ravel())

    for k in range(topo.n):
        p = int(topo.p[k])
        pts, W = space.volume_quadrature(k, p + 1)
        _, g = space.eval(k, pts)
        K = np.einsum("qa,qb,q->ab", g[:, :, 0], g[:, :, 0], W) + \
            np.einsum("qa,qb,q->ab", g[:, :, 1], g[:, :, 1], W)
        add(space.dofs(k), space.dofs(k), K)

    if not broken_only:
        for f in topo.subfaces:
            sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
            q = max(int(topo.p[k]) for k in sides) + 1
            pts, W, n = space.face_quadrature(f, q)
            interior = f.kp >= 0
            jump_parts, avg_parts, idx = [], [], []
            for si, k in enumerate(sides):
                v, g = space.eval(k, pts)
                sgn = 1.0 if si == 0 else -1.0
                jump_parts.append(sgn * v)                 # [[phi]] . n
                dn = g @ n                                  # grad phi . n
                avg_parts.append((0.5 if interior else 1.0) * dn)
                idx.append(space.dofs(k))
            J = np.concatenate(jump_parts, axis=1)        # (q, nloc)
            D = np.concatenate(avg_parts, axis=1)
            I = np.concatenate(idx)
            # rows: test function v (index a), cols: trial u (index b)
            F = -(J.T * W) @ D - (D.T * W) @ J
            if form == "sipg":
                F = F + penalty(space, f, eta, penalty_form) * ((J.T * W) @ J)
            elif form == "br2":
                coef = 0.25 if interior else 1.0
                for si, k in enumerate(sides):
                    v, _ = space.eval(k, pts)
                    b = (v.T * W) @ J                       # b[i, a] = int_e phi_i^k j_a
                    Minv = np.linalg.inv(space.mass(k))
                    F = F + eta * coef * (b.T @ Minv @ b)
            else:
                raise ValueError(form)
            add(I, I, F)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(space.n, space.n)).tocsr()
    A.sum_duplicates()
    return A


def br2_eta(topo: Topology) -> float:
    """Default BR2 penalty: the largest number of sub-faces of one element."""
    count = np.zeros(topo.n, dtype=np.int64)
    for f in topo.subfaces:
        count[f.km] += 1
        if f.kp >= 0:
            count[f.kp] += 1
    return float(count.max())


def element_rows(space: DGSpace, k: int, x: np.ndarray, eta: float, form: str = "sipg",
                 penalty_form: str = "paper") -> np.ndarray:
    """(A x) restricted to the DOFs of element k, assembling only the volume
    term of k and the sub-faces touching k (same definitions as `assemble`);
    used to check sampled outputs of very large meshes."""
    topo = space.topo
    p = int(topo.p[k])
    pts, W = space.volume_quadrature(k, p + 1)
    _, g = space.eval(k, pts)
    K = np.einsum("qa,qb,q->ab", g[:, :, 0], g[:, :, 0], W) + \
        np.einsum("qa,qb,q->ab", g[:, :, 1], g[:, :, 1], W)
    y = K @ x[space.dofs(k)]
    for f in topo.faces_of(k):
        sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
        q = max(int(topo.p[e]) for e in sides) + 1
        fpts, FW, n = space.face_quadrature(f, q)
        interior = f.kp >= 0
        J, D, I = [], [], []
        for si, e in enumerate(sides):
            v, gg = space.eval(e, fpts)
            J.append((1.0 if si == 0 else -1.0) * v)
            D.append((0.5 if interior else 1.0) * (gg @ n))
            I.append(space.dofs(e))
        Jm, Dm, Im = np.concatenate(J, axis=1), np.concatenate(D, axis=1), np.concatenate(I)
        F = -(Jm.T * FW) @ Dm - (Dm.T * FW) @ Jm
        if form == "sipg":
            F = F + penalty(space, f, eta, penalty_form) * ((Jm.T * FW) @ Jm)
        else:
            coef = 0.25 if interior else 1.0
            for e in sides:
                v, _ = space.eval(e, fpts)
                b = (v.T * FW) @ Jm
                F = F + eta * coef * (b.T @ np.linalg.inv(space.mass(e)) @ b)
        rows = slice(0, (p + 1) ** 2) if f.km == k else slice(len(I[0]), len(I[0]) + (p + 1) ** 2)
        y = y + F[rows] @ x[Im]
    return y
