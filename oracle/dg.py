"""Explicit assembly of the DG stiffness matrix (Section 2, Eq. fe-problem;
BR2 form of Section 4.4), on squares (2D) or cubes (3D).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Global numbering: element-major, element k owns (p_k+1)^d consecutive DOFs;
inside an element the nodal DOF (ix, iy[, iz]) has local index
ix + (p+1) iy [+ (p+1)^2 iz], with the Gauss-Lobatto nodes of Section 2.2 in
each direction.

Quadrature (exact on axis-aligned boxes): Gauss-Legendre with p+1 points per
direction for the volume, max(p-, p+)+1 points per tangential direction on
every sub-face.

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
mass matrix; on a boundary sub-face {tau} = tau.  With a coefficient a, both
sides' lifting energies of a sub-face carry the larger a of its two sides
(like the SIPG penalty).
On the boundary (homogeneous Dirichlet): [[u]] = u n, {grad u} = grad u.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import numpy as np
import scipy.sparse as sp

from . import basis
from .topology import Topology


class DGSpace:
    # quadrature points beyond the exact box rule (mapped elements: 1)
    qextra = 0

    def __init__(self, topo: Topology, lattice_h: float, coef=None):
        self.topo = topo
        self.dim = int(getattr(topo, "dim", 2))
        self.lh = float(lattice_h)
        # piecewise-constant diffusion coefficient a, one value per element
        # (the random-refinement problem of Section 4.3); None means a = 1
        self.coef = (np.ones(topo.n) if coef is None
                     else np.asarray(coef, dtype=np.float64).reshape(topo.n).copy())
        p = topo.p
        self.ndof_elem = (p + 1) ** self.dim
        self.offset = np.zeros(topo.n + 1, dtype=np.int64)
        self.offset[1:] = np.cumsum(self.ndof_elem)
        self.n = int(self.offset[-1])

    def h(self, k: int) -> float:
        return float(self.topo.size[k]) * self.lh

    def hpen(self, k: int) -> float:
        """Element size h_kappa of the SIPG penalty (the edge length)."""
        return self.h(k)

    def phys(self, pts: np.ndarray) -> np.ndarray:
        """Physical coordinates of quadrature points (boxes: the points)."""
        return pts

    def origin(self, k: int) -> np.ndarray:
        return self.topo.lo[k].astype(np.float64) * self.lh

    def node_coords(self, k: int) -> np.ndarray:
        """Physical coordinates of the (p+1)^d nodes, local order."""
        p = int(self.topo.p[k])
        g = basis.gll_nodes(p)
        if self.dim == 3:
            Z, Y, X = np.meshgrid(g, g, g, indexing="ij")   # iz outer, ix inner
            o = self.origin(k)
            h = self.h(k)
            return np.stack([o[0] + h * X.ravel(), o[1] + h * Y.ravel(), o[2] + h * Z.ravel()], axis=1)
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
        if self.dim == 3:
            l = [basis.lagrange(g, (pts[:, d] - o[d]) / h) for d in range(3)]
            dl = [basis.lagrange_deriv(g, (pts[:, d] - o[d]) / h) for d in range(3)]
            m = len(pts)

            def prod(fx, fy, fz):   # local index iz*(p+1)^2 + iy*(p+1) + ix
                return (fz[:, :, None, None] * fy[:, None, :, None] * fx[:, None, None, :]).reshape(m, -1)
            val = prod(l[0], l[1], l[2])
            grad = np.stack([prod(dl[0], l[1], l[2]) / h, prod(l[0], dl[1], l[2]) / h,
                             prod(l[0], l[1], dl[2]) / h], axis=2)
            return val, grad
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
        if self.dim == 3:
            Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
            W = np.einsum("a,b,c->abc", w, w, w).ravel()
            o = self.origin(k)
            h = self.h(k)
            pts = np.stack([o[0] + h * X.ravel(), o[1] + h * Y.ravel(), o[2] + h * Z.ravel()], axis=1)
            return pts, W * h ** 3
        X, Y = np.meshgrid(x, x)
        W = np.outer(w, w).ravel()
        o = self.origin(k)
        h = self.h(k)
        pts = np.stack([o[0] + h * X.ravel(), o[1] + h * Y.ravel()], axis=1)
        return pts, W * h * h

    def face_quadrature(self, f, q: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Points, weights (with the length / area) and unit normal of a sub-face."""
        x, w = basis.gauss(q)
        if self.dim == 3:
            (a, b), (l0, l1), (h0, h1) = f.ta, f.lo, f.hi
            U, T = np.meshgrid(x, x, indexing="ij")        # second tangential axis outer
            pts = np.zeros((q * q, 3))
            pts[:, f.axis] = f.c * self.lh
            pts[:, a] = (l0 + (h0 - l0) * T.ravel()) * self.lh
            pts[:, b] = (l1 + (h1 - l1) * U.ravel()) * self.lh
            n = np.zeros(3)
            n[f.axis] = f.normal_sign
            return pts, np.outer(w, w).ravel() * (h0 - l0) * (h1 - l1) * self.lh ** 2, n
        t = (f.t0 + (f.t1 - f.t0) * x) * self.lh
        c = np.full(q, f.c * self.lh)
        pts = np.stack([c, t], axis=1) if f.axis == 0 else np.stack([t, c], axis=1)
        n = np.zeros(2)
        n[f.axis] = f.normal_sign
        return pts, w * (f.t1 - f.t0) * self.lh, n

    def mass(self, k: int) -> np.ndarray:
        p = int(self.topo.p[k])
        pts, W = self.volume_quadrature(k, p + 1 + self.qextra)
        v, _ = self.eval(k, pts)
        return v.T @ (W[:, None] * v)

    def dofs(self, k: int) -> np.ndarray:
        return np.arange(self.offset[k], self.offset[k + 1])


def normal_derivative(g: np.ndarray, n: np.ndarray) -> np.ndarray:
    """grad phi . n at every point, for one normal (boxes) or one per point
    (mapped elements): g (npts, nloc, d), n (d,) or (npts, d)."""
    if n.ndim == 1:
        return g @ n
    return np.einsum("qid,qd->qi", g, n)


def penalty(space: DGSpace, f, eta: float, form: str) -> float:
    """SIPG penalty of a sub-face (Section 2): eta p_e^2 / h_e with p_e the
    larger degree and h_e the smaller size of the two sides, times the larger
    coefficient of the two sides."""
    t = space.topo
    if f.kp >= 0:
        pe = max(int(t.p[f.km]), int(t.p[f.kp]))
        he = min(space.hpen(f.km), space.hpen(f.kp))
        ae = max(space.coef[f.km], space.coef[f.kp])
    else:
        pe, he, ae = int(t.p[f.km]), space.hpen(f.km), space.coef[f.km]
    if form == "paper":
        return ae * eta * pe * pe / he
    if form == "p1sq":
        return ae * eta * (pe + 1) ** 2 / he
    raise ValueError(form)


def assemble(space: DGSpace, eta: float, form: str = "sipg",
             penalty_form: str = "paper", broken_only: bool = False) -> sp.csr_matrix:
    """Sparse DG matrix of -div(a grad u) = f.  form: "sipg" or "br2".
    broken_only: the broken Laplacian A-hat of Section 3.4 (volume terms only).
    With a coefficient a: a_k on the volume term of element k, the face
    averages of a grad u, the SIPG penalty times the larger a of the two sides,
    and both sides' BR2 lifting energies times that same larger a."""
    topo = space.topo
    rows, cols, vals = [], [], []

    def add(ri, ci, block):
        R, C = np.meshgrid(ri, ci, indexing="ij")
        rows.append(R.ravel())
        cols.append(C.ravel())
        vals.append(block.ravel())

    for k in range(topo.n):
        p = int(topo.p[k])
        pts, W = space.volume_quadrature(k, p + 1 + space.qextra)
        _, g = space.eval(k, pts)
        K = sum((g[:, :, d].T * W) @ g[:, :, d] for d in range(space.dim))
        add(space.dofs(k), space.dofs(k), space.coef[k] * K)

    if not broken_only:
        for f in topo.subfaces:
            sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
            q = max(int(topo.p[k]) for k in sides) + 1 + space.qextra
            pts, W, n = space.face_quadrature(f, q)
            interior = f.kp >= 0
            jump_parts, avg_parts, idx = [], [], []
            for si, k in enumerate(sides):
                v, g = space.eval(k, pts)
                sgn = 1.0 if si == 0 else -1.0
                jump_parts.append(sgn * v)                 # [[phi]] . n
                dn = normal_derivative(g, n)                # grad phi . n
                avg_parts.append((0.5 if interior else 1.0) * space.coef[k] * dn)   # {a grad phi} . n
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
                ae = max(space.coef[k] for k in sides)     # the larger a of the sub-face
                for si, k in enumerate(sides):
                    v, _ = space.eval(k, pts)
                    b = (v.T * W) @ J                       # b[i, a] = int_e phi_i^k j_a
                    Minv = np.linalg.inv(space.mass(k))
                    F = F + eta * coef * ae * (b.T @ Minv @ b)
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
    pts, W = space.volume_quadrature(k, p + 1 + space.qextra)
    _, g = space.eval(k, pts)
    K = sum((g[:, :, d].T * W) @ g[:, :, d] for d in range(space.dim))
    y = space.coef[k] * (K @ x[space.dofs(k)])
    for f in topo.faces_of(k):
        sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
        q = max(int(topo.p[e]) for e in sides) + 1 + space.qextra
        fpts, FW, n = space.face_quadrature(f, q)
        interior = f.kp >= 0
        J, D, I = [], [], []
        for si, e in enumerate(sides):
            v, gg = space.eval(e, fpts)
            J.append((1.0 if si == 0 else -1.0) * v)
            D.append((0.5 if interior else 1.0) * space.coef[e] * normal_derivative(gg, n))
            I.append(space.dofs(e))
        Jm, Dm, Im = np.concatenate(J, axis=1), np.concatenate(D, axis=1), np.concatenate(I)
        F = -(Jm.T * FW) @ Dm - (Dm.T * FW) @ Jm
        if form == "sipg":
            F = F + penalty(space, f, eta, penalty_form) * ((Jm.T * FW) @ Jm)
        else:
            coef = 0.25 if interior else 1.0
            ae = max(space.coef[e] for e in sides)
            for e in sides:
                v, _ = space.eval(e, fpts)
                b = (v.T * FW) @ Jm
                F = F + eta * coef * ae * (b.T @ np.linalg.inv(space.mass(e)) @ b)
        nk = (p + 1) ** space.dim
        rows = slice(0, nk) if f.km == k else slice(len(I[0]), len(I[0]) + nk)
        y = y + F[rows] @ x[Im]
    return y
