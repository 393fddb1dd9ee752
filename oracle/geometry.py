"""Mapped quadrilateral elements (Section 2: each element kappa carries a map
T_kappa from the reference square onto the element, and V_h is defined by
composing with it).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The mesh is still described by leaf boxes on a dyadic lattice; the boxes
are PRE-IMAGES.  One map Phi of the whole lattice domain [0, Lx] x [0, Ly]
onto a convex quadrilateral, bilinear in the lattice coordinates X and fixed
by the four corner images, carries them to the physical elements:
T_kappa = Phi o (affine map of [0,1]^2 onto the box).  Phi restricted to a
box is again bilinear, so every element is the general (bilinear) image of
the reference square: parallelograms when Phi is affine, general convex
quadrilaterals otherwise.  Lattice lines map to straight lines, so a hanging
sub-face is a straight segment of its master edge on both sides and the
nonconforming structure of the box mesh carries over unchanged.

A caller-supplied smooth map may take Phi's place (curved elements): the
sub-faces are then the images of the lattice segments, curved in general,
and both sides of a sub-face are evaluated at the same pre-image points, so
the hanging structure still matches exactly.

Readings (the paper fixes none of these for non-box elements):
  - quadrature: Gauss-Legendre with p+2 points per direction on the volume
    and max(p-, p+)+2 on a sub-face, in the pre-image coordinates (exact for
    affine Phi; the integrands are rational for a bilinear Phi and
    transcendental for a curved map);
  - the penalty's element size h_kappa = sqrt(|kappa|), the square root of
    the physical area (the edge length for a square), the area taken by the
    element's own volume rule;
  - physical normals n = J^{-T} nu / |J^{-T} nu| with nu the pre-image
    normal, and the arc length ds = |J t| dt along the pre-image tangent t.

Everything below evaluates the map and its Jacobian at points and hands the
DG assembly (dg.assemble) physical gradients, weights and normals; the
assembly itself is the same definition as on boxes.
"""
from __future__ import annotations

import numpy as np

from . import basis
from .dg import DGSpace


class BilinearMap:
    """Phi(X) for X in [0, Lx] x [0, Ly]; corners are the images of (0, 0),
    (Lx, 0), (0, Ly), (Lx, Ly), in that order."""

    def __init__(self, corners, Lx: float, Ly: float):
        c = np.asarray(corners, dtype=np.float64).reshape(4, 2)
        self.c = c
        self.L = (float(Lx), float(Ly))

    def __call__(self, X: np.ndarray) -> np.ndarray:
        s = X[:, 0] / self.L[0]
        t = X[:, 1] / self.L[1]
        w = np.stack([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t], axis=1)
        return w @ self.c

    def jacobian(self, X: np.ndarray) -> np.ndarray:
        """J[m, i, j] = d x_i / d X_j at every point."""
        s = X[:, 0] / self.L[0]
        t = X[:, 1] / self.L[1]
        ds = np.stack([-(1 - t), 1 - t, -t, t], axis=1) / self.L[0]     # d w / d X
        dt = np.stack([-(1 - s), -s, 1 - s, s], axis=1) / self.L[1]     # d w / d Y
        J = np.empty((len(X), 2, 2))
        J[:, :, 0] = ds @ self.c
        J[:, :, 1] = dt @ self.c
        return J


class MappedDGSpace(DGSpace):
    """DG space on the images of the lattice boxes under a bilinear map.

    Quadrature points handed around (eval, volume_quadrature,
    face_quadrature) are pre-image points; eval returns PHYSICAL gradients
    and the quadratures return physical weights and normals, so
    dg.assemble and dg.element_rows evaluate the physical bilinear form."""

    qextra = 1   # p+2 (volume) and max(p-, p+)+2 (faces) Gauss points

    def __init__(self, topo, lattice_h: float, corners=None, coef=None, mapping=None):
        """corners: the bilinear map's corner images; or mapping: any map of
        the lattice domain with __call__(X) -> x and jacobian(X) -> J (curved
        elements: the faces are the images of the lattice segments, curved
        in general, with the normal and arc length varying along them)."""
        if int(getattr(topo, "dim", 2)) != 2:
            raise ValueError("mapped elements: squares only")
        super().__init__(topo, lattice_h, coef)
        ext = topo.extent
        if mapping is not None:
            self.map = mapping
        else:
            self.map = BilinearMap(corners, ext[0] * self.lh, ext[1] * self.lh)
            X = np.array([[0.0, 0.0], [ext[0], 0.0], [0.0, ext[1]], [ext[0], ext[1]]]) * self.lh
            if not np.all(np.linalg.det(self.map.jacobian(X)) > 0.0):
                raise ValueError("the corners do not bound a convex, positively oriented quadrilateral")

    def phys(self, pts: np.ndarray) -> np.ndarray:
        return self.map(pts)

    def area(self, k: int) -> float:
        """|kappa| = int det J over the pre-image box by the element's own
        volume rule (p+2 points per direction; exact for a bilinear map, whose
        det J is linear)."""
        pts, W = DGSpace.volume_quadrature(self, k, int(self.topo.p[k]) + 1 + self.qextra)
        return float(W @ np.linalg.det(self.map.jacobian(pts)))

    def hpen(self, k: int) -> float:
        return float(np.sqrt(self.area(k)))

    def node_coords(self, k: int) -> np.ndarray:
        return self.map(DGSpace.node_coords(self, k))

    def eval(self, k: int, pts: np.ndarray):
        val, gX = DGSpace.eval(self, k, pts)             # gradients in X
        Jinv = np.linalg.inv(self.map.jacobian(pts))     # (m, 2, 2)
        # grad_x = J^{-T} grad_X: grad_x[m, a, i] = sum_j Jinv[m, j, i] gX[m, a, j]
        return val, np.einsum("mji,maj->mai", Jinv, gX)

    def volume_quadrature(self, k: int, q: int):
        pts, W = DGSpace.volume_quadrature(self, k, q)
        det = np.linalg.det(self.map.jacobian(pts))
        if not np.all(det > 0.0):
            raise ValueError("the map is not orientation preserving at a quadrature point")
        return pts, W * det

    def face_quadrature(self, f, q: int):
        pts, W, nu = DGSpace.face_quadrature(self, f, q)
        J = self.map.jacobian(pts)
        tang = np.zeros(2)
        tang[1 - f.axis] = 1.0
        W = W * np.linalg.norm(J @ tang, axis=1)
        n = np.einsum("mji,j->mi", np.linalg.inv(J), nu)       # J^{-T} nu
        n /= np.linalg.norm(n, axis=1)[:, None]
        return pts, W, n


def q1_quad_stiffness(V: np.ndarray) -> np.ndarray:
    """Stiffness of the 4 bilinear (Q1) functions on the quadrilateral with
    vertices V (4, 2), corner order (0,0), (1,0), (0,1), (1,1) of its
    reference square, by the 2 x 2 Gauss rule (exact on parallelograms)."""
    x, w = basis.gauss(2)
    K = np.zeros((4, 4))
    for s, ws in zip(x, w):
        for t, wt in zip(x, w):
            dNs = np.array([-(1 - t), 1 - t, -t, t])
            dNt = np.array([-(1 - s), -s, 1 - s, s])
            J = np.array([[dNs @ V[:, 0], dNt @ V[:, 0]], [dNs @ V[:, 1], dNt @ V[:, 1]]])
            G = np.linalg.inv(J).T @ np.stack([dNs, dNt])      # physical gradients (2, 4)
            K += ws * wt * np.linalg.det(J) * (G.T @ G)
    return K


def lor_element_mapped(space: MappedDGSpace, k: int) -> np.ndarray:
    """LOR block of a mapped element (Section 3.4): the Q1 stiffness on the
    images of the cells of the Gauss-Lobatto sub-grid."""
    p = int(space.topo.p[k])
    n = p + 1
    X = DGSpace.node_coords(space, k)          # pre-image sub-grid vertices, local order
    V = space.map(X)
    A = np.zeros((n * n, n * n))
    for j in range(p):
        for i in range(p):
            idx = [j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1]
            A[np.ix_(idx, idx)] += q1_quad_stiffness(V[idx])
    return A
