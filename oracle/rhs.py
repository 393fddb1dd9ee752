"""Load vectors b_i = int f phi_i (Eq. fe-problem, right-hand side) of the
synthetic sine right-hand side and of any f given as a function, with a
(p+3)-point Gauss rule per direction on each element (on mapped elements: in
the pre-image, f taken at the physical points, the weights carrying det J);
and the load vector with inhomogeneous Dirichlet data imposed weakly by SIPG
(the boundary terms that u = g moves to the right-hand side).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .dg import DGSpace


def sine_f(amps, waves, pts: np.ndarray) -> np.ndarray:
    out = np.zeros(len(pts))
    for a, k in zip(amps, waves):
        term = np.full(len(pts), float(a))
        for d in range(pts.shape[1]):
            term *= np.sin(np.pi * float(k[d]) * pts[:, d])
        out += term
    return out


def load_vector(space: DGSpace, amps, waves) -> np.ndarray:
    b = np.zeros(space.n)
    for k in range(space.topo.n):
        p = int(space.topo.p[k])
        pts, W = space.volume_quadrature(k, p + 3)
        v, _ = space.eval(k, pts)
        b[space.dofs(k)] = v.T @ (W * sine_f(amps, waves, space.phys(pts)))
    return b


def interpolate(space: DGSpace, fn) -> np.ndarray:
    """Nodal interpolant of fn(points) in the DG basis."""
    u = np.zeros(space.n)
    for k in range(space.topo.n):
        u[space.dofs(k)] = fn(space.node_coords(k))
    return u


def load_vector_fn(space: DGSpace, fn, extra: int = 3) -> np.ndarray:
    b = np.zeros(space.n)
    for k in range(space.topo.n):
        p = int(space.topo.p[k])
        pts, W = space.volume_quadrature(k, p + extra)
        v, _ = space.eval(k, pts)
        b[space.dofs(k)] = v.T @ (W * fn(space.phys(pts)))
    return b


def dirichlet_load(space: DGSpace, f_fn, g_fn, eta: float, penalty_form: str = "paper",
                   extra: int = 3) -> np.ndarray:
    """Load vector of -div(a grad u) = f with u = g on the boundary, imposed
    weakly by SIPG (Section 2 with inhomogeneous data): b_i = int f phi_i +
    sum over boundary sub-faces of int g (sigma phi_i - a grad phi_i . n).
    The boundary terms come from replacing [[u]] by u - g on the boundary in
    the consistency and penalty terms; with g = 0 this is load_vector_fn.
    Quadrature: p+extra points per direction (volume), p+extra on each
    boundary sub-face."""
    from .dg import normal_derivative, penalty
    b = load_vector_fn(space, f_fn, extra)
    for f in space.topo.subfaces:
        if f.kp >= 0:
            continue
        k = f.km
        p = int(space.topo.p[k])
        pts, W, n = space.face_quadrature(f, p + extra)
        v, g = space.eval(k, pts)
        gv = g_fn(space.phys(pts))
        sig = penalty(space, f, eta, penalty_form)
        dn = space.coef[k] * normal_derivative(g, n)
        b[space.dofs(k)] += (v.T * W) @ (sig * gv) - (dn.T * W) @ gv
    return b
