"""Load vector b_i = int f phi_i of the synthetic sine right-hand side
(Eq. fe-problem, right-hand side), with a (p+3)-point Gauss rule per
direction on each element (on mapped elements: in the pre-image, f taken at
the physical points, the weights carrying det J)."""
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
