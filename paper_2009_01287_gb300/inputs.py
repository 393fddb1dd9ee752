"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws meshes (leaf boxes
on an integer dyadic lattice, with a polynomial degree per leaf) and the
parameters of the right-hand side.  Everything that discretises or solves lives
elsewhere.

Mesh description (dimension d = 2 or 3):
    lo    int32 (n, d)  lower corner of each leaf in lattice units
    size  int32 (n,)    edge length in lattice units (a power of two)
    p     int32 (n,)    polynomial degree of the leaf
    extent int tuple    domain [0, extent_0] x ... in lattice units
    lattice_h float     physical length of one lattice unit

Refinement process (random-refinement experiment of Section 4.3, with the
probability / depth of the synthetic workloads): every base cell is refined
recursively; a cell at depth < max_depth is split into 2^d children with
probability `prob`, children visited in Morton (x-fastest) order; one PCG64
stream per mesh seed, all coin flips first, then the degrees.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class MeshDesc:
    dim: int
    lo: np.ndarray          # int32 (n, dim)
    size: np.ndarray        # int32 (n,)
    p: np.ndarray           # int32 (n,)
    extent: Tuple[int, ...]  # lattice units per axis
    lattice_h: float
    # float64 (n,) piecewise-constant diffusion coefficient a per leaf, or
    # None for a = 1
    coeff: Optional[np.ndarray] = None
    # float64 (4, 2) images of the lattice domain's corners (0, 0), (X, 0),
    # (0, Y), (X, Y) under the bilinear map that carries the leaf boxes to
    # quadrilaterals, or None for the boxes themselves (squares only)
    corners: Optional[np.ndarray] = None
    # or a smooth map of the lattice domain (curved elements): an object with
    # __call__(X) -> x and jacobian(X) -> J, J[m, i, j] = d x_i / d X_j
    mapping: Optional[object] = None

    @property
    def n_elems(self) -> int:
        return int(self.size.shape[0])

    def n_dofs(self) -> int:
        return int(np.sum((self.p.astype(np.int64) + 1) ** self.dim))


@dataclasses.dataclass
class SineRHS:
    """f(x) = sum_m a_m prod_d sin(pi k_{m,d} x_d) on the unit box."""
    amps: np.ndarray    # float64 (m,)
    waves: np.ndarray   # int32 (m, dim)


def _morton_key(coords: Sequence[int]) -> int:
    key = 0
    for bit in range(16):
        for d, c in enumerate(coords):
            key |= ((c >> bit) & 1) << (bit * len(coords) + d)
    return key


def _child_offsets(dim: int) -> List[Tuple[int, ...]]:
    # Morton order: x fastest.
    out = []
    for k in range(1 << dim):
        out.append(tuple((k >> d) & 1 for d in range(dim)))
    return out


def random_refined_mesh(dim: int, base: int, max_depth: int, prob: float,
                        pmin: int, pmax: int, seed: int,
                        base_y: Optional[int] = None) -> MeshDesc:
    """Base grid of `base`^dim unit cells, refined at random (see module doc)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cell = 1 << max_depth
    counts = [base] * dim
    if base_y is not None:
        counts[1] = base_y
    base_cells = [tuple(c) for c in np.ndindex(*reversed(counts))]
    base_cells = [tuple(reversed(c)) for c in base_cells]
    base_cells.sort(key=_morton_key)
    kids = _child_offsets(dim)
    los: List[Tuple[int, ...]] = []
    sizes: List[int] = []

    def visit(lo: Tuple[int, ...], size: int, depth: int) -> None:
        split = False
        if depth < max_depth:
            split = bool(rng.random() < prob)
        if not split:
            los.append(lo)
            sizes.append(size)
            return
        half = size // 2
        for off in kids:
            visit(tuple(l + o * half for l, o in zip(lo, off)), half, depth + 1)

    for bc in base_cells:
        visit(tuple(c * cell for c in bc), cell, 0)
    n = len(sizes)
    p = rng.integers(pmin, pmax + 1, size=n).astype(np.int32)
    extent = tuple(c * cell for c in counts)
    return MeshDesc(dim=dim, lo=np.asarray(los, dtype=np.int32).reshape(n, dim),
                    size=np.asarray(sizes, dtype=np.int32), p=p,
                    extent=extent, lattice_h=1.0 / float(base * cell))


def base_parity_coeff(mesh: MeshDesc, base: int, values=(1.0, 20.0)) -> np.ndarray:
    """Coefficient of the random-refinement problem (Section 4.3): a takes the
    two values by the parity of the lexicographic number (x fastest) of the
    base cell that holds each leaf."""
    cell = mesh.extent[0] // base
    bc = mesh.lo // cell
    num = np.zeros(mesh.n_elems, dtype=np.int64)
    stride = 1
    for d in range(mesh.dim):
        num += bc[:, d].astype(np.int64) * stride
        stride *= mesh.extent[d] // cell
    return np.where(num % 2 == 0, values[0], values[1]).astype(np.float64)


def with_coeff(mesh: MeshDesc, coeff: np.ndarray) -> MeshDesc:
    return dataclasses.replace(mesh, coeff=np.asarray(coeff, dtype=np.float64))


def with_corners(mesh: MeshDesc, corners) -> MeshDesc:
    return dataclasses.replace(mesh, corners=np.asarray(corners, dtype=np.float64).reshape(4, 2))


# corner images of the unit square for the mapped workloads: a sheared
# parallelogram (affine map) and a general convex quadrilateral (bilinear)
PARALLELOGRAM = ((0.0, 0.0), (1.0, 0.0), (0.35, 0.9), (1.35, 0.9))
QUADRILATERAL = ((0.0, 0.0), (1.2, 0.1), (0.15, 0.95), (1.05, 1.25))


def lshape(mesh: MeshDesc) -> MeshDesc:
    """The leaves of a square lattice mesh outside its lower-left quarter: an
    L-shaped domain with the re-entrant corner at the lattice's centre (the
    extents must be even in base cells, so that no leaf straddles the hole)."""
    hx, hy = mesh.extent[0] // 2, mesh.extent[1] // 2
    x0, y0, s = mesh.lo[:, 0], mesh.lo[:, 1], mesh.size
    inside = (x0 + s <= hx) & (y0 + s <= hy)
    if np.any((x0 < hx) & (y0 < hy) & ~inside):
        raise ValueError("a leaf straddles the hole")
    keep = ~inside
    return dataclasses.replace(mesh, lo=mesh.lo[keep].copy(), size=mesh.size[keep].copy(), p=mesh.p[keep].copy(),
                               coeff=None if mesh.coeff is None else mesh.coeff[keep].copy())


def with_mapping(mesh: MeshDesc, mapping) -> MeshDesc:
    return dataclasses.replace(mesh, mapping=mapping)


class WavyMap:
    """A curved domain for the mapped-element workloads (problem geometry, an
    input like the mesh): x = X + ax L sin(pi Y / L), y = Y + ay L sin(pi X / L)
    on the lattice domain [0, L]^2.  Lattice lines become sine curves, so
    every element and every sub-face is curved and the left and bottom sides
    of the domain bulge."""

    def __init__(self, L: float = 1.0, ax: float = 0.06, ay: float = 0.04):
        self.L, self.ax, self.ay = float(L), float(ax), float(ay)

    def __call__(self, X: np.ndarray) -> np.ndarray:
        L = self.L
        return np.stack([X[:, 0] + self.ax * L * np.sin(np.pi * X[:, 1] / L),
                         X[:, 1] + self.ay * L * np.sin(np.pi * X[:, 0] / L)], axis=1)

    def jacobian(self, X: np.ndarray) -> np.ndarray:
        L = self.L
        J = np.zeros((len(X), 2, 2))
        J[:, 0, 0] = 1.0
        J[:, 0, 1] = self.ax * np.pi * np.cos(np.pi * X[:, 1] / L)
        J[:, 1, 0] = self.ay * np.pi * np.cos(np.pi * X[:, 0] / L)
        J[:, 1, 1] = 1.0
        return J


def uniform_mesh(dim: int, base: int, p: int) -> MeshDesc:
    """Conforming `base`^dim grid of unit squares/cubes with uniform degree p."""
    cells = [tuple(reversed(c)) for c in np.ndindex(*([base] * dim))]
    n = len(cells)
    return MeshDesc(dim=dim, lo=np.asarray(cells, dtype=np.int32).reshape(n, dim),
                    size=np.ones(n, dtype=np.int32), p=np.full(n, p, dtype=np.int32),
                    extent=tuple([base] * dim), lattice_h=1.0 / base)


def sine_rhs(dim: int, seed: int, n_modes: int = 4, kmax: int = 8) -> SineRHS:
    rng = np.random.Generator(np.random.PCG64(seed))
    amps = rng.standard_normal(n_modes)
    waves = rng.integers(1, kmax + 1, size=(n_modes, dim)).astype(np.int32)
    return SineRHS(amps=amps, waves=waves)


def random_vector(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n)


# ---------------------------------------------------------------- workloads

def config0() -> Tuple[MeshDesc, SineRHS]:
    """2D, 8x8 conforming squares, p = 2 (576 DOFs)."""
    return uniform_mesh(2, 8, 2), sine_rhs(2, 0)


def config1(seed: int = 0) -> Tuple[MeshDesc, SineRHS]:
    """2D hp-random: 32x32 base, prob 0.3, depth <= 3, p ~ U{1..6} (~1e5 DOFs)."""
    return random_refined_mesh(2, 32, 3, 0.3, 1, 6, seed), sine_rhs(2, seed)


def config1_coeff(seed: int = 0) -> Tuple[MeshDesc, SineRHS]:
    """The 2D hp-random workload with the coefficient a in {1, 20} of the
    random-refinement problem (by base-cell parity)."""
    mesh, rhs = config1(seed)
    return with_coeff(mesh, base_parity_coeff(mesh, 32)), rhs


def config1_mapped(seed: int = 0, corners=QUADRILATERAL) -> Tuple[MeshDesc, SineRHS]:
    """The 2D hp-random workload carried by the bilinear map of the unit
    square onto a general convex quadrilateral."""
    mesh, rhs = config1(seed)
    return with_corners(mesh, corners), rhs


def config1_curved(seed: int = 0) -> Tuple[MeshDesc, SineRHS]:
    """The 2D hp-random workload on the curved domain of WavyMap."""
    mesh, rhs = config1(seed)
    return with_mapping(mesh, WavyMap()), rhs


def config2(seed: int = 0, base: int = 16) -> Tuple[MeshDesc, SineRHS]:
    """3D hp-random: base^3 hexes, prob 0.2, depth <= 2, p ~ U{1..5}."""
    return random_refined_mesh(3, base, 2, 0.2, 1, 5, seed), sine_rhs(3, seed)


def config3_problem(k: int, dof_lo: int = 1000, dof_hi: int = 300000
                    ) -> Tuple[MeshDesc, SineRHS]:
    """Problem k of the batched workload: base N = round(exp U[ln 4, ln 64]),
    prob 0.3, depth <= 3, p ~ U{1..8}; redrawn until the DOFs fall in range."""
    rng = np.random.Generator(np.random.PCG64(1_000_003 + k))
    for attempt in range(1000):
        n = int(round(math.exp(rng.uniform(math.log(4), math.log(64)))))
        mesh = random_refined_mesh(2, n, 3, 0.3, 1, 8, seed=k * 1000 + attempt)
        if dof_lo <= mesh.n_dofs() <= dof_hi:
            return mesh, sine_rhs(2, k)
    raise RuntimeError("no mesh in the DOF range")


def small_hp_mesh(seed: int, base: int = 3, depth: int = 2, prob: float = 0.4,
                  pmin: int = 1, pmax: int = 4, dim: int = 2) -> MeshDesc:
    """Small irregular hp mesh for parity tests."""
    return random_refined_mesh(dim, base, depth, prob, pmin, pmax, seed)


def serving_meshes(m: int, seed: int = 0, dof_lo: float = 5e3, dof_hi: float = 2e6) -> List[MeshDesc]:
    """m distinct meshes for the served workload, alternately squares (prob
    0.3, depth <= 3) and cubes (prob 0.2, depth <= 2), p ~ U{1..6}, DOF targets
    log-uniform in [dof_lo, dof_hi]; the base grid is chosen from the expected
    DOFs per base cell (about 99 for squares, 605 for cubes)."""
    rng = np.random.Generator(np.random.PCG64(777 + seed))
    out = []
    for j in range(m):
        target = math.exp(rng.uniform(math.log(dof_lo), math.log(dof_hi)))
        if j % 2 == 1:
            base = max(1, int(round((target / 605.0) ** (1.0 / 3.0))))
            out.append(random_refined_mesh(3, base, 2, 0.2, 1, 6, seed=9000 + j))
        else:
            base = max(2, int(round(math.sqrt(target / 99.0))))
            out.append(random_refined_mesh(2, base, 3, 0.3, 1, 6, seed=9000 + j))
    return out
