"""Mesh topology of a 2D leaf-box mesh, computed by brute force (Section 2, 3.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Elements are axis-aligned squares on an integer lattice.  A side s of an
element is 0: left (x = x0), 1: right, 2: bottom (y = y0), 3: top.  On a side
the tangential coordinate t runs along the other axis, increasing.

Definitions (Section 3.2 and the hanging-node discussion before Lemma 7):
* sub-face: a maximal segment shared by one side of an element and the
  opposite side of a neighbour (interior), or a full side on the domain
  boundary;
* a vertex is hanging when it lies in the relative interior of a side of an
  element of which it is not a corner, regular otherwise;
* a master edge is a side that is not strictly contained in the opposite side
  of a neighbour (a conforming side is a master edge shared by two elements);
* an hp-vertex is a hanging vertex whose containing elements do not all have
  the same degree.
"""
from __future__ import annotations

import dataclasses
from collections import defaultdict
from typing import Dict, List, Optional, Tuple

import numpy as np

SIDE_AXIS = (0, 0, 1, 1)     # normal axis of each side
SIDE_SIGN = (-1, 1, -1, 1)   # outward normal sign


@dataclasses.dataclass
class SubFace:
    km: int                  # element on the minus side
    kp: int                  # element on the plus side, -1 on the boundary
    axis: int                # normal axis (0: x, 1: y)
    c: int                   # lattice coordinate of the line
    t0: int                  # tangential interval [t0, t1] (lattice)
    t1: int
    normal_sign: int         # +1: normal points in +axis direction from km


@dataclasses.dataclass
class MasterEdge:
    axis: int                # normal axis of the line carrying the edge
    c: int
    t0: int
    t1: int
    owners: List[int]        # elements whose side equals the edge
    slaves: List[int]        # elements whose side lies strictly inside
    boundary: bool
    p: int                   # min degree over owners and slaves
    hanging: List[Tuple[int, int]]  # hanging vertices in the edge interior


class Topology:
    def __init__(self, lo: np.ndarray, size: np.ndarray, p: np.ndarray,
                 extent: Tuple[int, int]):
        self.lo = np.asarray(lo, dtype=np.int64)
        self.size = np.asarray(size, dtype=np.int64)
        self.p = np.asarray(p, dtype=np.int64)
        self.extent = tuple(int(e) for e in extent)
        self.n = len(self.size)
        self._check_cover()
        self._build_sides()
        self._build_subfaces()
        self._build_vertices()
        self._build_masters()

    # ------------------------------------------------------------------
    def side_segment(self, k: int, s: int) -> Tuple[int, int, int, int]:
        """(axis, c, t0, t1) of side s of element k."""
        x0, y0 = int(self.lo[k, 0]), int(self.lo[k, 1])
        h = int(self.size[k])
        if s == 0:
            return 0, x0, y0, y0 + h
        if s == 1:
            return 0, x0 + h, y0, y0 + h
        if s == 2:
            return 1, y0, x0, x0 + h
        return 1, y0 + h, x0, x0 + h

    def corners(self, k: int) -> List[Tuple[int, int]]:
        x0, y0 = int(self.lo[k, 0]), int(self.lo[k, 1])
        h = int(self.size[k])
        return [(x0, y0), (x0 + h, y0), (x0, y0 + h), (x0 + h, y0 + h)]

    def _check_cover(self) -> None:
        """The domain is the union of the leaves: they may not overlap; lattice
        cells no leaf covers are holes (an L-shaped domain, say), whose edges
        are boundary like the lattice's own."""
        occ = np.zeros(self.extent[::-1], dtype=np.int32)
        for k in range(self.n):
            x0, y0 = self.lo[k]
            h = self.size[k]
            if x0 < 0 or y0 < 0 or x0 + h > self.extent[0] or y0 + h > self.extent[1]:
                raise ValueError("leaf outside the lattice")
            occ[y0:y0 + h, x0:x0 + h] += 1
        if np.any(occ > 1):
            raise ValueError("leaves overlap")
        self.covered = occ == 1

    def _build_sides(self) -> None:
        # line key (axis, c) -> list of (element, side, t0, t1)
        self.lines: Dict[Tuple[int, int], List[Tuple[int, int, int, int]]] = defaultdict(list)
        for k in range(self.n):
            for s in range(4):
                ax, c, t0, t1 = self.side_segment(k, s)
                self.lines[(ax, c)].append((k, s, t0, t1))

    def _build_subfaces(self) -> None:
        self.subfaces: List[SubFace] = []
        for (ax, c), items in sorted(self.lines.items()):
            minus = [it for it in items if it[1] in (1, 3)]   # right / top sides
            plus = [it for it in items if it[1] in (0, 2)]    # left / bottom sides
            for (km, sm, a0, a1) in minus:
                for (kp, sp, b0, b1) in plus:
                    t0, t1 = max(a0, b0), min(a1, b1)
                    if t1 > t0:
                        self.subfaces.append(SubFace(km, kp, ax, c, t0, t1, +1))
            # the parts of a side that no opposite side covers are boundary
            # (the lattice's edge, or the edge of a hole)
            for group, opp, sign in ((plus, minus, -1), (minus, plus, +1)):
                for (k, s, a0, a1) in group:
                    cov = sorted((max(a0, b0), min(a1, b1)) for (_, _, b0, b1) in opp if min(a1, b1) > max(a0, b0))
                    t = a0
                    for (u0, u1) in cov:
                        if u0 > t:
                            self.subfaces.append(SubFace(k, -1, ax, c, t, u0, sign))
                        t = max(t, u1)
                    if t < a1:
                        self.subfaces.append(SubFace(k, -1, ax, c, t, a1, sign))

    def _build_vertices(self) -> None:
        self.vertices = sorted({v for k in range(self.n) for v in self.corners(k)})
        self.vertex_elems: Dict[Tuple[int, int], List[int]] = defaultdict(list)
        for k in range(self.n):
            for v in self.corners(k):
                self.vertex_elems[v].append(k)

    def containing_side(self, v: Tuple[int, int]) -> Optional[Tuple[int, int]]:
        """(element, side) whose side contains v in its relative interior."""
        x, y = v
        for (k, s, t0, t1) in self.lines.get((0, x), []):
            if t0 < y < t1:
                return k, s
        for (k, s, t0, t1) in self.lines.get((1, y), []):
            if t0 < x < t1:
                return k, s
        return None

    def is_hanging(self, v: Tuple[int, int]) -> bool:
        return self.containing_side(v) is not None

    def on_boundary(self, v: Tuple[int, int]) -> bool:
        """A vertex of the domain boundary: one of the four lattice cells around
        it is outside the lattice or a hole."""
        x, y = v
        for cy in (y - 1, y):
            for cx in (x - 1, x):
                if not (0 <= cx < self.extent[0] and 0 <= cy < self.extent[1]) or not self.covered[cy, cx]:
                    return True
        return False

    def _build_masters(self) -> None:
        self.masters: Dict[Tuple[int, int, int, int], MasterEdge] = {}
        self.side_master: Dict[Tuple[int, int], Tuple[int, int, int, int]] = {}
        bnd: Dict[Tuple[int, int, int, int], bool] = {}
        for (ax, c), items in self.lines.items():
            for (k, s, t0, t1) in items:
                opp = [it for it in items if (it[1] in (0, 2)) != (s in (0, 2))]
                container = [it for it in opp if it[2] <= t0 and t1 <= it[3]
                             and (it[3] - it[2]) > (t1 - t0)]
                if container:
                    kk, ss, u0, u1 = container[0]
                    key = (ax, c, u0, u1)
                else:
                    key = (ax, c, t0, t1)
                    # a boundary edge: no element across it (lattice edge or hole)
                    bnd[key] = not any(min(t1, it[3]) > max(t0, it[2]) for it in opp)
                self.side_master[(k, s)] = key
        for (k, s), key in self.side_master.items():
            ax, c, t0, t1 = key
            if key not in self.masters:
                self.masters[key] = MasterEdge(ax, c, t0, t1, [], [], bnd[key], 10 ** 9, [])
            m = self.masters[key]
            seg = self.side_segment(k, s)
            if (seg[2], seg[3]) == (t0, t1):
                m.owners.append(k)
            else:
                m.slaves.append(k)
        on_line: Dict[Tuple[int, int], List[int]] = defaultdict(list)
        for v in self.vertices:
            on_line[(0, v[0])].append(v[1])
            on_line[(1, v[1])].append(v[0])
        for key, m in self.masters.items():
            m.p = int(min(self.p[k] for k in m.owners + m.slaves))
            for tan in sorted(on_line[(m.axis, m.c)]):
                if m.t0 < tan < m.t1:
                    m.hanging.append((m.c, tan) if m.axis == 0 else (tan, m.c))

    def faces_of(self, k: int) -> List[SubFace]:
        if not hasattr(self, "_faces_of"):
            self._faces_of = defaultdict(list)
            for f in self.subfaces:
                self._faces_of[f.km].append(f)
                if f.kp >= 0:
                    self._faces_of[f.kp].append(f)
        return self._faces_of[k]

    # ------------------------------------------------------------------
    def elements_containing(self, v: Tuple[int, int]) -> List[int]:
        x0, y0 = self.lo[:, 0], self.lo[:, 1]
        inside = ((x0 <= v[0]) & (v[0] <= x0 + self.size)
                  & (y0 <= v[1]) & (v[1] <= y0 + self.size))
        return [int(k) for k in np.nonzero(inside)[0]]

    def is_hp_vertex(self, v: Tuple[int, int]) -> bool:
        if not self.is_hanging(v):
            return False
        ps = {int(self.p[k]) for k in self.elements_containing(v)}
        return len(ps) > 1

    def master_of_vertex(self, v: Tuple[int, int]) -> Tuple[int, int, int, int]:
        k, s = self.containing_side(v)
        return self.side_master[(k, s)]
