"""Sub-faces of a 3D leaf-box mesh (Section 2, read for hexahedra).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper states the method for quadrilaterals; in three dimensions the same
definitions hold with the faces of axis-aligned cubes: a sub-face is a maximal
rectangle shared by the upper face of one element and the lower face of a
neighbour (interior), or a full face on the domain boundary.  Nonconforming
neighbours meet on a rectangle that is the intersection of the two squares.

Elements are cubes on an integer lattice; the face of element k at
x_axis = lo[k, axis] (+ size[k]) is its lower (upper) face along that axis.
A sub-face stores its normal axis, the plane coordinate, the two tangential
axes in increasing order and the tangential rectangle [lo, hi] (lattice units).
Built with one occupancy map per plane, so it scales to the full 3D workload.
"""
from __future__ import annotations

import dataclasses
from collections import defaultdict
from typing import Dict, List, Tuple

import numpy as np


@dataclasses.dataclass
class SubFace3:
    km: int                  # element on the minus side (its upper face)
    kp: int                  # element on the plus side (its lower face), -1 on the boundary
    axis: int                # normal axis
    c: int                   # lattice coordinate of the plane
    ta: Tuple[int, int]      # tangential axes, increasing
    lo: Tuple[int, int]      # tangential rectangle, lattice units
    hi: Tuple[int, int]
    normal_sign: int         # +1: normal points in +axis direction from km


class Topology3:
    dim = 3

    def __init__(self, lo: np.ndarray, size: np.ndarray, p: np.ndarray,
                 extent: Tuple[int, int, int]):
        self.lo = np.asarray(lo, dtype=np.int64)
        self.size = np.asarray(size, dtype=np.int64)
        self.p = np.asarray(p, dtype=np.int64)
        self.extent = tuple(int(e) for e in extent)
        self.n = len(self.size)
        self._check_cover()
        self._build_subfaces()

    def _check_cover(self) -> None:
        vol = int(np.sum(self.size ** 3))
        if vol != self.extent[0] * self.extent[1] * self.extent[2]:
            raise ValueError("leaves do not tile the domain")
        occ = np.zeros(self.extent[::-1], dtype=np.int32)
        for k in range(self.n):
            x0, y0, z0 = self.lo[k]
            h = self.size[k]
            occ[z0:z0 + h, y0:y0 + h, x0:x0 + h] += 1
        if not np.all(occ == 1):
            raise ValueError("leaves overlap or leave gaps")

    def _build_subfaces(self) -> None:
        # plane (axis, c) -> elements with their lower / upper face on it
        lower: Dict[Tuple[int, int], List[int]] = defaultdict(list)
        upper: Dict[Tuple[int, int], List[int]] = defaultdict(list)
        for k in range(self.n):
            for ax in range(3):
                lower[(ax, int(self.lo[k, ax]))].append(k)
                upper[(ax, int(self.lo[k, ax] + self.size[k]))].append(k)
        self.subfaces: List[SubFace3] = []
        for (ax, c) in sorted(set(lower) | set(upper)):
            t = tuple(a for a in range(3) if a != ax)
            ext = (self.extent[t[0]], self.extent[t[1]])
            if 0 < c < self.extent[ax]:
                owner = np.full((ext[1], ext[0]), -1, dtype=np.int64)   # [u, t] lattice cell -> plus elem
                for k in lower[(ax, c)]:
                    a0, b0 = int(self.lo[k, t[0]]), int(self.lo[k, t[1]])
                    h = int(self.size[k])
                    owner[b0:b0 + h, a0:a0 + h] = k
                for km in upper[(ax, c)]:
                    a0, b0 = int(self.lo[km, t[0]]), int(self.lo[km, t[1]])
                    h = int(self.size[km])
                    for kp in np.unique(owner[b0:b0 + h, a0:a0 + h]):
                        kp = int(kp)
                        if kp < 0:
                            raise ValueError("face without neighbour inside the domain")
                        lo0 = max(a0, int(self.lo[kp, t[0]]))
                        lo1 = max(b0, int(self.lo[kp, t[1]]))
                        hi0 = min(a0 + h, int(self.lo[kp, t[0]] + self.size[kp]))
                        hi1 = min(b0 + h, int(self.lo[kp, t[1]] + self.size[kp]))
                        self.subfaces.append(SubFace3(km, kp, ax, c, t, (lo0, lo1), (hi0, hi1), +1))
            elif c == 0:
                for k in lower[(ax, c)]:
                    a0, b0 = int(self.lo[k, t[0]]), int(self.lo[k, t[1]])
                    h = int(self.size[k])
                    self.subfaces.append(SubFace3(k, -1, ax, c, t, (a0, b0), (a0 + h, b0 + h), -1))
            else:
                for k in upper[(ax, c)]:
                    a0, b0 = int(self.lo[k, t[0]]), int(self.lo[k, t[1]])
                    h = int(self.size[k])
                    self.subfaces.append(SubFace3(k, -1, ax, c, t, (a0, b0), (a0 + h, b0 + h), +1))

    def faces_of(self, k: int) -> List[SubFace3]:
        if not hasattr(self, "_faces_of"):
            self._faces_of = defaultdict(list)
            for f in self.subfaces:
                self._faces_of[f.km].append(f)
                if f.kp >= 0:
                    self._faces_of[f.kp].append(f)
        return self._faces_of[k]
