"""Conforming prolongation and the V_J / V_e split on box meshes of any
dimension, built from master entities (Section 3, read for hexahedra).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper states Section 3 for quadrilaterals.  Here every closed element is
split into entities (vertices, edges, faces, the interior: the boxes obtained
by fixing each axis at the lower end, the upper end, or letting it span), and
the mesh skeleton is partitioned into MASTER entities: the master of an
element entity Z is the entity of largest dimension, then largest size, among
the entities of all elements whose relative interior contains the midpoint of
Z (a hanging vertex lies in the interior of a master edge or face, a hanging
face inside a larger face, a fine edge inside a coarse face).  On dyadic box
meshes relint(Z) lies inside relint(master(Z)).

Conforming space V_C = V_h cap H^1_0: on every master entity M not on the
boundary a tensor Lagrange polynomial of degree p_M at the Gauss-Lobatto
points of M (the "min rule": p_M = the lowest degree of the elements touching
relint(M), then lowered to the degree of every master entity whose boundary
contains an edge or face of M, so that the traces agree); its unknowns are the interior
grid points of M ((p_M - 1)^dim M; one for a vertex).  The value at a grid
point on the boundary of M is the value of the master entity containing that
point (transitively).  P holds the value of every conforming basis function at
every DG node.

Numbering ("first touch"): elements in order, nodes in local lexicographic
order; an element-interior node gets the next number; a node on element
entity Z numbers the unknowns of M = master(Z), lexicographically, when Z and
M have the same dimension and M is not yet numbered.  On squares this is the
numbering of the 2D construction.

V_J / V_e (Section 3.3, read for hexahedra): an element-boundary node is J when
it sits at a regular vertex, or when the master entity M containing it is an
interior entity with no slave and equal degrees on all its elements, or when
the closure of M contains no hp-vertex (a hanging vertex whose elements do not
all have the same degree).  The other boundary nodes are E; V_e are the
connected components of the E nodes under "both traces nonzero on a common
sub-face".
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from . import basis
from .dg import DGSpace
from .space import E_NODE, I_NODE, J_NODE

Box = Tuple[Tuple[int, ...], Tuple[int, ...]]


def box_dim(b: Box) -> int:
    return sum(1 for a, c in zip(*b) if c > a)


def box_size(b: Box) -> int:
    return max(c - a for a, c in zip(*b))


class ConformingSpaceN:
    def __init__(self, space: DGSpace, hp_closure: bool = True, ve_growth: bool = None,
                 remark_cases: bool = False):
        self.space = space
        self.remark_cases = remark_cases
        self.hp_closure = hp_closure
        self.ve_growth = (space.dim == 2) if ve_growth is None else ve_growth
        self.topo = space.topo
        t = self.topo
        self.dim = space.dim
        self.lo = np.asarray(t.lo, dtype=np.int64)
        self.hi = self.lo + np.asarray(t.size, dtype=np.int64)[:, None]
        self.ext = tuple(int(e) for e in t.extent)
        self._master_cache: Dict[Box, Box] = {}
        self._build_masters()
        self._number()
        self._build_P()
        self._classify()

    # ------------------------------------------------------------ geometry
    def elem_box(self, k: int) -> Box:
        return tuple(int(v) for v in self.lo[k]), tuple(int(v) for v in self.hi[k])

    def elem_entity(self, k: int, sel) -> Box:
        """sel[d] in {0: lower end, 1: span, 2: upper end}."""
        lo, hi = self.elem_box(k)
        a = tuple(lo[d] if s in (0, 1) else hi[d] for d, s in enumerate(sel))
        b = tuple(hi[d] if s in (1, 2) else lo[d] for d, s in enumerate(sel))
        return a, b

    def touching(self, m2) -> np.ndarray:
        """Elements whose closed box contains the point m2 / 2 (lattice units)."""
        m2 = np.asarray(m2)
        inside = np.all((2 * self.lo <= m2) & (m2 <= 2 * self.hi), axis=1)
        return np.nonzero(inside)[0]

    def entity_at(self, k: int, m2) -> Box:
        lo, hi = self.elem_box(k)
        sel = [0 if m2[d] == 2 * lo[d] else (2 if m2[d] == 2 * hi[d] else 1) for d in range(self.dim)]
        return self.elem_entity(k, sel)

    def master_of(self, z: Box) -> Box:
        if z in self._master_cache:
            return self._master_cache[z]
        m2 = tuple(a + b for a, b in zip(*z))
        best = None
        for k in self.touching(m2):
            c = self.entity_at(int(k), m2)
            key = (box_dim(c), box_size(c))
            if best is None or key > best[0]:
                best = (key, c)
        self._master_cache[z] = best[1]
        return best[1]

    def on_boundary(self, b: Box) -> bool:
        return any(b[0][d] == b[1][d] and b[0][d] in (0, self.ext[d]) for d in range(self.dim))

    def sub_boxes(self, b: Box) -> List[Box]:
        """Proper faces of the closed box b (every spanning axis fixed, freed or not)."""
        span = [d for d in range(self.dim) if b[1][d] > b[0][d]]
        out = []
        for choice in itertools.product((0, 1, 2), repeat=len(span)):
            if all(c == 1 for c in choice):
                continue
            lo, hi = list(b[0]), list(b[1])
            for d, c in zip(span, choice):
                if c == 0:
                    hi[d] = lo[d]
                elif c == 2:
                    lo[d] = hi[d]
            out.append((tuple(lo), tuple(hi)))
        return out

    # ------------------------------------------------------------ masters
    def _build_masters(self) -> None:
        t = self.topo
        self.elems_of: Dict[Box, List[int]] = {}
        self.owners: Dict[Box, List[int]] = {}
        self.slaved: Dict[Box, bool] = {}
        for k in range(t.n):
            for sel in itertools.product((0, 1, 2), repeat=self.dim):
                z = self.elem_entity(k, sel)
                m = self.master_of(z)
                self.elems_of.setdefault(m, []).append(k)
                if z != m:
                    self.slaved[m] = True
                else:
                    self.owners.setdefault(m, []).append(k)
        self.pdeg: Dict[Box, int] = {m: int(min(t.p[k] for k in ks)) for m, ks in self.elems_of.items()}
        changed = True
        while changed:
            changed = False
            for m in list(self.pdeg):
                if box_dim(m) == 0:
                    continue
                for z in self.sub_boxes(m):
                    if box_dim(z) == 0:
                        continue   # a point value puts no degree condition
                    mm = self.master_of(z)
                    if self.pdeg[mm] > self.pdeg[m]:
                        self.pdeg[mm] = self.pdeg[m]
                        changed = True

    # ------------------------------------------------------------ numbering
    def _node_entity(self, k: int, idx) -> Tuple[Box, tuple]:
        p = int(self.topo.p[k])
        sel = tuple(0 if i == 0 else (2 if i == p else 1) for i in idx)
        return self.elem_entity(k, sel), sel

    def _local_nodes(self, k: int):
        p = int(self.topo.p[k])
        for rev in itertools.product(range(p + 1), repeat=self.dim):
            yield tuple(reversed(rev))   # x fastest

    def _grid_interior(self, m: Box):
        """Interior grid multi-indices of master m (first spanning axis fastest)."""
        q = self.pdeg[m]
        nspan = box_dim(m)
        for rev in itertools.product(range(1, q), repeat=nspan):
            yield tuple(reversed(rev))

    def _number(self) -> None:
        t = self.topo
        self.interior_dofs: Dict[Tuple[int, tuple], int] = {}
        self.master_dofs: Dict[Box, Dict[tuple, int]] = {}
        n = 0
        for k in range(t.n):
            ebox = self.elem_box(k)
            for idx in self._local_nodes(k):
                z, _ = self._node_entity(k, idx)
                if z == ebox:
                    self.interior_dofs[(k, idx)] = n
                    n += 1
                    continue
                m = self.master_of(z)
                if box_dim(z) != box_dim(m) or m in self.master_dofs:
                    continue
                if self.on_boundary(m):
                    self.master_dofs[m] = {}
                    continue
                d = {}
                for g in self._grid_interior(m):
                    d[g] = n
                    n += 1
                self.master_dofs[m] = d
        self.n = n

    # ------------------------------------------------------------ P
    def value_at(self, m: Box, pos) -> Dict[int, float]:
        """Conforming function on master entity m at lattice position `pos`
        (a point of the closed box m), as a combination of unknowns."""
        if self.on_boundary(m):
            return {}
        span = [d for d in range(self.dim) if m[1][d] > m[0][d]]
        if not span:
            return {self.master_dofs[m][()]: 1.0}
        q = self.pdeg[m]
        g = basis.gll_nodes(q)
        ls = [basis.lagrange(g, (pos[d] - m[0][d]) / float(m[1][d] - m[0][d]))[0] for d in span]
        out: Dict[int, float] = {}
        for rev in itertools.product(range(q + 1), repeat=len(span)):
            gi = tuple(reversed(rev))
            w = 1.0
            for a, l in zip(gi, ls):
                w *= l[a]
            if w == 0.0:
                continue
            if all(0 < a < q for a in gi):
                c = self.master_dofs[m][gi]
                out[c] = out.get(c, 0.0) + w
                continue
            y = list(m[0])
            lo, hi = list(m[0]), list(m[1])
            for d, a in zip(span, gi):
                y[d] = m[0][d] + (m[1][d] - m[0][d]) * g[a]
                if a == 0:
                    hi[d] = lo[d]
                elif a == q:
                    lo[d] = hi[d]
            sub = self.master_of((tuple(lo), tuple(hi)))
            for c, v in self.value_at(sub, y).items():
                out[c] = out.get(c, 0.0) + w * v
        return out

    def _build_P(self) -> None:
        t = self.topo
        rows, cols, vals = [], [], []
        for k in range(t.n):
            p = int(t.p[k])
            g = basis.gll_nodes(p)
            h = int(t.size[k])
            ebox = self.elem_box(k)
            base = int(self.space.offset[k])
            for li, idx in enumerate(self._local_nodes(k)):
                z, _ = self._node_entity(k, idx)
                if z == ebox:
                    d = {self.interior_dofs[(k, idx)]: 1.0}
                else:
                    pos = [float(self.lo[k, a]) + h * g[idx[a]] for a in range(self.dim)]
                    d = self.value_at(self.master_of(z), pos)
                for c, w in d.items():
                    if w != 0.0:
                        rows.append(base + li)
                        cols.append(c)
                        vals.append(w)
        self.P = sp.csr_matrix((vals, (rows, cols)), shape=(self.space.n, self.n))

    # ------------------------------------------------------------ V_J / V_e
    def is_hp_vertex(self, v: Tuple[int, ...]) -> bool:
        vb = (tuple(v), tuple(v))
        if box_dim(self.master_of(vb)) == 0:
            return False
        ps = {int(self.topo.p[k]) for k in self.touching(tuple(2 * c for c in v))}
        return len(ps) > 1

    def master_good(self, m: Box) -> bool:
        ks = self.elems_of[m]
        if not self.on_boundary(m) and not self.slaved.get(m, False) and \
                len({int(self.topo.p[k]) for k in ks}) == 1:
            return True
        if self.remark_cases and self.slaved.get(m, False):
            own = self.owners.get(m, [])
            fine = [k for k in ks if k not in own]
            if own and max(int(self.topo.p[k]) for k in own) <= min(int(self.topo.p[k]) for k in fine):
                return True
        vs = self._vertices_in(m)
        if not self.hp_closure:   # relative interior of M only
            vs = [v for v in vs if all(m[0][d] < v[d] < m[1][d] for d in range(self.dim) if m[1][d] > m[0][d])]
        return not any(self.is_hp_vertex(v) for v in vs)

    def _vertices_in(self, m: Box) -> List[Tuple[int, ...]]:
        if not hasattr(self, "_corners"):
            cs = set()
            for k in range(self.topo.n):
                lo, hi = self.elem_box(k)
                for c in itertools.product(*[(lo[d], hi[d]) for d in range(self.dim)]):
                    cs.add(c)
            self._corners = np.array(sorted(cs), dtype=np.int64)
        lo, hi = np.array(m[0]), np.array(m[1])
        sel = np.all((self._corners >= lo) & (self._corners <= hi), axis=1)
        return [tuple(int(a) for a in c) for c in self._corners[sel]]

    def _classify(self) -> None:
        t = self.topo
        kind = np.zeros(self.space.n, dtype=np.int8)
        good: Dict[Box, bool] = {}
        for k in range(t.n):
            ebox = self.elem_box(k)
            base = int(self.space.offset[k])
            for li, idx in enumerate(self._local_nodes(k)):
                z, _ = self._node_entity(k, idx)
                if z == ebox:
                    kind[base + li] = I_NODE
                    continue
                m = self.master_of(z)
                if box_dim(m) == 0:
                    kind[base + li] = J_NODE
                    continue
                if m not in good:
                    good[m] = self.master_good(m)
                kind[base + li] = J_NODE if good[m] else E_NODE
        self.kind = kind
        self._blocks()

    def _blocks(self) -> None:
        """V_e: connected components of the E nodes under shared sub-faces
        (growth to closure); without growth, the E nodes of each master
        entity (the initial sets V_e^(0))."""
        t = self.topo
        if not self.ve_growth:
            groups: Dict[Box, List[int]] = {}
            for k in range(t.n):
                base = int(self.space.offset[k])
                for li, idx in enumerate(self._local_nodes(k)):
                    if self.kind[base + li] == E_NODE:
                        z, _ = self._node_entity(k, idx)
                        groups.setdefault(self.master_of(z), []).append(base + li)
            self.blocks = sorted((np.asarray(sorted(v), dtype=np.int64) for v in groups.values()),
                                 key=lambda b: int(b[0]))
            return
        side_faces: Dict[Tuple[int, int], List[int]] = {}
        for fi, f in enumerate(t.subfaces):
            ax = f.axis
            side_faces.setdefault((f.km, 2 * ax + (1 if f.normal_sign > 0 else 0)), []).append(fi)
            if f.kp >= 0:
                side_faces.setdefault((f.kp, 2 * ax), []).append(fi)
        members: Dict[int, List[int]] = {}
        for k in range(t.n):
            p = int(t.p[k])
            base = int(self.space.offset[k])
            for li, idx in enumerate(self._local_nodes(k)):
                r = base + li
                if self.kind[r] != E_NODE:
                    continue
                for d in range(self.dim):
                    for end, s in ((0, 2 * d), (p, 2 * d + 1)):
                        if idx[d] == end:
                            for fi in side_faces.get((k, s), []):
                                members.setdefault(fi, []).append(r)
        parent = {int(r): int(r) for r in np.nonzero(self.kind == E_NODE)[0]}

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for fi in sorted(members):
            mem = members[fi]
            for a in mem[1:]:
                ra, rb = find(a), find(mem[0])
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
        comps: Dict[int, List[int]] = {}
        for r in sorted(parent):
            comps.setdefault(find(r), []).append(r)
        self.blocks = [np.asarray(v, dtype=np.int64) for _, v in sorted(comps.items())]
