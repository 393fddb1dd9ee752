"""Conforming prolongation and the boundary-space decomposition (Section 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conforming basis (Section 3.2.1, conforming nodal points): Lagrange basis at
* every regular vertex not on the boundary (V_C is read as V_h cap H^1_0,
  since the problem has homogeneous Dirichlet conditions),
* the interior Gauss-Lobatto points of degree p_S on every interior master
  edge S, p_S = the lowest degree of any element containing S (the rule for
  h-, p- and hp-interfaces),
* the interior Gauss-Lobatto points of every element.
A hanging vertex carries no unknown: its value is the value of the master edge
whose interior contains it (applied transitively).  P is the natural
injection V_C -> V_h (Section 3.4): column c holds the values of conforming
basis function c at every DG node.

Conforming numbering ("first touch"): walk the elements in order and their
nodes in local lexicographic order; an element-interior node gets the next
number; a corner gets its vertex's number if the vertex is regular, interior
and not yet numbered; an edge-interior node numbers all p_S - 1 interior nodes
of its master edge S, in increasing tangential coordinate, if not yet done.

Node classes (Section 3.3): I = element-interior node (handled by V_C only);
J = boundary-of-element node in V_J (point Jacobi); E = the rest of V_B.
V_J holds the nodes at regular vertices, and those on (or hanging in) a
master edge S that is conforming with equal degrees, or whose closed edge
contains no hp-vertex, or - with the remark on further cases enabled (off by
default) - whose coarse element has degree no higher than every fine element
along S.  V_e (Section 3.3, growth by jump overlap) are the
connected components of the E nodes under "the traces are both nonzero on a
common sub-face".
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from . import basis
from .dg import DGSpace

I_NODE, J_NODE, E_NODE = 0, 1, 2


def node_kind(p: int, ix: int, iy: int) -> str:
    bx = ix in (0, p)
    by = iy in (0, p)
    if bx and by:
        return "corner"
    if bx or by:
        return "edge"
    return "interior"


def node_side(p: int, ix: int, iy: int) -> int:
    """Side index of an edge-interior node."""
    if ix == 0:
        return 0
    if ix == p:
        return 1
    if iy == 0:
        return 2
    return 3


class ConformingSpace:
    def __init__(self, space: DGSpace, remark_cases: bool = False):
        self.space = space
        self.topo = space.topo
        self.remark_cases = remark_cases
        self._number()
        self._build_P()
        self._classify()

    # ------------------------------------------------------------------
    def _node_geom(self, k: int, ix: int, iy: int):
        t = self.topo
        p = int(t.p[k])
        x0, y0 = int(t.lo[k, 0]), int(t.lo[k, 1])
        h = int(t.size[k])
        return p, x0, y0, h

    def _number(self) -> None:
        t = self.topo
        self.vertex_dof: Dict[Tuple[int, int], int] = {}
        self.master_dofs: Dict[tuple, List[int]] = {}
        self.interior_dofs: Dict[Tuple[int, int, int], int] = {}
        n = 0
        for k in range(t.n):
            p = int(t.p[k])
            corners = t.corners(k)
            for iy in range(p + 1):
                for ix in range(p + 1):
                    kind = node_kind(p, ix, iy)
                    if kind == "interior":
                        self.interior_dofs[(k, ix, iy)] = n
                        n += 1
                    elif kind == "corner":
                        v = corners[(1 if ix == p else 0) + (2 if iy == p else 0)]
                        if (v not in self.vertex_dof and not t.on_boundary(v)
                                and not t.is_hanging(v)):
                            self.vertex_dof[v] = n
                            n += 1
                    else:
                        key = t.side_master[(k, node_side(p, ix, iy))]
                        if key not in self.master_dofs:
                            m = t.masters[key]
                            if m.boundary:
                                self.master_dofs[key] = []
                            else:
                                self.master_dofs[key] = list(range(n, n + m.p - 1))
                                n += m.p - 1
        self.n = n

    def vertex_value(self, v) -> Dict[int, float]:
        t = self.topo
        if t.on_boundary(v):
            return {}
        if v in self.vertex_dof:
            return {self.vertex_dof[v]: 1.0}
        key = t.master_of_vertex(v)
        m = t.masters[key]
        tan = v[1] if m.axis == 0 else v[0]
        return self.edge_value(key, tan)

    def edge_value(self, key, tan: float) -> Dict[int, float]:
        """Conforming function on master edge `key` at tangential lattice
        coordinate `tan`, as a combination of conforming DOFs."""
        t = self.topo
        m = t.masters[key]
        lam = (tan - m.t0) / float(m.t1 - m.t0)
        l = basis.lagrange(basis.gll_nodes(m.p), lam)[0]
        out: Dict[int, float] = {}

        def acc(d, w):
            for c, val in d.items():
                out[c] = out.get(c, 0.0) + w * val

        if m.axis == 0:
            va, vb = (m.c, m.t0), (m.c, m.t1)
        else:
            va, vb = (m.t0, m.c), (m.t1, m.c)
        if l[0] != 0.0:
            acc(self.vertex_value(va), l[0])
        if l[m.p] != 0.0:
            acc(self.vertex_value(vb), l[m.p])
        for j, c in enumerate(self.master_dofs.get(key, [])):
            out[c] = out.get(c, 0.0) + l[j + 1]
        return out

    def _build_P(self) -> None:
        t = self.topo
        rows, cols, vals = [], [], []
        for k in range(t.n):
            p = int(t.p[k])
            g = basis.gll_nodes(p)
            corners = t.corners(k)
            x0, y0 = int(t.lo[k, 0]), int(t.lo[k, 1])
            h = int(t.size[k])
            base = int(self.space.offset[k])
            for iy in range(p + 1):
                for ix in range(p + 1):
                    r = base + iy * (p + 1) + ix
                    kind = node_kind(p, ix, iy)
                    if kind == "interior":
                        d = {self.interior_dofs[(k, ix, iy)]: 1.0}
                    elif kind == "corner":
                        d = self.vertex_value(corners[(1 if ix == p else 0) + (2 if iy == p else 0)])
                    else:
                        s = node_side(p, ix, iy)
                        key = t.side_master[(k, s)]
                        tan = (y0 + h * g[iy]) if s in (0, 1) else (x0 + h * g[ix])
                        d = self.edge_value(key, tan)
                    for c, w in d.items():
                        if w != 0.0:
                            rows.append(r)
                            cols.append(c)
                            vals.append(w)
        self.P = sp.csr_matrix((vals, (rows, cols)), shape=(self.space.n, self.n))

    # ------------------------------------------------------------------
    def master_good(self, key) -> bool:
        """Nodes on (or hanging in) master edge S go to V_J when S is a
        conforming edge with equal degrees on both sides, or S contains no
        hp-vertex (the closed edge: its interior hanging vertices and its
        endpoints), or - remark on further cases - S's coarse element has
        degree no higher than every fine element along S."""
        t = self.topo
        m = t.masters[key]
        if len(m.owners) == 2 and int(t.p[m.owners[0]]) == int(t.p[m.owners[1]]):
            return True
        ends = [(m.c, m.t0), (m.c, m.t1)] if m.axis == 0 else [(m.t0, m.c), (m.t1, m.c)]
        if not any(t.is_hp_vertex(v) for v in m.hanging + ends):
            return True
        if self.remark_cases and m.slaves:
            pc = min(int(t.p[k]) for k in m.owners)
            if all(pc <= int(t.p[k]) for k in m.slaves):
                return True
        return False

    def _classify(self) -> None:
        t = self.topo
        kind = np.zeros(self.space.n, dtype=np.int8)
        for k in range(t.n):
            p = int(t.p[k])
            corners = t.corners(k)
            base = int(self.space.offset[k])
            for iy in range(p + 1):
                for ix in range(p + 1):
                    r = base + iy * (p + 1) + ix
                    nk = node_kind(p, ix, iy)
                    if nk == "interior":
                        kind[r] = I_NODE
                    elif nk == "corner":
                        v = corners[(1 if ix == p else 0) + (2 if iy == p else 0)]
                        if not t.is_hanging(v):
                            kind[r] = J_NODE
                        else:
                            kind[r] = J_NODE if self.master_good(t.master_of_vertex(v)) else E_NODE
                    else:
                        key = t.side_master[(k, node_side(p, ix, iy))]
                        kind[r] = J_NODE if self.master_good(key) else E_NODE
        self.kind = kind
        self._blocks()

    def _node_sides(self, k: int, ix: int, iy: int) -> List[int]:
        p = int(self.topo.p[k])
        out = []
        if ix == 0:
            out.append(0)
        if ix == p:
            out.append(1)
        if iy == 0:
            out.append(2)
        if iy == p:
            out.append(3)
        return out

    def _blocks(self) -> None:
        """Connected components of the E nodes (growth of Section 3.3)."""
        t = self.topo
        sp_ = self.space
        # sub-faces touching each (element, side)
        side_faces: Dict[Tuple[int, int], List[int]] = {}
        for fi, f in enumerate(t.subfaces):
            if f.axis == 0:
                sm = 1 if f.normal_sign > 0 else 0
                sp_side = 0
            else:
                sm = 3 if f.normal_sign > 0 else 2
                sp_side = 2
            side_faces.setdefault((f.km, sm), []).append(fi)
            if f.kp >= 0:
                side_faces.setdefault((f.kp, sp_side), []).append(fi)
        face_members: Dict[int, List[int]] = {}
        for k in range(t.n):
            p = int(t.p[k])
            base = int(sp_.offset[k])
            for iy in range(p + 1):
                for ix in range(p + 1):
                    r = base + iy * (p + 1) + ix
                    if self.kind[r] != E_NODE:
                        continue
                    for s in self._node_sides(k, ix, iy):
                        for fi in side_faces.get((k, s), []):
                            face_members.setdefault(fi, []).append(r)
        parent = {}

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for r in np.nonzero(self.kind == E_NODE)[0]:
            parent[int(r)] = int(r)
        for fi, mem in face_members.items():
            for a in mem[1:]:
                ra, rb = find(a), find(mem[0])
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
        comps: Dict[int, List[int]] = {}
        for r in sorted(parent):
            comps.setdefault(find(r), []).append(r)
        self.blocks = [np.asarray(v, dtype=np.int64) for _, v in sorted(comps.items())]
