"""Pins of the oracle's conforming prolongation and boundary-space
decomposition (Section 3.2, 3.3, 3.4)."""
import numpy as np
import pytest

from oracle import basis, solver
from oracle.space import E_NODE, I_NODE, J_NODE
from paper_2009_01287_gb300 import inputs


def jump_constraints(prob):
    """Rows: [[u]] at max(p)+1 Gauss points of every interior sub-face and the
    trace at those of every boundary sub-face (zero iff u in H^1_0)."""
    sp_ = prob.space
    rows = []
    for f in prob.topo.subfaces:
        sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
        q = max(int(prob.topo.p[k]) for k in sides) + 1
        pts, _, _ = sp_.face_quadrature(f, q)
        R = np.zeros((q, sp_.n))
        for si, k in enumerate(sides):
            v, _ = sp_.eval(k, pts)
            R[:, sp_.dofs(k)] += (1.0 if si == 0 else -1.0) * v
        rows.append(R)
    return np.concatenate(rows)


@pytest.mark.parametrize("seed,pmin,pmax,depth", [(0, 1, 4, 2), (1, 1, 5, 3), (2, 2, 3, 3), (5, 3, 3, 2)])
def test_range_of_P_is_H10_subspace(seed, pmin, pmax, depth):
    """range(P) = V_h cap H^1_0 (Section 3.4, natural injection), checked by
    SVD on arbitrarily irregular hp meshes (multi-level hanging chains)."""
    mesh = inputs.small_hp_mesh(seed, base=2, depth=depth, prob=0.5, pmin=pmin, pmax=pmax)
    prob = solver.build_problem(mesh)
    C = jump_constraints(prob)
    P = prob.cs.P.toarray()
    assert np.abs(C @ P).max() < 1e-11
    s = np.linalg.svd(C, compute_uv=False)
    null_dim = prob.space.n - int(np.sum(s > 1e-9 * s[0]))
    assert null_dim == P.shape[1]
    assert np.linalg.matrix_rank(P) == P.shape[1]


def test_P_is_identity_at_coincident_nodes():
    """A conforming basis function equals 1 at its own nodal point: on a
    conforming uniform-p mesh, P is a 0/1 matrix with one 1 per row off the
    boundary."""
    mesh = inputs.uniform_mesh(2, 3, 3)
    prob = solver.build_problem(mesh)
    P = prob.cs.P.toarray()
    assert set(np.unique(np.round(P, 12))) <= {0.0, 1.0}
    coords = np.concatenate([prob.space.node_coords(k) for k in range(prob.topo.n)])
    on_bdry = np.any((np.abs(coords) < 1e-12) | (np.abs(coords - 1) < 1e-12), axis=1)
    np.testing.assert_allclose(P.sum(axis=1), np.where(on_bdry, 0.0, 1.0), atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_boundary_space_decomposition(seed):
    """V_B = (+)_e V_e (+) V_J with disjoint V_e (Section 3.3): every node on
    an element boundary is J or in exactly one block, interior nodes in none,
    and two E nodes of different blocks never share a sub-face."""
    mesh = inputs.small_hp_mesh(seed, base=3, depth=3, prob=0.4, pmin=1, pmax=5)
    prob = solver.build_problem(mesh)
    cs = prob.cs
    owner = -np.ones(prob.space.n, dtype=np.int64)
    for bi, b in enumerate(cs.blocks):
        assert np.all(owner[b] < 0)
        owner[b] = bi
    for k in range(prob.topo.n):
        p = int(prob.topo.p[k])
        loc = cs.kind[prob.space.dofs(k)].reshape(p + 1, p + 1)
        assert np.all(loc[1:-1, 1:-1] == I_NODE)
        edge = np.ones((p + 1, p + 1), dtype=bool)
        edge[1:-1, 1:-1] = False
        assert np.all(loc[edge] != I_NODE)
    assert np.all((owner >= 0) == (cs.kind == E_NODE))
    # jump-overlap closure: E nodes on a common sub-face are in one block
    sp_ = prob.space
    for f in prob.topo.subfaces:
        sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
        pts, _, _ = sp_.face_quadrature(f, 3)
        members = set()
        for k in sides:
            v, _ = sp_.eval(k, pts)
            dofs = sp_.dofs(k)[np.abs(v).max(axis=0) > 1e-12]
            members |= {int(owner[d]) for d in dofs if cs.kind[d] == E_NODE}
        assert len(members) <= 1


def test_conforming_mesh_has_no_blocks():
    """Conforming mesh, uniform p: every boundary node is in V_J and the
    method reduces to LOR + point Jacobi (Section 4.1)."""
    mesh, _ = inputs.config0()
    prob = solver.build_problem(mesh, eta=10.0, penalty_form="p1sq")
    assert len(prob.cs.blocks) == 0
    assert prob.cs.P.shape[1] == 15 * 15
