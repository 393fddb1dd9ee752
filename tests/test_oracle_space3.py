"""Pins of the oracle's conforming prolongation and V_J / V_e split on cube
meshes (Section 3 read for hexahedra), of the 3D low-order-refined matrix,
and of the generic master-entity construction against the square-mesh one."""
import itertools

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import lor, solver
from oracle.space import E_NODE, I_NODE, J_NODE
from oracle.space3 import ConformingSpaceN
from paper_2009_01287_gb300 import inputs


def continuity_constraints(space):
    """Rows: [[u]] at (max p + 2)^2 Gauss points of every interior sub-face and
    the trace on every boundary sub-face (zero iff u in H^1_0)."""
    topo = space.topo
    rows = []
    for f in topo.subfaces:
        sides = [f.km] + ([f.kp] if f.kp >= 0 else [])
        q = max(int(topo.p[k]) for k in sides) + 2
        pts, _, _ = space.face_quadrature(f, q)
        R = np.zeros((len(pts), space.n))
        for si, k in enumerate(sides):
            v, _ = space.eval(k, pts)
            R[:, space.dofs(k)] += (1.0 if si == 0 else -1.0) * v
        rows.append(R)
    return np.vstack(rows)


MESHES = [
    ("h-only", lambda: inputs.small_hp_mesh(0, base=2, depth=2, prob=0.4, pmin=2, pmax=2, dim=3)),
    ("hp-a", lambda: inputs.small_hp_mesh(0, base=2, depth=1, prob=0.5, pmin=1, pmax=3, dim=3)),
    ("hp-b", lambda: inputs.small_hp_mesh(1, base=2, depth=2, prob=0.3, pmin=1, pmax=3, dim=3)),
    ("hp-c", lambda: inputs.small_hp_mesh(3, base=2, depth=2, prob=0.4, pmin=1, pmax=2, dim=3)),
]


@pytest.mark.parametrize("name,mk", MESHES, ids=[m[0] for m in MESHES])
def test_range_of_P_is_continuous_H10(name, mk):
    """range(P) = V_h cap H^1_0 by SVD on irregular hp cube meshes: P maps into
    continuous functions vanishing on the boundary, has full column rank, and
    its rank equals the dimension of the null space of the jump constraints."""
    prob = solver.build_problem(mk())
    C = continuity_constraints(prob.space)
    P = prob.cs.P.toarray()
    assert np.abs(C @ P).max() < 1e-11
    s = np.linalg.svd(C, compute_uv=False)
    null_dim = prob.space.n - int(np.sum(s > 1e-10 * s[0]))
    assert np.linalg.matrix_rank(P) == P.shape[1] == null_dim


def test_P_on_conforming_mesh_is_the_nodal_gather():
    """Conforming uniform cube mesh: P is a 0/1 matrix, and P P^T equals the
    node-coincidence matrix of the interior DG nodes (built from coordinates)."""
    mesh = inputs.uniform_mesh(3, 2, 2)
    prob = solver.build_problem(mesh)
    P = prob.cs.P.toarray()
    assert set(np.unique(np.round(P, 12))) <= {0.0, 1.0}
    X = np.concatenate([prob.space.node_coords(k) for k in range(prob.topo.n)])
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    same = np.all(np.abs(X[:, None, :] - X[None, :, :]) < 1e-12, axis=2) & inner[:, None] & inner[None, :]
    assert np.array_equal(P @ P.T, same.astype(float))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_generic_construction_equals_square_mesh_one(seed):
    """On squares the master-entity construction reproduces the 2D conforming
    space exactly: numbering, P, node classes and V_e blocks."""
    mesh = inputs.small_hp_mesh(seed, base=3, depth=3, prob=0.4, pmax=5)
    prob = solver.build_problem(mesh)
    g = ConformingSpaceN(prob.space)
    assert g.n == prob.cs.n
    assert abs(g.P - prob.cs.P).max() == 0.0
    assert np.array_equal(g.kind, prob.cs.kind)
    assert len(g.blocks) == len(prob.cs.blocks)
    assert all(np.array_equal(a, b) for a, b in zip(g.blocks, prob.cs.blocks))


@pytest.mark.parametrize("name,mk", MESHES[1:], ids=[m[0] for m in MESHES[1:]])
def test_boundary_space_decomposition3(name, mk):
    """V_B = (+)_e V_e (+) V_J: interior nodes are I, every element-boundary node
    is J or in exactly one block; the blocks are the E nodes of one master entity."""
    prob = solver.build_problem(mk())
    cs = prob.cs
    count = np.zeros(prob.space.n, dtype=int)
    for b in cs.blocks:
        count[b] += 1
        assert np.all(cs.kind[b] == E_NODE)
    assert np.array_equal(count, (cs.kind == E_NODE).astype(int))
    for k in range(prob.topo.n):
        p = int(prob.topo.p[k])
        base = int(prob.space.offset[k])
        for li, idx in enumerate(cs._local_nodes(k)):
            interior = all(0 < i < p for i in idx)
            assert (cs.kind[base + li] == I_NODE) == interior


def test_lor_q1_cell_closed_form():
    """Unit-cube Q1 stiffness: diagonal 1/3, edge neighbour 0, face-diagonal
    -1/12, body-diagonal -1/12; a box scales each axis term."""
    K = lor.q1_cell_stiffness3(1.0, 1.0, 1.0)
    assert np.allclose(np.diag(K), 1.0 / 3.0)
    assert abs(K[0, 1]) < 1e-15 and abs(K[0, 3] + 1.0 / 12.0) < 1e-15 and abs(K[0, 7] + 1.0 / 12.0) < 1e-15
    assert np.allclose(K.sum(axis=1), 0.0)
    # a x b x c box: the x-term of the diagonal is (b c / a) / 9, likewise y, z
    a, b, c = 2.0, 1.0, 0.5
    K2 = lor.q1_cell_stiffness3(a, b, c)
    assert np.isclose(K2[0, 0], (b * c / a + a * c / b + a * b / c) / 9.0, rtol=1e-14)


def test_lor_p1_equals_high_order():
    """For p = 1 the LOR sub-mesh is the element itself: the LOR element matrix
    equals the Q1 stiffness of the element."""
    from oracle import basis
    h = 0.5
    A = lor.lor_element(1, h, dim=3)
    g = basis.gll_nodes(1)
    xg, wg = basis.gauss(2)
    l, dl = basis.lagrange(g, xg), basis.lagrange_deriv(g, xg)
    M1, K1 = (l.T * wg) @ l, (dl.T * wg) @ dl
    ref = h * (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(K1, np.kron(M1, M1)))
    assert np.abs(A - ref).max() < 1e-14


def _kappa(prob, **kw):
    pc = solver.Preconditioner(prob, lor="exact", **kw)
    ev = sl.eigvals(pc.matrix() @ prob.A.toarray()).real
    return ev.max() / ev.min()


def test_kappa_blocks_versus_jacobi_over_eta_3d():
    """On hanging hp cube meshes the V_e blocks (the E nodes of each master
    entity; the growth to closure would join almost all E nodes into one block)
    keep kappa(BA) several times below point Jacobi on V_B at every penalty
    eta = 10 .. 10^4, and its growth in eta stays well below linear."""
    mesh = inputs.small_hp_mesh(1, base=2, depth=2, prob=0.3, pmin=1, pmax=3, dim=3)
    ks, kj = [], []
    for eta in (10.0, 1e3, 1e4):
        prob = solver.build_problem(mesh, eta=eta)
        ks.append(_kappa(prob))
        kj.append(_kappa(prob, smoother="jacobi_only"))
    assert all(a * 2.0 < b for a, b in zip(ks, kj))
    assert ks[-1] / ks[0] < 0.1 * 1e4 / 10.0


def test_kappa_conforming_3d_small():
    """Conforming uniform cube meshes: V_E is empty, B reduces to the LOR
    conforming solve plus point Jacobi, and kappa(BA) is small."""
    for p in (1, 2, 3):
        prob = solver.build_problem(inputs.uniform_mesh(3, 2, p))
        assert len(prob.cs.blocks) == 0
        assert _kappa(prob) < 60.0


def test_pcg_3d_reaches_direct_solution():
    """PCG with B (AMG V-cycle on the 3D LOR matrix) on a hanging hp cube mesh
    converges to the direct solution of A u = b."""
    import scipy.sparse.linalg as spla
    from oracle import rhs
    mesh = inputs.small_hp_mesh(0, base=2, depth=2, prob=0.3, pmin=1, pmax=3, dim=3)
    prob = solver.build_problem(mesh, form="br2")
    r = inputs.sine_rhs(3, 1)
    b = rhs.load_vector(prob.space, r.amps, r.waves)
    pc = solver.Preconditioner(prob, lor="amg")
    res = solver.pcg(prob.A, b, pc.apply, 1e-10, 1000)
    assert res.converged
    u = spla.spsolve(prob.A.tocsc(), b)
    assert np.abs(res.x - u).max() < 1e-7 * np.abs(u).max()
