"""Pins of the oracle's DG matrix (Section 2, Eq. fe-problem; BR2 of Section
4.4) against consistency, closed forms and a textbook continuous assembly."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis, dg, rhs, solver
from oracle.topology import Topology
from paper_2009_01287_gb300 import inputs


def _mesh(lo, size, p, extent, lh):
    return inputs.MeshDesc(2, np.asarray(lo, dtype=np.int32), np.asarray(size, dtype=np.int32),
                           np.asarray(p, dtype=np.int32), tuple(extent), lh)


U = lambda X: X[:, 0] * (1 - X[:, 0]) * X[:, 1] * (1 - X[:, 1])
F = lambda X: 2 * X[:, 1] * (1 - X[:, 1]) + 2 * X[:, 0] * (1 - X[:, 0])   # -Laplace(U)


@pytest.mark.parametrize("form", ["sipg", "br2"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_manufactured_q2_reproduced(form, seed):
    """A Q2 solution vanishing on the boundary lies in V_h (p >= 2) and both
    forms are consistent, so A u_I = (f, phi) exactly (hanging, variable p)."""
    mesh = inputs.small_hp_mesh(seed, base=3, depth=2, prob=0.5, pmin=2, pmax=5)
    prob = solver.build_problem(mesh, form=form)
    u = rhs.interpolate(prob.space, U)
    b = rhs.load_vector_fn(prob.space, F)
    assert np.abs(prob.A @ u - b).max() < 1e-11 * np.abs(b).max() * 100


@pytest.mark.parametrize("form", ["sipg", "br2"])
def test_symmetric_positive_definite(form):
    mesh = inputs.small_hp_mesh(3, base=3, depth=2, prob=0.5, pmin=1, pmax=4)
    prob = solver.build_problem(mesh, form=form)
    A = prob.A.toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_sipg_penalty_closed_form():
    """u = 1 on the left square of a 2x1 mesh, 0 on the right: gradients
    vanish, so a(u,u) = sum over faces of sigma |[[u]]|^2 |e|:
    interior face sigma_int * h + three boundary faces sigma_L * h."""
    h = 0.5
    for pl, pr in [(1, 1), (2, 3), (4, 2)]:
        mesh = _mesh([(0, 0), (1, 0)], [1, 1], [pl, pr], (2, 1), h)
        prob = solver.build_problem(mesh, form="sipg", eta=7.0)
        nl = (pl + 1) ** 2
        u = np.zeros(prob.space.n)
        u[:nl] = 1.0
        s_int = 7.0 * max(pl, pr) ** 2 / h
        s_bnd = 7.0 * pl ** 2 / h
        expect = s_int * h + 3 * s_bnd * h
        assert abs(u @ prob.A @ u - expect) < 1e-12 * expect


def test_br2_penalty_closed_form():
    """Same piecewise constant: the lifting energy of a unit jump on a side of
    a Q_p square equals the 1D inverse-trace constant (p+1)^2 (scale free in
    2D), with factor 1/4 on an interior face and 1 on a boundary face."""
    for pl, pr in [(1, 1), (2, 3), (5, 2)]:
        mesh = _mesh([(0, 0), (1, 0)], [1, 1], [pl, pr], (2, 1), 0.25)
        prob = solver.build_problem(mesh, form="br2", eta=3.0)
        u = np.zeros(prob.space.n)
        u[:(pl + 1) ** 2] = 1.0
        expect = 3.0 * (0.25 * ((pl + 1) ** 2 + (pr + 1) ** 2) + 3 * (pl + 1) ** 2)
        assert abs(u @ prob.A @ u - expect) < 1e-11 * expect


def _continuous_stiffness(n, p):
    """Textbook continuous Q_p stiffness on an n x n grid of [0,1]^2 (global
    nodes by position, Dirichlet nodes removed), from the 1D GLL matrices."""
    g = basis.gll_nodes(p)
    xg, wg = basis.gauss(p + 1)
    l, d = basis.lagrange(g, xg), basis.lagrange_deriv(g, xg)
    M1 = l.T @ (wg[:, None] * l)
    K1 = d.T @ (wg[:, None] * d)
    Ke = np.kron(M1, K1) + np.kron(K1, M1)      # local (iy, ix) ordering
    N = n * p + 1
    K = np.zeros((N * N, N * N))
    for ey in range(n):
        for ex in range(n):
            idx = [(ey * p + iy) * N + ex * p + ix for iy in range(p + 1) for ix in range(p + 1)]
            K[np.ix_(idx, idx)] += Ke
    inner = [j * N + i for j in range(1, N - 1) for i in range(1, N - 1)]
    return K[np.ix_(inner, inner)], N


@pytest.mark.parametrize("p", [1, 2, 3])
def test_conforming_restriction_is_textbook_fem(p):
    """On a conforming uniform mesh, P^T A P (A the SIPG matrix) is the
    standard continuous stiffness matrix (jumps vanish on V_C)."""
    n = 3
    mesh = inputs.uniform_mesh(2, n, p)
    prob = solver.build_problem(mesh, eta=50.0)
    P = prob.cs.P.toarray()
    Kc = P.T @ prob.A.toarray() @ P
    K, N = _continuous_stiffness(n, p)
    # match conforming DOFs to grid nodes by position
    coords = np.concatenate([prob.space.node_coords(k) for k in range(prob.topo.n)])
    gx = basis.gll_nodes(p)
    grid = np.unique(np.round([(e + gx[i]) / n for e in range(n) for i in range(p + 1)], 14))
    assert len(grid) == N
    perm = []
    for c in range(P.shape[1]):
        r = np.argmax(P[:, c])
        x, y = coords[r]
        i = int(np.argmin(np.abs(grid - x)))
        j = int(np.argmin(np.abs(grid - y)))
        perm.append((j - 1) * (N - 2) + (i - 1))
    Kp = K[np.ix_(perm, perm)]
    np.testing.assert_allclose(Kc, Kp, atol=1e-11 * np.abs(K).max())


def test_planted_mistake_fails_manufactured():
    """A dropped consistency term must break the manufactured-solution pin."""
    mesh = inputs.small_hp_mesh(0, base=3, depth=2, prob=0.5, pmin=2, pmax=4)
    prob = solver.build_problem(mesh)
    u = rhs.interpolate(prob.space, U)
    b = rhs.load_vector_fn(prob.space, F)
    Ahat = dg.assemble(prob.space, 100.0, broken_only=True)
    assert np.abs(Ahat @ u - b).max() > 1e-3 * np.abs(b).max()
