"""Pins of the oracle on domains with a hole (an L-shaped domain, the first
adaptive-refinement problem of Section 4.2): the hole's edges are boundary for
the DG form, the conforming space and the load vector."""
import numpy as np
import pytest

from oracle import rhs, solver
from paper_2009_01287_gb300 import inputs
from test_oracle_space import jump_constraints


def _lmesh(seed, pmin=1, pmax=4, depth=2):
    return inputs.lshape(inputs.small_hp_mesh(seed, base=4, depth=depth, prob=0.5, pmin=pmin, pmax=pmax))


def test_lshape_reproduces_polynomial_with_boundary_data():
    mesh = _lmesh(1, pmin=2)
    u = lambda x: 1.0 + x[:, 0] - 0.5 * x[:, 1] + x[:, 0] * x[:, 1] + 0.3 * x[:, 0] ** 2
    f = lambda x: np.full(len(x), -0.6)
    prob = solver.build_problem(mesh)
    b = rhs.dirichlet_load(prob.space, f, u, 100.0)
    x = np.linalg.solve(prob.A.toarray(), b)
    ui = rhs.interpolate(prob.space, u)
    assert np.abs(x - ui).max() <= 1e-10 * np.abs(ui).max()
    # the hole's two edges carry boundary sub-faces
    half = mesh.extent[0] // 2
    hole = [f for f in prob.topo.subfaces if f.kp < 0 and f.c == half and
            (f.t1 <= half)]
    assert len(hole) >= 2


@pytest.mark.parametrize("seed,pmin,pmax", [(0, 1, 3), (2, 2, 4)])
def test_lshape_range_of_P_is_H10(seed, pmin, pmax):
    prob = solver.build_problem(_lmesh(seed, pmin, pmax))
    C = jump_constraints(prob)
    P = prob.cs.P.toarray()
    assert np.abs(C @ P).max() < 1e-11
    s = np.linalg.svd(C, compute_uv=False)
    assert prob.space.n - int(np.sum(s > 1e-9 * s[0])) == P.shape[1]
    assert np.linalg.matrix_rank(P) == P.shape[1]


def test_lshape_spd_and_area():
    prob = solver.build_problem(_lmesh(3))
    A = prob.A.toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0
    b = rhs.load_vector_fn(prob.space, lambda x: np.ones(len(x)))
    assert abs(b.sum() - 0.75) <= 1e-13            # three quarters of the unit square


def test_straddling_leaf_refused():
    mesh = inputs.uniform_mesh(2, 1, 1)            # one leaf over the whole lattice
    mesh = inputs.MeshDesc(dim=2, lo=mesh.lo * 2, size=mesh.size * 2, p=mesh.p, extent=(2, 2), lattice_h=0.5)
    with pytest.raises(ValueError):
        inputs.lshape(mesh)
